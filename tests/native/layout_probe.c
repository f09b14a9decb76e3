/* Prints the sizes and field offsets of the ABI structs, so the Python
 * binding's ctypes layouts can be checked against the C header. */
#include <stddef.h>
#include <stdio.h>
#include "../../include/knnjoin.h"
int main(void)
{
    printf("config %zu %zu %zu %zu %zu\n", sizeof(knnjoin_config), offsetof(knnjoin_config, width_mult),
           offsetof(knnjoin_config, hbm_budget_bytes), offsetof(knnjoin_config, workers),
           offsetof(knnjoin_config, large_first));
    printf("job %zu %zu\n", sizeof(knnjoin_job), offsetof(knnjoin_job, out_dist));
    printf("stats %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(knnjoin_stats),
           offsetof(knnjoin_stats, candidates), offsetof(knnjoin_stats, ms_index), offsetof(knnjoin_stats, ms_wall),
           offsetof(knnjoin_stats, ms_pass), offsetof(knnjoin_stats, pass_candidates),
           offsetof(knnjoin_stats, width_mult), offsetof(knnjoin_stats, chunks),
           offsetof(knnjoin_stats, buffer_entries));
    return 0;
}
