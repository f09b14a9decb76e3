// tail.cuh -- brute-force tail: the last few uncertified queries of a join
// against every point (paper Sec. 5.4: the remark that the final failing
// queries of its GPU-Only runs could be finished another way).
//
// A ring pass over the whole grid would give each group of up to 16 such
// queries a single warp that walks all n points; here the (query, point)
// pairs are spread over the whole GPU instead:
//   1. the exact K-th smallest FP32 filter value T of each query over all
//      points but itself, by a radix select on the value's bits: four rounds
//      of a 256-bin histogram of the pairs that match the prefix found so
//      far (k_tail_hist over (chunk, query) blocks, k_tail_select per query);
//   2. every point whose FP32 value lies in the band of T, T (1 + 2^-15) +
//      2^-120 (a superset of the exact top K, as in the scan), appended to
//      the query's list (k_tail_collect);
//   3. per query, one warp scores the list with the canonical exact distance,
//      sorts it by (D, original id) and writes the first K -- certified, since
//      every point was considered (k_tail_finish).  A list longer than
//      TAIL_CAP (massive ties) leaves the query for a whole-grid scan pass.
#pragma once
#include "common.cuh"
#include "dist32.cuh"
#include "exact.cuh"
#include "scan.cuh"

namespace knn {

constexpr int TAIL_CAP = 256;  // band entries one warp sorts (8 per lane)

struct TailArgs {
    const float *xsort;     // data coordinates in key order, padded rows
    const float *qxsort;    // query coordinates in query-key order, padded rows
    const uint32_t *perm;   // data key order -> original id
    const uint32_t *qperm;  // query key order -> original query row
    const uint32_t *list;   // [m] the tail's sorted query positions
    int m;
    int64_t n;
    int K;
    int self;               // 1: a query's own point is not its neighbour
    int fixed_ok, F;        // fixed-point frame of the exact distances
    uint32_t *prefix;       // [m] radix-select prefix (the K-th value's bits found so far)
    uint32_t *rank;         // [m] rank still sought within the prefix (1-based)
    uint32_t *hist;         // [m][256] histogram of the current round (zero before a round)
    uint32_t *cnt;          // [m] band entries found (zero before the collect)
    uint32_t *band;         // [m][TAIL_CAP] their data positions
    uint32_t *status;       // [nq] per sorted query position: 0 certified, 2 left for a scan pass
    int32_t *out_ids;
    double *out_dist;
    int64_t row0, out_rows;
    int sorted_rows;
};

// Row s of padded coordinates (pad_dim(DIM) floats per row).
template <int DIM>
__device__ __forceinline__ void tail_point(const float *__restrict__ xs, uint32_t s, float (&c)[DIM])
{
    const float *r = xs + (size_t)s * pad_dim(DIM);
#pragma unroll
    for (int k = 0; k < DIM; ++k) c[k] = __ldg(r + k);
}

template <int DIM>
__device__ __forceinline__ void tail_query(const TailArgs &t, int j, float (&q)[DIM], uint32_t &own)
{
    const uint32_t s = t.list[j];
    tail_point<DIM>(t.qxsort, s, q);
    own = t.self ? s : 0xffffffffu;
}

// Round `shift` (24, 16, 8, 0) of the radix select: block (c, j) counts, for
// query j, the points of chunk c whose FP32 value matches the prefix found
// so far, by the value's next 8 bits.
template <int DIM>
__global__ void k_tail_hist(const TailArgs t, int shift, int64_t chunk)
{
    __shared__ uint32_t h[256];
    const int j = blockIdx.y;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    float q[DIM];
    uint32_t own;
    tail_query<DIM>(t, j, q, own);
    const uint32_t pre = t.prefix[j];
    const uint32_t mask = shift >= 24 ? 0u : ~0u << (shift + 8);
    const int64_t b = (int64_t)blockIdx.x * chunk, e = min(t.n, b + chunk);
    for (int64_t p = b + threadIdx.x; p < e; p += blockDim.x) {
        if ((uint32_t)p == own) continue;
        float c[DIM];
        tail_point<DIM>(t.xsort, (uint32_t)p, c);
        const uint32_t v = __float_as_uint(dist2_f32<DIM>(q, c));
        if ((v & mask) == pre) atomicAdd(&h[(v >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&t.hist[(size_t)j * 256 + i], h[i]);
}

// One warp per query: the bin of this round holding the sought rank; the
// prefix gains its 8 bits and the rank drops by the counts below it; the
// histogram is cleared for the next round.
__global__ void k_tail_select(const TailArgs t, int shift)
{
    const int j = blockIdx.x, lane = threadIdx.x & 31;
    uint32_t *h = t.hist + (size_t)j * 256;
    uint32_t v[8], sum = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        v[e] = h[lane * 8 + e];
        sum += v[e];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    const uint32_t r = t.rank[j];
    const uint32_t hit = __ballot_sync(FULL, inc >= r);
    const int src = hit ? __ffs(hit) - 1 : 31;
    uint32_t digit = 0, below = 0;
    if (lane == src) {
        uint32_t run = inc - sum;
        bool found = false;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            if (!found && run + v[e] >= r) {
                digit = lane * 8 + e;
                below = run;
                found = true;
            }
            run += v[e];
        }
    }
    digit = __shfl_sync(FULL, digit, src);
    below = __shfl_sync(FULL, below, src);
    __syncwarp();
#pragma unroll
    for (int e = 0; e < 8; ++e) h[lane * 8 + e] = 0;
    if (lane == 0) {
        t.prefix[j] |= digit << shift;
        t.rank[j] = r - below;
    }
}

// Block (c, j): the points of chunk c in query j's band, appended to its
// list (positions past TAIL_CAP are counted, not stored).
template <int DIM>
__global__ void k_tail_collect(const TailArgs t, int64_t chunk)
{
    const int j = blockIdx.y;
    float q[DIM];
    uint32_t own;
    tail_query<DIM>(t, j, q, own);
    const float thr = band_thr(t.prefix[j]);
    const int64_t b = (int64_t)blockIdx.x * chunk, e = min(t.n, b + chunk);
    for (int64_t p = b + threadIdx.x; p < e; p += blockDim.x) {
        if ((uint32_t)p == own) continue;
        float c[DIM];
        tail_point<DIM>(t.xsort, (uint32_t)p, c);
        if (dist2_f32<DIM>(q, c) <= thr) {
            const uint32_t at = atomicAdd(&t.cnt[j], 1u);
            if (at < (uint32_t)TAIL_CAP) t.band[(size_t)j * TAIL_CAP + at] = (uint32_t)p;
        }
    }
}

// One warp per query: exact canonical distances of the band, sorted by
// (D, original id); the first K are the query's row.
template <int DIM>
__global__ void k_tail_finish(const TailArgs t)
{
    constexpr int E = TAIL_CAP / 32;
    const int j = blockIdx.x, lane = threadIdx.x & 31;
    const uint32_t s = t.list[j];
    const uint32_t c = t.cnt[j];
    // massive ties (or, should the band ever hold fewer than K, anything
    // amiss): a whole-grid scan pass takes the query
    if (c > (uint32_t)TAIL_CAP || c < (uint32_t)t.K) {
        if (lane == 0) t.status[s] = 2;
        return;
    }
    float q[DIM];
    tail_point<DIM>(t.qxsort, s, q);
    int32_t qi[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) qi[k] = t.fixed_ok ? to_fixed(q[k], t.F) : 0;
    uint64_t D[E];
    uint32_t I[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const uint32_t g = (uint32_t)(lane * E + e);
        D[e] = ~0ull;
        I[e] = ~0u;
        if (g < c) {
            const uint32_t p = t.band[(size_t)j * TAIL_CAP + g];
            float x[DIM];
            tail_point<DIM>(t.xsort, p, x);
            uint64_t bits = 0;
            bool done = false;
            if (t.fixed_ok) {
                int32_t xi[DIM];
#pragma unroll
                for (int k = 0; k < DIM; ++k) xi[k] = to_fixed(x[k], t.F);
                done = canon_d2_fixed<DIM>(qi, xi, t.F, bits);
            }
            if (!done) bits = canon_d2_fp64<DIM>(q, x);
            D[e] = bits;
            I[e] = t.perm[p];
        }
    }
    warp_bitonic<E>(D, I, lane);
    const int64_t rowq = (int64_t)(t.sorted_rows ? s : t.qperm[s]) - t.row0;
    const bool rowin = rowq >= 0 && rowq < t.out_rows;
    const int64_t row = rowq * t.K;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int g = lane * E + e;
        if (g < t.K && rowin) {
            t.out_ids[row + g] = (int32_t)I[e];
            t.out_dist[row + g] = __longlong_as_double((long long)D[e]);  // D; k_sqrt_rows converts
        }
    }
    if (lane == 0) t.status[s] = 0;
}

}  // namespace knn
