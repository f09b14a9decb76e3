// knnjoin.cu -- host orchestration and the C ABI (include/knnjoin.h).
//
// A join runs on one CUDA stream:
//   a1 k_prep (data, and queries for R x S) -> a2 k_eps_pairs, k_eps_rows,
//   k_eps_hist x2, k_eps_count (parameter stages 0-2 inside them), k_params
//   -> a3 k_keys -> a4 radix sort -> a5 k_gather -> pass loop { level cell
//   tables (dense or hash map), groups of the active queries, density order,
//   work items, a7-a11 k_scan2 (k_scan for buffer overflows), compaction of
//   the uncertified queries; the last few by the brute-force tail of
//   tail.cuh } until no query is left -> k_sqrt_rows -> result copy to the
//   host if the outputs live there.
// The pass loop is the device re-queue of Alg. 1 (failed queries go back to
// the queue); each pass scans a ring of cells twice as wide as the last.
// Variants on the same loop: R x S (queries with their own keys and order),
// the paper's policy (epochs of one pass on a re-indexed grid, capped
// certificate), chunked output (one pass loop per chunk of query rows).
// Around it: the context, the worker pool for batched and served joins, the
// autotuner's table, and the allocation-free entry point.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <tuple>
#include <memory>
#include <mutex>
#include <set>
#include <stdexcept>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/knnjoin.h"
#include "common.cuh"
#include "grid.cuh"
#include "primitives.cuh"
#include "scan.cuh"
#include "scan2_launch.h"
#include "diag.cuh"
#include "tail.cuh"

using namespace knn;

namespace {

struct KnnError {
    knnjoin_status st;
    std::string msg;
};

[[noreturn]] void fail(knnjoin_status st, const std::string &msg) { throw KnnError{st, msg}; }

void ck(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) fail(KNN_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call) ck((call), #call)

int grid_for(int64_t n, int threads, int nsm, int per_sm = 8)
{
    int64_t b = (n + threads - 1) / threads;
    int64_t cap = (int64_t)nsm * per_sm;
    return (int)std::max<int64_t>(1, std::min(b, cap));
}

// ---------------------------------------------------------------------------
// Scratch memory: named device buffers that grow and are reused across joins.
// ---------------------------------------------------------------------------
struct Allocator {
    void *(*alloc)(size_t, void *) = nullptr;
    void (*free)(void *, void *) = nullptr;
    void *user = nullptr;
    // without hooks: a stream-ordered pool owned by the context (allocation
    // and release are ordered on the pipeline's stream and never synchronise
    // the device, so pipelines of the worker pool do not stall each other)
    cudaMemPool_t pool = nullptr;
    // message of a NULL from the hook (null: the generic one)
    const char *nomem_msg = nullptr;
    void *get(size_t bytes, cudaStream_t s)
    {
        void *p = nullptr;
        if (alloc) {
            p = alloc(bytes, user);
            if (!p)
                fail(KNN_ERR_NOMEM, nomem_msg ? std::string(nomem_msg)
                                              : "allocator hook returned NULL for " + std::to_string(bytes) + " bytes");
            if ((uintptr_t)p & 15) {  // kernels read scratch with 16-byte vector loads
                if (free) free(p, user);
                fail(KNN_ERR_INVALID, "allocator hook returned a pointer not aligned to 16 bytes");
            }
            return p;
        }
        cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMalloc(&p, bytes);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            fail(KNN_ERR_NOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
        }
        ck(e, "device allocation");
        return p;
    }
    void put(void *p, cudaStream_t s)
    {
        if (!p) return;
        if (free) free(p, user);
        else if (pool) cudaFreeAsync(p, s);
        else cudaFree(p);
    }
};

struct Scratch {
    Allocator *al = nullptr;
    cudaStream_t stream = nullptr;
    struct Buf {
        void *p = nullptr;
        size_t cap = 0;
    };
    std::map<std::string, Buf> bufs;
    template <class T>
    T *get(const std::string &name, size_t count)
    {
        size_t bytes = std::max<size_t>(count * sizeof(T), 256);
        Buf &b = bufs[name];
        if (b.cap < bytes) {
            al->put(b.p, stream);
            b.p = nullptr;
            b.cap = 0;
            size_t nb = std::max(bytes, b.cap + b.cap / 4);
            b.p = al->get(nb, stream);
            b.cap = nb;
        }
        return (T *)b.p;
    }
    void release()
    {
        for (auto &kv : bufs) al->put(kv.second.p, stream);
        bufs.clear();
    }
};

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Where a caller's buffer lives for a join on GPU `dev`: false for host
// memory (pageable or pinned), true for memory that GPU reads and writes as
// its own (its device memory, or managed memory).  Device memory of another
// GPU is an argument error: kernels on `dev` would access a peer's memory
// (a fault without peer access, a stray peer write with it).
bool device_side(const void *p, int dev, const char *what)
{
    cudaPointerAttributes at;
    if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    if (at.type != cudaMemoryTypeDevice) return false;
    if (at.device != dev)
        fail(KNN_ERR_INVALID, std::string(what) + " is device memory of GPU " + std::to_string(at.device) +
                                  ", not of GPU " + std::to_string(dev) + " that runs the join");
    return true;
}

// Named NVTX range for the lifetime of the object (tracing with nsys/ncu;
// no-ops without a tool attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// ---------------------------------------------------------------------------
// Autotuned cell-width multipliers, keyed by (d, K, floor(log2 n)), shared by
// a context's pipelines and kept in an optional JSON file.  The multiplier
// only changes speed: results are identical for every value.
// ---------------------------------------------------------------------------
struct TuneTable {
    std::mutex mu;
    std::map<std::tuple<int, int, int>, float> wm;
    std::map<std::tuple<int, int, int>, int> buf;  // tuned candidate-buffer entries / 32 (E), if any
    std::string path;
    float fixed = 0.0f;     // the caller's width_mult (> 0 overrides tuning)
    float dflt = 1.25f;

    static int nlog2(int64_t n)
    {
        int b = 0;
        while (b < 62 && ((int64_t)1 << (b + 1)) <= n) ++b;
        return b;
    }
    float lookup(int d, int K, int64_t n)
    {
        if (fixed > 0.0f) return fixed;
        std::lock_guard<std::mutex> lk(mu);
        auto it = wm.find(std::make_tuple(d, K, nlog2(n)));
        return it == wm.end() ? dflt : it->second;
    }
    // tuned buffer size E for (d, K, n), 0 = the default (the smallest holding K + 32)
    int lookup_E(int d, int K, int64_t n)
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = buf.find(std::make_tuple(d, K, nlog2(n)));
        return it == buf.end() ? 0 : it->second;
    }
    void set(int d, int K, int64_t n, float v, int E = 0)
    {
        std::lock_guard<std::mutex> lk(mu);
        wm[std::make_tuple(d, K, nlog2(n))] = v;
        if (E > 0) buf[std::make_tuple(d, K, nlog2(n))] = E;
        save_locked();
    }
    // {"knnjoin_tune": 1, "entries": [{"d": 2, "K": 32, "nlog2": 20, "width_mult": 1.125, "buffer": 2}, ...]}
    void load()
    {
        if (path.empty()) return;
        FILE *f = fopen(path.c_str(), "r");
        if (!f) return;
        std::string text;
        char chunk[4096];
        size_t nread;
        while ((nread = fread(chunk, 1, sizeof(chunk), f)) > 0) text.append(chunk, nread);
        fclose(f);
        std::lock_guard<std::mutex> lk(mu);
        for (size_t at = text.find("{\"d\":"); at != std::string::npos; at = text.find("{\"d\":", at + 1)) {
            int d = 0, K = 0, nl = 0;
            float v = 0.0f;
            int E = 0;
            const int got = sscanf(text.c_str() + at, "{\"d\": %d, \"K\": %d, \"nlog2\": %d, \"width_mult\": %f, "
                                   "\"buffer\": %d", &d, &K, &nl, &v, &E);
            if (got >= 4 && v > 0.0f && v < 16.0f) wm[std::make_tuple(d, K, nl)] = v;
            if (got == 5 && (E == 2 || E == 4 || E == 8)) buf[std::make_tuple(d, K, nl)] = E;
        }
    }
    void save_locked()
    {
        if (path.empty()) return;
        FILE *f = fopen(path.c_str(), "w");
        if (!f) return;
        fprintf(f, "{\"knnjoin_tune\": 1, \"entries\": [");
        bool first = true;
        for (auto &e : wm) {
            auto b = buf.find(e.first);
            fprintf(f, "%s\n {\"d\": %d, \"K\": %d, \"nlog2\": %d, \"width_mult\": %.6g, \"buffer\": %d}",
                    first ? "" : ",", std::get<0>(e.first), std::get<1>(e.first), std::get<2>(e.first), e.second,
                    b == buf.end() ? 0 : b->second);
            first = false;
        }
        fprintf(f, "\n]}\n");
        fclose(f);
    }
};

// ---------------------------------------------------------------------------
// One join pipeline (stream + scratch + pinned readback).
// ---------------------------------------------------------------------------
// Hash map from the cell keys of one grid level to their runs of points.
// Brute-force tail (tail.cuh) for dimension DIM: four radix-select rounds,
// the band collection and the per-query finish, on stream s.
template <int DIM>
void tail_launch_dim(const TailArgs &t, int64_t chunk, unsigned chunks, cudaStream_t s, int64_t &launches)
{
    const dim3 g(chunks, (unsigned)t.m);
    for (int shift = 24; shift >= 0; shift -= 8) {
        k_tail_hist<DIM><<<g, 256, 0, s>>>(t, shift, chunk); ++launches;
        k_tail_select<<<t.m, 32, 0, s>>>(t, shift); ++launches;
    }
    k_tail_collect<DIM><<<g, 256, 0, s>>>(t, chunk); ++launches;
    k_tail_finish<DIM><<<t.m, 32, 0, s>>>(t); ++launches;
}

void tail_launch(int d, const TailArgs &t, int64_t chunk, unsigned chunks, cudaStream_t s, int64_t &launches)
{
    switch (d) {
    case 1: tail_launch_dim<1>(t, chunk, chunks, s, launches); break;
    case 2: tail_launch_dim<2>(t, chunk, chunks, s, launches); break;
    case 3: tail_launch_dim<3>(t, chunk, chunks, s, launches); break;
    case 4: tail_launch_dim<4>(t, chunk, chunks, s, launches); break;
    case 5: tail_launch_dim<5>(t, chunk, chunks, s, launches); break;
    case 6: tail_launch_dim<6>(t, chunk, chunks, s, launches); break;
    case 7: tail_launch_dim<7>(t, chunk, chunks, s, launches); break;
    default: tail_launch_dim<8>(t, chunk, chunks, s, launches); break;
    }
}

// A tail of m queries against n points goes to the brute force when
// m * n is at most this (about 3.4 10^8 distance evaluations over its five
// sweeps of the pairs, a fraction of a millisecond); larger tails take a
// whole-grid scan pass.
constexpr double TAIL_BF_PAIRS = (double)(1 << 26);

struct LevelTab {
    uint4 *slot = nullptr;
    uint32_t mask = 0;
    bool built = false;
    uint2 *dense = nullptr;  // dense cell table (small grids) instead of the hash map
};

struct Pipeline {
    int device = 0;
    int nsm = 148;
    cudaStream_t s = nullptr;
    Scratch sc;
    uint32_t *pinned = nullptr;      // small host readback area (4 KB)
    // word offset in `pinned` of the staging copy of the levels' cell tables
    static constexpr int LEVELS_STAGING_WORD = 512;
    uint32_t *pinned_dev = nullptr;  // its device mapping (null: copy engine readbacks)
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    knnjoin_stats stats{};
    float width_mult = 1.25f;      // used when no tune table is attached
    TuneTable *tune = nullptr;
    float force_wm = 0.0f;         // > 0: this multiplier (autotuning runs)
    int force_E = 0;               // > 0: this buffer size (autotuning runs)
    int policy = 0;                // knnjoin_config.policy
    int tail_queries = 0;          // knnjoin_config.tail_queries
    size_t out_chunk_bytes = 0;    // knnjoin_config.out_chunk_mb (0: automatic)
    int64_t launches = 0;
    cudaEvent_t evs[2] = {nullptr, nullptr};
    cudaEvent_t uev = nullptr;  // this join's work up to a union scan (batch_union)
    // worker pipelines: a join with at least BIG_JOB_ENTRIES output entries
    // and host outputs holds this token from its first pass until its kernels
    // end and releases it before copying its results to the host, so such
    // joins take turns on the SMs for their scans, and one join's copy (and
    // the next one's point upload and index build) overlap another's scan
    std::mutex *big_token = nullptr;
    static constexpr int64_t BIG_JOB_ENTRIES = (int64_t)1 << 25;
    // resident index (knnjoin_index_*): res_mode 1 makes run() index the
    // data and keep it -- sorted keys, permutation, gathered coordinates,
    // parameters and, as they are built, the level hash maps; res_mode 2
    // makes run() answer R x S queries against what was kept
    int res_mode = 0;
    // cost-balanced shards: run() computes sorted query positions [row_b,
    // row_e) (output row = position - row_b) and writes the original row of
    // each output row to shard_rows_out (int64, host or device)
    bool shard_sorted = false;
    int64_t *shard_rows_out = nullptr;
    // diagnostic (knnjoin_work_queue): the first pass's work queue, as the
    // cell count of each query in queue order
    std::vector<int64_t> *queue_out = nullptr;
    // batched joins scanned together: the scan of each pass goes through this
    // coordinator (one launch over the work items of every join of the batch)
    struct UnionScan *uscan = nullptr;
    uint64_t *res_keys = nullptr;
    uint32_t *res_perm = nullptr;
    float *res_xsort = nullptr;
    GridParams res_hp{};
    float res_wm = 0.0f;
    LevelTab res_tabs[MAX_LEVELS];

    void init(int dev, cudaStream_t stream, Allocator *al)
    {
        device = dev;
        s = stream;
        sc.al = al;
        sc.stream = stream;
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        // readbacks go through mapped host memory written by a one-warp
        // kernel, so they never queue behind a large result copy of another
        // join on the copy engines
        CK(cudaHostAlloc(&pinned, 4096, cudaHostAllocMapped));
        CK(cudaHostGetDevicePointer((void **)&pinned_dev, pinned, 0));
        for (auto &e : ev) CK(cudaEventCreate(&e));
        for (auto &e : evs) CK(cudaEventCreate(&e));
        CK(cudaEventCreateWithFlags(&uev, cudaEventDisableTiming));
    }
    void release()
    {
        sc.release();
        if (pinned) cudaFreeHost(pinned);
        pinned = nullptr;
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        for (auto &e : evs)
            if (e) cudaEventDestroy(e);
        if (uev) cudaEventDestroy(uev);
        uev = nullptr;
    }

    // run later joins on stream t (waits for this pipeline's work so far)
    void set_stream(cudaStream_t t)
    {
        if (t == s) return;
        CK(cudaStreamSynchronize(s));
        s = t;
        sc.stream = t;
    }

    // copy `bytes` (a multiple of 4) from device memory to host_dst, a
    // position in `pinned`; complete once the stream is synchronised
    void fetch(uint32_t *host_dst, const void *src, size_t bytes)
    {
        if (pinned_dev) {
            k_fetch<<<1, 32, 0, s>>>(pinned_dev + (host_dst - pinned), (const uint32_t *)src, (int)(bytes / 4));
            ++launches;
        } else {
            CK(cudaMemcpyAsync(host_dst, src, bytes, cudaMemcpyDeviceToHost, s));
        }
    }

    // *a + *b (both device words), read back once this stream has synchronised
    int64_t read_total(const uint32_t *a, const uint32_t *b)
    {
        if (pinned_dev) {
            k_fetch_sum2<<<1, 32, 0, s>>>(pinned_dev, a, b);
            ++launches;
            CK(cudaStreamSynchronize(s));
            return (int64_t)pinned[0];
        }
        fetch(pinned, a, 4);
        fetch(pinned + 1, b, 4);
        CK(cudaStreamSynchronize(s));
        return (int64_t)pinned[0] + pinned[1];
    }

    template <class T>
    T read1(const T *dev)
    {
        static_assert(sizeof(T) % 4 == 0, "readback size");
        fetch(pinned, dev, sizeof(T));
        CK(cudaStreamSynchronize(s));
        T v;
        memcpy(&v, pinned, sizeof(T));
        return v;
    }

    // exclusive scan of m uint32 values (in may equal out)
    void scan(const uint32_t *in, uint32_t *out, int64_t m, int depth = 0)
    {
        if (m <= 0) return;
        int64_t nb = (m + SCAN_TILE - 1) / SCAN_TILE;
        uint32_t *sums = sc.get<uint32_t>("scan_sums" + std::to_string(depth), (size_t)nb + 1);
        k_scan_tiles<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, sums, m); ++launches;
        if (nb > 1 && nb <= SCAN_TILE) {
            // each tile adds the sum of the tiles before it, formed in place
            k_scan_add_direct<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(out, sums, m); ++launches;
        } else if (nb > 1) {
            scan(sums, sums, nb, depth + 1);
            k_scan_add<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(out, sums, m); ++launches;
        }
    }

    // a5: the cell table of level L over the n sorted keys -- the runs of
    // equal key >> d L, each cell's [begin, end) of sorted positions.  A
    // level whose grid has at most max(2n, 2^16) cells gets a dense table
    // (one load per neighbour lookup, no host readback here), any other a
    // hash map of 16-byte slots.  flags, rid, cbegin: n-entry scratch;
    // small[0] receives the cell count.
    LevelTab cell_table(const uint64_t *keys, int64_t n, int d, int L, const GridParams &hp, uint32_t *flags,
                        uint32_t *rid, uint32_t *cbegin, uint32_t *small)
    {
        const int shift = d * L;
        k_run_flags<<<grid_for(n, 256, nsm), 256, 0, s>>>(keys, nullptr, n, shift, flags); ++launches;
        scan(flags, rid, n);
        k_run_begin<<<grid_for(n, 256, nsm), 256, 0, s>>>(flags, rid, n, cbegin, small + 0); ++launches;
        DenseDims dd{};
        double G = 1.0;
        for (int k = 0; k < d; ++k) {
            dd.stride[k] = (uint32_t)G;
            G *= (double)((hp.cmax0[k] >> L) + 1);
        }
        if (G <= std::max(2.0 * (double)n, 65536.0)) {
            uint2 *tab = sc.get<uint2>("dense" + std::to_string(L), (size_t)G);
            CK(cudaMemsetAsync(tab, 0, sizeof(uint2) * (size_t)G, s));
            k_dense_insert<<<grid_for(n, 256, nsm), 256, 0, s>>>(keys, cbegin, small + 0, shift, d, hp.bits - L, dd,
                                                                  tab); ++launches;
            return {nullptr, 0, true, tab};
        }
        uint32_t ncells = read1(small + 0);
        uint32_t H = 1;
        while (H < 2 * ncells) H <<= 1;
        uint4 *slot = sc.get<uint4>("hslot" + std::to_string(L), H);
        CK(cudaMemsetAsync(slot, 0xff, sizeof(uint4) * H, s));
        k_hash_insert<<<grid_for(ncells, 256, nsm), 256, 0, s>>>(keys, cbegin, small + 0, shift, slot, H - 1); ++launches;
        return {slot, H - 1, true, nullptr};
    }

    template <class K>
    void radix_sort(K *&keys, uint32_t *&vals, K *&kalt, uint32_t *&valt, int64_t n, int bits)
    {
        if (n <= 1 || bits <= 0) return;
        int nb = (int)((n + RS_TILE - 1) / RS_TILE);
        uint32_t *hist = sc.get<uint32_t>("rs_hist", (size_t)256 * nb);
        for (int shift = 0; shift < bits; shift += 8) {
            k_rs_hist<K><<<nb, RS_THREADS, 0, s>>>(keys, n, shift, hist, nb); ++launches;
            scan(hist, hist, (int64_t)256 * nb);
            k_rs_scatter<K><<<nb, RS_THREADS, 0, s>>>(keys, vals, kalt, valt, n, shift, hist, nb); ++launches;
            std::swap(keys, kalt);
            std::swap(vals, valt);
        }
    }

    // self-join of the n points, or (qry_in != null) the K nearest of the n
    // points for each of the nq query points; only query rows [row_b, row_e)
    // (row_e < 0: all) are computed, into outputs of row_e - row_b rows
    void run(const float *pts_in, int64_t n, int d, int K, int32_t *ids_in, double *dist_in,
             const float *qry_in = nullptr, int64_t nq_in = 0, int64_t row_b = 0, int64_t row_e = -1);

    // start level of every sorted position of a self-join (sliding-window
    // cell counts over the sorted keys)
    void start_levels(const uint64_t *keys, int64_t n, int d, int K, float wmul, const GridParams &hp,
                      uint32_t *lvl)
    {
        // target count of a query's parent cell: between the expected counts
        // of the ideal level's parent and of the ideal level itself
        const double Vd = std::pow(M_PI, d / 2.0) / std::tgamma(d / 2.0 + 1.0);
        const double ideal = std::pow(2.0 * (double)wmul, d) * (double)K / Vd;
        int64_t H = (int64_t)std::max(2.0, std::floor(ideal / std::pow(2.0, d / 2.0)));
        if (hp.finer == 0) {
            // no density skew: every query starts at the search-distance width
            k_fill_u32<<<grid_for(n, 256, nsm), 256, 0, s>>>(lvl, n, hp.start_level); ++launches;
        } else if (n >= H && hp.top_level > 0) {
            const int64_t nw = n - H + 1;
            uint8_t *pm = sc.get<uint8_t>("win_pm", nw), *smn = sc.get<uint8_t>("win_sm", nw);
            const int64_t nblk = (nw + H - 1) / H;
            k_window_blocks<<<grid_for(nblk, 128, nsm, 16), 128, 0, s>>>(keys, nw, H, d, pm, smn); ++launches;
            k_start_levels<<<grid_for(n, 256, nsm), 256, 0, s>>>(pm, smn, n, H, hp.top_level, hp.start_level, lvl);
            ++launches;
        } else {
            k_fill_u32<<<grid_for(n, 256, nsm), 256, 0, s>>>(lvl, n, hp.top_level); ++launches;
        }
    }

    // cut points of nshards cost-balanced ranges of sorted query positions
    // (bounds[0] = 0 .. bounds[nshards] = n) and each range's estimated cost
    // Diagnostic (knnjoin_index_dump): index the points (a1-a5) as a join
    // does, copy the sorted keys, the permutation and the grid to the host,
    // build level L's cell table as the scan would, and look up the probe keys
    // in it.
    void index_dump(const float *pts, int64_t n, int d, int K, int L, uint64_t *keys_out, uint32_t *perm_out,
                    double *grid_out, const uint64_t *probe, int64_t nprobe, uint32_t *runs_out)
    {
        const int saved_mode = res_mode;
        res_mode = 1;
        try {
            run(pts, n, d, K, nullptr, nullptr);
        } catch (...) {
            res_mode = saved_mode;
            throw;
        }
        res_mode = saved_mode;
        const GridParams hp = res_hp;
        if (L < 0 || L > hp.bits) fail(KNN_ERR_INVALID, "level must be in [0, bits per dimension]");
        if (keys_out) CK(cudaMemcpyAsync(keys_out, res_keys, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost, s));
        if (perm_out) CK(cudaMemcpyAsync(perm_out, res_perm, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, s));
        if (grid_out) {
            grid_out[0] = hp.w0;
            grid_out[1] = hp.bits;
            grid_out[2 + 2 * d] = -1.0;  // no table built (no probes)
            for (int k = 0; k < d; ++k) {
                grid_out[2 + k] = hp.lo[k];
                grid_out[2 + d + k] = hp.cmax0[k];
            }
        }
        if (nprobe > 0) {
            uint32_t *flags = sc.get<uint32_t>("flags", n), *rid = sc.get<uint32_t>("rid", n);
            uint32_t *cbegin = sc.get<uint32_t>("cbegin", n + 1), *small = sc.get<uint32_t>("small", 16);
            const LevelTab t = cell_table(res_keys, n, d, L, hp, flags, rid, cbegin, small);
            if (grid_out) grid_out[2 + 2 * d] = t.dense ? 1.0 : 0.0;
            DenseDims stride{}, cm{};
            uint32_t G = 1;
            for (int k = 0; k < d; ++k) {
                stride.stride[k] = G;
                cm.stride[k] = (uint32_t)(hp.cmax0[k] >> L);
                G *= cm.stride[k] + 1u;  // only used with a dense table (G within 32 bits)
            }
            uint64_t *pk = sc.get<uint64_t>("probe_keys", (size_t)nprobe);
            uint2 *pr = sc.get<uint2>("probe_runs", (size_t)nprobe);
            CK(cudaMemcpyAsync(pk, probe, sizeof(uint64_t) * nprobe, cudaMemcpyHostToDevice, s));
            k_probe_cells<<<grid_for(nprobe, 256, nsm), 256, 0, s>>>(pk, nprobe, d, hp.bits - L, stride, cm, t.dense,
                                                                      t.slot, t.mask, pr); ++launches;
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(runs_out, pr, sizeof(uint2) * nprobe, cudaMemcpyDeviceToHost, s));
        }
        CK(cudaStreamSynchronize(s));
    }

    void shard_bounds(const float *pts, int64_t n, int d, int K, int nshards, int64_t *bounds, double *costs);
};

__global__ void k_init_reduce(PrepReduce *r)
{
    int t = threadIdx.x;
    if (t < MAX_DIM) {
        r->lo_enc[t] = 0xffffffffu;
        r->hi_enc[t] = 0u;
    }
    if (t == 0) {
        r->min_lsb = 1 << 30;
        r->max_msb = -(1 << 30);
        r->nonfinite = 0;
        r->eps_sum = 0.0;
        r->eps_pairs = 0;
    }
    for (int i = t; i < 2 * 1024; i += blockDim.x) (&r->hist[0][0])[i] = 0;
    for (int i = t; i < 256; i += blockDim.x) r->scount[i] = 0;
}

size_t scan_smem_bytes(int d, int noff, int CH, int B)
{
    size_t s = (size_t)noff * 8 + (size_t)((noff + 1 + 3) & ~3) * 4 + (size_t)d * CH * 4 + (size_t)CH * 4;
    s += (size_t)SCAN_WARPS * B * 4 * 2 + (size_t)SCAN_WARPS * 256 * 4;
    s += (size_t)SCAN_WARPS * B * (8 + 4 + 4);
    return s;
}

template <int DIM>
void launch_scan(Pipeline &P, const ScanArgs &a, size_t smem)
{
    static bool configured[64] = {};
    int dev = P.device;
    if (!configured[dev & 63]) {
        CK(cudaFuncSetAttribute(k_scan<DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        configured[dev & 63] = true;
    }
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_scan<DIM>, SCAN_CTA, smem));
    if (occ < 1) fail(KNN_ERR_INVALID, "scan kernel does not fit on an SM (K or d too large)");
    unsigned grid = (unsigned)std::min<int64_t>(a.nitems, (int64_t)occ * P.nsm);
    if (grid == 0) return;
    k_scan<DIM><<<grid, SCAN_CTA, smem, P.s>>>(a);
    ++P.launches;
    CK(cudaGetLastError());
}

void dispatch_scan(Pipeline &P, int d, const ScanArgs &a, size_t smem)
{
    switch (d) {
    case 1: launch_scan<1>(P, a, smem); break;
    case 2: launch_scan<2>(P, a, smem); break;
    case 3: launch_scan<3>(P, a, smem); break;
    case 4: launch_scan<4>(P, a, smem); break;
    case 5: launch_scan<5>(P, a, smem); break;
    case 6: launch_scan<6>(P, a, smem); break;
    case 7: launch_scan<7>(P, a, smem); break;
    case 8: launch_scan<8>(P, a, smem); break;
    default: fail(KNN_ERR_INVALID, "d out of range");
    }
}

int bitlen32(uint32_t v) { return v ? 32 - __builtin_clz(v) : 0; }

size_t scan2_smem_bytes(int d, int QM, int E)
{
    return (size_t)S2_WARPS * scan2_warp_bytes(d, QM, E);
}

// The scan kernel k_scan2 for dimension d (its instances live in one
// translation unit per d, scan2_launch.cu); mega: the long-run walk that
// skips mega-tiles.
void dispatch_scan2(Pipeline &P, int d, int E, bool mega, const ScanArgs &a, size_t smem)
{
    bool nofit = false;
    cudaError_t e;
    switch (d) {
    case 1: e = scan2_launch<1>(a, E, mega, smem, P.s, P.nsm, P.device, &nofit, &P.launches); break;
    case 2: e = scan2_launch<2>(a, E, mega, smem, P.s, P.nsm, P.device, &nofit, &P.launches); break;
    case 3: e = scan2_launch<3>(a, E, mega, smem, P.s, P.nsm, P.device, &nofit, &P.launches); break;
    case 4: e = scan2_launch<4>(a, E, mega, smem, P.s, P.nsm, P.device, &nofit, &P.launches); break;
    case 5: e = scan2_launch<5>(a, E, mega, smem, P.s, P.nsm, P.device, &nofit, &P.launches); break;
    case 6: e = scan2_launch<6>(a, E, mega, smem, P.s, P.nsm, P.device, &nofit, &P.launches); break;
    case 7: e = scan2_launch<7>(a, E, mega, smem, P.s, P.nsm, P.device, &nofit, &P.launches); break;
    case 8: e = scan2_launch<8>(a, E, mega, smem, P.s, P.nsm, P.device, &nofit, &P.launches); break;
    default: fail(KNN_ERR_INVALID, "d out of range");
    }
    if (e == cudaErrorInvalidValue) fail(KNN_ERR_INVALID, "internal: bad buffer size");
    ck(e, "scan kernel launch");
    if (nofit) fail(KNN_ERR_INVALID, "scan kernel does not fit on an SM");
}

// The scan kernel over several joins of dimension d (k_scan2_multi).
void dispatch_scan2_multi(Pipeline &P, int d, int E, bool mega, const MultiScanArgs &p, size_t smem)
{
    bool nofit = false;
    cudaError_t e;
    switch (d) {
    case 1: e = scan2_launch_multi<1>(p, E, mega, smem, P.s, P.nsm, P.device, &nofit, &P.launches); break;
    case 2: e = scan2_launch_multi<2>(p, E, mega, smem, P.s, P.nsm, P.device, &nofit, &P.launches); break;
    case 3: e = scan2_launch_multi<3>(p, E, mega, smem, P.s, P.nsm, P.device, &nofit, &P.launches); break;
    case 4: e = scan2_launch_multi<4>(p, E, mega, smem, P.s, P.nsm, P.device, &nofit, &P.launches); break;
    case 5: e = scan2_launch_multi<5>(p, E, mega, smem, P.s, P.nsm, P.device, &nofit, &P.launches); break;
    case 6: e = scan2_launch_multi<6>(p, E, mega, smem, P.s, P.nsm, P.device, &nofit, &P.launches); break;
    case 7: e = scan2_launch_multi<7>(p, E, mega, smem, P.s, P.nsm, P.device, &nofit, &P.launches); break;
    case 8: e = scan2_launch_multi<8>(p, E, mega, smem, P.s, P.nsm, P.device, &nofit, &P.launches); break;
    default: fail(KNN_ERR_INVALID, "d out of range");
    }
    if (e == cudaErrorInvalidValue) fail(KNN_ERR_INVALID, "internal: bad buffer size");
    ck(e, "batched scan kernel launch");
    if (nofit) fail(KNN_ERR_INVALID, "scan kernel does not fit on an SM");
}

// Work items of up to S2_MULTI_JOBS joins as one queue: entry = job << 24 |
// item, sort key = QM - (queries of the item), so that a stable sort puts
// full items (dense cells) first across the joins, each join's own density
// order kept among equal keys.
struct UnionSrc {
    const uint2 *items[S2_MULTI_JOBS];
    uint32_t off[S2_MULTI_JOBS + 1];  // prefix sums of the joins' item counts
    int njobs;
    int qm;
};

__global__ void k_union_entries(const UnionSrc src, uint32_t *__restrict__ keys, uint32_t *__restrict__ vals)
{
    const uint32_t total = src.off[src.njobs];
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        int lo = 0, hi = src.njobs - 1;  // the job whose range holds t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (src.off[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const uint32_t item = t - src.off[lo];
        const uint32_t q = src.items[lo][item].y & 0xffffu;
        keys[t] = (uint32_t)src.qm - min(q, (uint32_t)src.qm);
        vals[t] = ((uint32_t)lo << 24) | item;
    }
}

// Batched joins scanned together (knnjoin_config.batch_union).  Every join
// of the batch runs its own pass loop on its own stream and host thread; at
// the scan of a pass it hands its arguments here and waits until every join
// still running has done the same (or left), and the last to arrive makes
// the launches: one per group of joins with the same d, buffer size and
// long-run walk (at most S2_MULTI_JOBS joins each), over the union of their
// work items ordered dense first across the joins (Sec. 4.5 work queue,
// its high-density-first priority applied across joins).
struct UnionScan {
    struct Entry {
        ScanArgs a;
        int d, E;
        bool mega;
        size_t smem;
        cudaEvent_t ready;
    };
    std::mutex mu;
    std::condition_variable cv;
    int members = 0, arrived = 0;
    uint64_t round = 0;
    std::vector<Entry> entries;
    Pipeline co;  // the coordinator's stream and scratch (queue build, launches)
    cudaEvent_t done = nullptr;
    knnjoin_status err = KNN_OK;
    std::string msg;
    int64_t launches = 0, rounds = 0;

    // (a round that closes early, launching for the joins present after a
    // short wait, was measured slower: more, smaller launches)
    void scan(Pipeline &P, int d, int E, bool mega, const ScanArgs &a, size_t smem)
    {
        CK(cudaEventRecord(P.uev, P.s));
        std::unique_lock<std::mutex> lk(mu);
        if (err != KNN_OK) fail(err, msg);
        entries.push_back({a, d, E, mega, smem, P.uev});
        ++arrived;
        const uint64_t my = round;
        if (arrived == members) launch_locked();
        else cv.wait(lk, [&] { return round != my; });
        if (err != KNN_OK) fail(err, msg);
        CK(cudaStreamWaitEvent(P.s, done, 0));
    }
    // a join has finished (or failed): the others no longer wait for it
    void leave()
    {
        std::lock_guard<std::mutex> lk(mu);
        --members;
        if (arrived > 0 && arrived == members) launch_locked();
    }
    void launch_locked()
    {
        try {
            for (auto &e : entries) CK(cudaStreamWaitEvent(co.s, e.ready, 0));
            std::map<std::tuple<int, int, bool>, std::vector<int>> groups;
            for (int j = 0; j < (int)entries.size(); ++j)
                groups[std::make_tuple(entries[j].d, entries[j].E, entries[j].mega)].push_back(j);
            for (auto &g : groups) {
                const std::vector<int> &idx = g.second;
                const int d = std::get<0>(g.first), E = std::get<1>(g.first);
                const bool mega = std::get<2>(g.first);
                for (size_t c0 = 0; c0 < idx.size(); c0 += S2_MULTI_JOBS) {
                    const int nj = (int)std::min<size_t>(S2_MULTI_JOBS, idx.size() - c0);
                    std::unique_ptr<MultiScanArgs> p(new MultiScanArgs());
                    memset(p.get(), 0, sizeof(MultiScanArgs));
                    UnionSrc src;
                    memset(&src, 0, sizeof(src));
                    uint64_t total = 0;
                    for (int j = 0; j < nj; ++j) {
                        const ScanArgs &a = entries[idx[c0 + j]].a;
                        p->jobs[j] = a;
                        src.items[j] = a.items;
                        src.off[j] = (uint32_t)total;
                        if (a.nitems >= (1u << 24)) fail(KNN_ERR_INVALID, "batched scan: a join has too many work items");
                        total += a.nitems;
                    }
                    if (total >= (1ull << 31)) fail(KNN_ERR_INVALID, "batched scan: too many work items");
                    src.off[nj] = (uint32_t)total;
                    src.njobs = nj;
                    src.qm = scan2_queries_per_item(E);
                    uint32_t *keys = co.sc.get<uint32_t>("u_keys", total), *vals = co.sc.get<uint32_t>("u_vals", total);
                    uint32_t *k2 = co.sc.get<uint32_t>("u_keys2", total), *v2 = co.sc.get<uint32_t>("u_vals2", total);
                    k_union_entries<<<grid_for((int64_t)total, 256, co.nsm), 256, 0, co.s>>>(src, keys, vals);
                    ++launches;
                    co.radix_sort<uint32_t>(keys, vals, k2, v2, (int64_t)total, bitlen32((uint32_t)src.qm));
                    uint32_t *counter = co.sc.get<uint32_t>("u_counter", 1);
                    CK(cudaMemsetAsync(counter, 0, 4, co.s));
                    p->counter = counter;
                    p->uitems = vals;
                    p->nuitems = (uint32_t)total;
                    p->njobs = nj;
                    dispatch_scan2_multi(co, d, E, mega, *p, entries[idx[c0]].smem);
                }
            }
            CK(cudaEventRecord(done, co.s));
        } catch (const KnnError &e) {
            err = e.st;
            msg = e.msg;
        }
        ++round;
        ++rounds;
        arrived = 0;
        entries.clear();
        cv.notify_all();
    }
};

#ifdef KNN_CHECKS
// Failed-check words of every kernel unit (checked builds).
unsigned all_check_words(bool clear)
{
    unsigned w = 0, z = 0, h = 0;
    if (cudaMemcpyFromSymbol(&h, g_check_word, sizeof(h)) == cudaSuccess && h) {
        w |= h;
        if (clear) cudaMemcpyToSymbol(g_check_word, &z, sizeof(z));
    }
    w |= scan2_check_word<1>(clear) | scan2_check_word<2>(clear) | scan2_check_word<3>(clear) |
         scan2_check_word<4>(clear) | scan2_check_word<5>(clear) | scan2_check_word<6>(clear) |
         scan2_check_word<7>(clear) | scan2_check_word<8>(clear);
    return w;
}
#endif

void Pipeline::run(const float *pts_in, int64_t n, int d, int K, int32_t *ids_in, double *dist_in,
                   const float *qry_in, int64_t nq_in, int64_t row_b, int64_t row_e)
{
    NvtxRange trace_join(qry_in ? "knnjoin: R x S join" : "knnjoin: self-join");
    const bool self = qry_in == nullptr;
    const int64_t nq = self ? n : nq_in;  // queries (output rows)
    const int rmode = res_mode;           // 1: build a resident index, 2: query one
    if (row_e < 0) row_e = nq;
    const int64_t nrows = row_e - row_b;  // output rows (a shard of the queries, or all)
    const bool sharded = nrows < nq || shard_sorted;
    if (shard_sorted && (!self || policy != 0 || rmode != 0))
        fail(KNN_ERR_INVALID, "cost-balanced shards: self-joins under the default policy only");
    CK(cudaSetDevice(device));
    const bool pts_dev = device_side(pts_in, device, "points");
    const bool ids_dev = device_side(ids_in, device, "out_ids");
    const bool dist_dev = device_side(dist_in, device, "out_dist");
    // large joins whose results go to host memory take turns (see big_token)
    // (taken just before the first pass, so that the copy of the points and
    // the index build overlap the scan of the join holding the token)
    std::unique_lock<std::mutex> turn;
    const bool take_turn = big_token && !(ids_dev && dist_dev) && nrows * (int64_t)K >= BIG_JOB_ENTRIES;
    memset(&stats, 0, sizeof(stats));
    launches = 0;
    double ms_scan = 0.0;
    stats.n = nrows;
    stats.d = d;
    stats.K = K;

    const float *pts = pts_in;
    if (!pts_dev && rmode != 2) {  // a resident index keeps the data on the device
        float *p = sc.get<float>("pts_in", (size_t)n * d);
        CK(cudaMemcpyAsync(p, pts_in, sizeof(float) * n * d, cudaMemcpyHostToDevice, s));
        pts = p;
    }
    const float *qry = pts;
    if (!self) {
        qry = qry_in;
        if (!device_side(qry_in, device, "queries")) {
            float *p = sc.get<float>("qry_in", (size_t)nq * d);
            CK(cudaMemcpyAsync(p, qry_in, sizeof(float) * nq * d, cudaMemcpyHostToDevice, s));
            qry = p;
        }
    }
    // results bound for host memory that would not fit on the device (or
    // exceed out_chunk_bytes) are computed in chunks of query rows, each
    // copied out before the next
    int64_t chunk_rows = nrows;
    if (policy == 0 && rmode != 1 && !(ids_dev && dist_dev) && !shard_sorted) {
        const size_t row_bytes = (size_t)K * (sizeof(int32_t) + sizeof(double));
        size_t limit = out_chunk_bytes;
        if (limit == 0) {
            size_t freeb = 0, totalb = 0;
            CK(cudaMemGetInfo(&freeb, &totalb));
            if ((size_t)nrows * row_bytes > freeb / 2) limit = freeb / 4;
        }
        if (limit > 0 && (size_t)nrows * row_bytes > limit)
            chunk_rows = std::max<int64_t>(1, (int64_t)(limit / row_bytes));
    }
    const bool chunked = chunk_rows < nrows;
    stats.chunks = (nrows + chunk_rows - 1) / chunk_rows;
    // chunks go through scratch buffers (both outputs), whole results straight
    // to device outputs
    int32_t *ids = !chunked && (ids_dev || rmode == 1) ? ids_in : sc.get<int32_t>("ids_out", (size_t)chunk_rows * K);
    double *dist = !chunked && (dist_dev || rmode == 1) ? dist_in : sc.get<double>("dist_out", (size_t)chunk_rows * K);
    CK(cudaEventRecord(ev[0], s));

    // a1
    std::unique_ptr<NvtxRange> trace_phase(new NvtxRange("a1-a2 bounding box, search distance"));
    PrepReduce *red = sc.get<PrepReduce>("red", 1);
    GridParams *gp = sc.get<GridParams>("gp", 1);
    unsigned long long *st = sc.get<unsigned long long>("stats", 8);
    CK(cudaMemsetAsync(st, 0, 8 * sizeof(unsigned long long), s));
    const float wmul = force_wm > 0.0f ? force_wm : (tune ? tune->lookup(d, K, n) : width_mult);
    stats.width_mult = wmul;
    ParamsIn pin;
    pin.n = n;
    pin.d = d;
    pin.K = K;
    pin.S = std::min<int64_t>(n, 256);
    pin.m = std::min<int64_t>(n, 65536);
    pin.width_mult = wmul;
    pin.start_level = 0;
    pin.max_finer = 3;
    if (policy == 1) {  // the paper's policy: cell side = eps = eps_min, one level
        pin.width_mult = 1.0f;
        pin.max_finer = 0;
        stats.width_mult = 1.0;
    }
    float *xs = nullptr, *rxs = nullptr;
    GridParams hp;
    if (rmode == 2) {
        // resident index: the data side is kept; prepare the queries only.
        // The grid and the fixed-point frame are the data's: a query outside
        // the data's box falls in a boundary cell (cell_of clamps), which
        // keeps every gap and certificate a lower bound, and a batch whose
        // coordinates leave the fixed-point frame uses the FP64 scoring path.
        PrepReduce *qred = sc.get<PrepReduce>("qred", 1);
        k_init_reduce<<<1, 256, 0, s>>>(qred); ++launches;
        rxs = sc.get<float>("rxs", (size_t)nq * d);
        k_prep<<<grid_for(nq, 256, nsm), 256, 0, s>>>(qry, nq, d, rxs, qred); ++launches;
        CK(cudaGetLastError());
        fetch(pinned, &qred->min_lsb, 3 * sizeof(int));
        CK(cudaStreamSynchronize(s));
        int qf[3];
        memcpy(qf, pinned, sizeof(qf));
        if (qf[2]) fail(KNN_ERR_INVALID, "queries contain a NaN or infinite coordinate");
        hp = res_hp;
        stats.width_mult = res_wm;
        if (hp.fixed_ok && qf[1] >= qf[0]) hp.fixed_ok = (qf[0] >= -hp.F && qf[1] + hp.F <= 29) ? 1 : 0;
    } else {
        k_init_reduce<<<1, 256, 0, s>>>(red); ++launches;
        xs = sc.get<float>("xs", (size_t)n * d);
        k_prep<<<grid_for(n, 256, nsm), 256, 0, s>>>(pts, n, d, xs, red); ++launches;
        // R x S: the bounding box and fixed-point frame cover the queries too, so
        // every query lies in the grid; the search distance and the index are
        // the data set's
        if (!self) {
            rxs = sc.get<float>("rxs", (size_t)nq * d);
            k_prep<<<grid_for(nq, 256, nsm), 256, 0, s>>>(qry, nq, d, rxs, red); ++launches;
        }
        // a2
        int64_t smp = std::min<int64_t>(2000, std::max<int64_t>(2, llround(0.001 * (double)n)));
        smp = std::min(smp, n);
        k_eps_pairs<<<grid_for(smp * smp, 256, nsm), 256, 0, s>>>(xs, n, d, smp, red); ++launches;
        float *srow = sc.get<float>("eps_srow", (size_t)pin.S * 8);
        float *mrow = sc.get<float>("eps_mrow", (size_t)pin.m * 8);
        k_eps_rows<<<grid_for(pin.S + pin.m, 256, nsm), 256, 0, s>>>(xs, n, d, pin.S, pin.m, srow, mrow); ++launches;
        // subset points x slices of the samples (4 slices: enough warps to
        // fill the GPU at m = 65,536)
        const dim3 gm((unsigned)((pin.m + 255) / 256), 4);
        const bool p4 = d <= 4;  // rows compared over 4 floats, else 8
        // parameter stages 0-2 are formed inside the histogram kernels (each
        // block from the reductions before it), stage 3 after the counts
        if (p4) k_eps_hist<4><<<gm, 256, 0, s>>>(srow, mrow, n, pin.S, pin.m, gp, red, 0, pin);
        else k_eps_hist<8><<<gm, 256, 0, s>>>(srow, mrow, n, pin.S, pin.m, gp, red, 0, pin);
        ++launches;
        if (p4) k_eps_hist<4><<<gm, 256, 0, s>>>(srow, mrow, n, pin.S, pin.m, gp, red, 1, pin);
        else k_eps_hist<8><<<gm, 256, 0, s>>>(srow, mrow, n, pin.S, pin.m, gp, red, 1, pin);
        ++launches;
        if (p4) k_eps_count<4><<<gm, 256, 0, s>>>(srow, mrow, n, d, pin.S, pin.m, gp, red, pin);
        else k_eps_count<8><<<gm, 256, 0, s>>>(srow, mrow, n, d, pin.S, pin.m, gp, red, pin);
        ++launches;
        k_params<<<1, 32, 0, s>>>(red, gp, pin, 3); ++launches;
        CK(cudaGetLastError());
        hp = read1(gp);
        if (hp.nonfinite) fail(KNN_ERR_INVALID, "points contain a NaN or infinite coordinate");
    }
    stats.eps_mean = hp.eps_mean;
    stats.eps_min = hp.eps_min;
    stats.cell_width = hp.w0;
    stats.key_bits = hp.key_bits;
    stats.fixed_point = hp.fixed_ok;
    stats.start_level = hp.start_level;

    // Epochs: one under the default policy.  Under the paper's policy each
    // epoch indexes the data on a grid of cell side eps, runs one pass over
    // the queries not done yet with the certificate radius capped at eps, and
    // widens eps by eps_min / 2 (Sec. 4.4 re-indexing; after 256 epochs eps
    // doubles instead, which bounds the number of epochs).
    int pass = 0;
    int64_t cand_before = 0;
    int64_t tail_cand = 0;  // pairs the brute-force tail evaluated
    int first_level = -1;
    uint32_t *done = nullptr;  // per original query row (paper's policy)
    if (policy == 1) {
        done = sc.get<uint32_t>("done", nq);
        CK(cudaMemsetAsync(done, 0, sizeof(uint32_t) * nq, s));
    }
    float eps_mult = 1.0f;
    // tail strategy (Sec. 5.4): at most `tail_limit` queries left -> one pass
    // over the whole grid (level top_level: a box holding every point, which
    // certifies every query)
    const int64_t tail_limit = tail_queries < 0 ? -1
                               : tail_queries > 0 ? (int64_t)tail_queries
                                                  : std::max<int64_t>(1024, nq / 100);
    bool tail_epoch = false;  // the paper's policy: this epoch is the tail pass
    uint32_t *last_perm = nullptr;  // the last epoch's sorted -> original map
    for (int epoch = 0;; ++epoch) {
        // a3-a5
        trace_phase.reset(new NvtxRange("a3-a6 keys, sort, gather, start levels"));
        uint64_t *keys = res_keys;
        uint32_t *perm = res_perm;
        float *xsort = res_xsort;
        if (rmode != 2) {
            uint64_t *kalt = sc.get<uint64_t>("keys_alt", n);
            uint32_t *palt = sc.get<uint32_t>("perm_alt", n);
            keys = sc.get<uint64_t>("keys", n);
            perm = sc.get<uint32_t>("perm", n);
            k_keys<<<grid_for(n, 256, nsm), 256, 0, s>>>(xs, n, gp, keys, perm); ++launches;
            radix_sort<uint64_t>(keys, perm, kalt, palt, n, hp.key_bits);
            xsort = sc.get<float>("xsort", (size_t)n * pad_dim(d));
            k_gather<<<grid_for(n, 256, nsm), 256, 0, s>>>(xs, n, d, perm, xsort); ++launches;
        }
        last_perm = perm;
        if (rmode == 1) {
            // resident index built: keep the data side and stop (no queries)
            CK(cudaGetLastError());
            res_keys = keys;
            res_perm = perm;
            res_xsort = xsort;
            res_hp = hp;
            res_wm = stats.width_mult;
            for (auto &t : res_tabs) t = LevelTab{};
            CK(cudaEventRecord(ev[1], s));
            CK(cudaEventRecord(ev[2], s));
            CK(cudaStreamSynchronize(s));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, ev[0], ev[2]));
            stats.ms_total = ms;
            stats.ms_index = ms;
            stats.launches = launches;
            return;
        }
        // queries: keys on the data grid, sorted, gathered (the data arrays for a self-join)
        uint64_t *qkeys = keys;
        uint32_t *qperm = perm;
        float *qxsort = xsort;
        if (!self) {
            uint64_t *ralt = sc.get<uint64_t>("rkeys_alt", nq);
            uint32_t *rpalt = sc.get<uint32_t>("rperm_alt", nq);
            qkeys = sc.get<uint64_t>("rkeys", nq);
            qperm = sc.get<uint32_t>("rperm", nq);
            k_keys<<<grid_for(nq, 256, nsm), 256, 0, s>>>(rxs, nq, gp, qkeys, qperm); ++launches;
            radix_sort<uint64_t>(qkeys, qperm, ralt, rpalt, nq, hp.key_bits);
            qxsort = sc.get<float>("rxsort", (size_t)nq * pad_dim(d));
            k_gather<<<grid_for(nq, 256, nsm), 256, 0, s>>>(rxs, nq, d, qperm, qxsort); ++launches;
        }
        CK(cudaGetLastError());
        if (epoch == 0) CK(cudaEventRecord(ev[1], s));

        // start level of every query (sliding-window cell counts)
        uint32_t *lvl = sc.get<uint32_t>("lvl", nq);
        if (policy == 1) {
            k_fill_u32<<<grid_for(nq, 256, nsm), 256, 0, s>>>(lvl, nq, tail_epoch ? (uint32_t)hp.top_level : 0u);
            ++launches;
        } else if (!self) {
            // R x S: every query starts at the search-distance width (queries in
            // sparse regions move up a level per pass until certified)
            k_fill_u32<<<grid_for(nq, 256, nsm), 256, 0, s>>>(lvl, nq, hp.start_level); ++launches;
        } else {
            start_levels(keys, n, d, K, wmul, hp, lvl);
        }

        // pass loop
        // query-side arrays are indexed by sorted query position
        const int64_t nmax = std::max(n, nq);
        uint32_t *active = sc.get<uint32_t>("active", nq), *active2 = sc.get<uint32_t>("active2", nq);
        uint32_t *ovl = sc.get<uint32_t>("ovl", nq);
        uint32_t *flags = sc.get<uint32_t>("flags", nmax), *rid = sc.get<uint32_t>("rid", nmax);
        uint32_t *cbegin = sc.get<uint32_t>("cbegin", n + 1);
        uint32_t *small = sc.get<uint32_t>("small", 16);
        uint32_t *status = sc.get<uint32_t>("fail", nq);  // per sorted query position
        float *seed = sc.get<float>("seed", nq);           // per sorted query position, +inf to start
        k_fill_u32<<<grid_for(nq, 256, nsm), 256, 0, s>>>((uint32_t *)seed, nq, 0x7f800000u); ++launches;
        uint32_t *lkey = sc.get<uint32_t>("lkey", nq), *lkey2 = sc.get<uint32_t>("lkey2", nq);
        int64_t m = 0, row0 = 0;
        // general kernel (scan.cuh)
        const int B1 = std::max(128, 1 << bitlen32((uint32_t)(2 * K - 1)));
        const int CH = d <= 6 ? 1024 : 512;
        int noff = 1;
        for (int k = 0; k < d; ++k) noff *= 3;
        const size_t smem1 = scan_smem_bytes(d, noff, CH, B1);
        // fast kernel (scan2.cuh)
        const bool fast = K + 32 <= 256;
        // candidate buffer of 32 * E2 entries per query: the smallest holding
        // K + 32, or a larger one the autotuner found faster for this class
        const int E2min = K + 32 <= 64 ? 2 : (K + 32 <= 128 ? 4 : 8);
        int E2 = E2min;
        {
            const int tE = force_E > 0 ? force_E : (tune && policy == 0 ? tune->lookup_E(d, K, n) : 0);
            if (tE >= E2min && tE <= 8) E2 = tE;
        }
        stats.buffer_entries = 32 * E2;
        const int QM = scan2_queries_per_item(E2);
        const size_t smem2 = scan2_smem_bytes(d, QM, E2);

        // per-level cell hash maps, built on first use (a resident index
        // keeps its maps from one call to the next)
        LevelTab local_tabs[MAX_LEVELS];
        LevelTab *tabs = rmode == 2 ? res_tabs : local_tabs;
        auto build_level = [&](int L) {
            if (!tabs[L].built) tabs[L] = cell_table(keys, n, d, L, hp, flags, rid, cbegin, small);
        };

        // work items of a (level, position)-ordered list of sorted positions
        auto make_items = [&](const uint32_t *list, int64_t mm, int qpi, uint32_t &nitems) -> uint2 * {
            uint32_t *gbegin = sc.get<uint32_t>("gbegin", mm + 1);
            k_run_flags_lv<<<grid_for(mm, 256, nsm), 256, 0, s>>>(qkeys, list, lvl, mm, d, flags); ++launches;
            scan(flags, rid, mm);
            k_run_begin<<<grid_for(mm, 256, nsm), 256, 0, s>>>(flags, rid, mm, gbegin, small + 1); ++launches;
            // small[2] (the largest group) is zero here: set by the pass's k_pass_init
            uint32_t *skey = sc.get<uint32_t>("skey", mm), *sval = sc.get<uint32_t>("sval", mm);
            uint32_t *skey2 = sc.get<uint32_t>("skey2", mm), *sval2 = sc.get<uint32_t>("sval2", mm);
            k_group_sizes<<<grid_for(mm, 256, nsm), 256, 0, s>>>(gbegin, small + 1, skey, sval, small + 2); ++launches;
            fetch(pinned, small + 1, 8);
            CK(cudaStreamSynchronize(s));
            uint32_t ng = pinned[0], maxsz = pinned[1];
            if (ng <= (uint32_t)GROUP_SORT_SMALL && bitlen32(maxsz) <= 20) {
                // few groups: one block sorts them (one launch instead of the
                // radix sort's three or more per digit)
                k_group_sort_small<<<1, 1024, 0, s>>>(skey, small + 1, small + 2, sval); ++launches;
            } else {
                k_group_sortkey<<<grid_for(ng, 256, nsm), 256, 0, s>>>(skey, small + 1, small + 2); ++launches;
                radix_sort<uint32_t>(skey, sval, skey2, sval2, ng, bitlen32(maxsz));
            }
            if (queue_out && queue_out->empty()) {
                std::vector<uint32_t> hg(ng + 1), hs(ng);
                CK(cudaMemcpyAsync(hg.data(), gbegin, sizeof(uint32_t) * (ng + 1), cudaMemcpyDeviceToHost, s));
                CK(cudaMemcpyAsync(hs.data(), sval, sizeof(uint32_t) * ng, cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                for (uint32_t g = 0; g < ng; ++g) {
                    const uint32_t sz = hg[hs[g] + 1] - hg[hs[g]];
                    queue_out->insert(queue_out->end(), sz, (int64_t)sz);
                }
            }
            uint32_t *nit = sc.get<uint32_t>("nit", ng), *ioff = sc.get<uint32_t>("ioff", ng);
            k_group_nitems<<<grid_for(ng, 256, nsm), 256, 0, s>>>(gbegin, sval, small + 1, qpi, nit); ++launches;
            scan(nit, ioff, ng);
            nitems = (uint32_t)read_total(ioff + ng - 1, nit + ng - 1);
            uint2 *items = sc.get<uint2>("items", nitems);
            k_group_items<<<grid_for(ng, 256, nsm), 256, 0, s>>>(gbegin, sval, small + 1, qpi, ioff, list, lvl, items); ++launches;
            return items;
        };
        // entries of `list` whose status is `value`, in order, into `out`
        auto select_list = [&](const uint32_t *list, int64_t mm, uint32_t value, uint32_t *out) -> int64_t {
            k_status_flags<<<grid_for(mm, 256, nsm), 256, 0, s>>>(list, status, mm, value, flags); ++launches;
            scan(flags, rid, mm);
            const int64_t cntv = read_total(rid + mm - 1, flags + mm - 1);
            if (cntv > 0) {
                k_compact<<<grid_for(mm, 256, nsm), 256, 0, s>>>(list, flags, rid, mm, out); ++launches;
            }
            return cntv;
        };

        if (take_turn && !turn.owns_lock()) turn = std::unique_lock<std::mutex>(*big_token);
        for (int64_t r0 = row_b; r0 < row_e; r0 += chunk_rows) {
            const int64_t r1 = std::min(row_e, r0 + chunk_rows);
            k_iota<<<grid_for(nq, 256, nsm), 256, 0, s>>>(active, nq); ++launches;
            m = nq;
            if (policy == 1 && epoch > 0) {
                // the queries not done yet, by their position in this epoch's order
                k_undone_flags<<<grid_for(nq, 256, nsm), 256, 0, s>>>(qperm, done, nq, flags); ++launches;
                scan(flags, rid, nq);
                m = read_total(rid + nq - 1, flags + nq - 1);
                k_compact<<<grid_for(nq, 256, nsm), 256, 0, s>>>(active, flags, rid, nq, active2); ++launches;
                std::swap(active, active2);
            }
            if ((chunked || sharded) && m > 0) {
                // this chunk's queries: the entries of the active list (all
                // queries, or those not done yet) whose original row is in [r0, r1)
                if (shard_sorted) {
                    k_pos_flags<<<grid_for(m, 256, nsm), 256, 0, s>>>(active, m, (uint32_t)r0, (uint32_t)r1, flags);
                } else {
                    k_row_flags<<<grid_for(m, 256, nsm), 256, 0, s>>>(active, qperm, m, (uint32_t)r0, (uint32_t)r1, flags);
                }
                ++launches;
                scan(flags, rid, m);
                const int64_t mr = read_total(rid + m - 1, flags + m - 1);
                k_compact<<<grid_for(m, 256, nsm), 256, 0, s>>>(active, flags, rid, m, active2); ++launches;
                std::swap(active, active2);
                m = mr;
            }
            row0 = r0;
            // level range of the next pass, when the last pass's summary gave it
            bool range_known = false;
            uint32_t next_lmin = 0, next_lmax = 0;
            while (m > 0) {
                char pass_name[32];
                snprintf(pass_name, sizeof(pass_name), "pass %d", pass);
                trace_phase.reset(new NvtxRange(pass_name));
                if (pass > (policy == 1 ? 8192 : 4 * MAX_LEVELS)) fail(KNN_ERR_CUDA, "internal: too many passes");
                // order the active list by level (stable: positions stay ordered
                // within a level) and build the levels' hash maps
                k_pass_init<<<1, 32, 0, s>>>(small); ++launches;
                k_level_keys<<<grid_for(m, 256, nsm), 256, 0, s>>>(active, lvl, m, lkey, small + 4); ++launches;
                uint32_t lmin = next_lmin, lmax = next_lmax;
                if (!range_known) {
                    fetch(pinned, small + 4, 8);
                    CK(cudaStreamSynchronize(s));
                    lmin = pinned[0];
                    lmax = pinned[1];
                }
                range_known = false;
                if (lmax >= (uint32_t)MAX_LEVELS || lmin > lmax) fail(KNN_ERR_CUDA, "internal: level out of range");
                if (first_level < 0) first_level = (int)lmin;
                if (lmin != lmax) {
                    uint32_t *kk = lkey, *kk2 = lkey2;
                    radix_sort<uint32_t>(kk, active, kk2, active2, m, bitlen32(lmax));
                }
                for (uint32_t L = lmin; L <= lmax; ++L) build_level((int)L);

                ScanArgs a;
                memset(&a, 0, sizeof(a));
                a.xsort = xsort;
                a.perm = perm;
                a.keys = keys;
                a.qxsort = qxsort;
                a.qkeys = qkeys;
                a.qperm = qperm;
                a.self = self ? 1 : 0;
                a.rcap = policy == 1 && !tail_epoch && epoch < 4096 ? hp.w0 : 0.0f;
                a.row0 = row0;
                a.sorted_rows = shard_sorted ? 1 : 0;
                a.out_rows = chunked ? chunk_rows : nrows;
                a.nq = nq;
                a.counter = small + 3;
                {
                    // the levels' cell tables, staged in the pinned readback
                    // area (unchanged until this stream has synchronised)
                    LevelRef *lr_host = (LevelRef *)(pinned + LEVELS_STAGING_WORD);
                    for (int L = 0; L < MAX_LEVELS; ++L) lr_host[L] = {tabs[L].slot, tabs[L].dense, tabs[L].mask, 0u};
                    LevelRef *lr_dev = sc.get<LevelRef>("levels", MAX_LEVELS);
                    CK(cudaMemcpyAsync(lr_dev, lr_host, sizeof(LevelRef) * MAX_LEVELS, cudaMemcpyHostToDevice, s));
                    a.levels = lr_dev;
                }
                a.fail = status;
                a.seed = seed;
                a.out_ids = ids;
                a.out_dist = dist;
                a.stats = st;
                a.n = n;
                a.K = K;
                a.bits = hp.bits;
                for (int k = 0; k < d; ++k) {
                    a.cmax0[k] = hp.cmax0[k];
                    a.lo[k] = hp.lo[k];
                }
                a.w0 = hp.w0;
                a.fixed_ok = hp.fixed_ok;
                a.F = hp.F;
                a.B = B1;
                a.CH = CH;
                a.noff = noff;

                uint32_t nitems = 0;
                a.items = make_items(active, m, fast ? QM : SCAN_WARPS, nitems);
                a.active = active;
                a.nactive = m;
                a.nitems = nitems;
                CK(cudaEventRecord(evs[0], s));
                // skewed data, or a re-queued pass: walk long runs by
                // mega-tiles (a query's box may hold long runs far from it)
                if (fast && uscan) uscan->scan(*this, d, E2, pass > 0 || hp.finer > 0, a, smem2);
                else if (fast) dispatch_scan2(*this, d, E2, pass > 0 || hp.finer > 0, a, smem2);
                else dispatch_scan(*this, d, a, smem1);
                CK(cudaEventRecord(evs[1], s));
                // the scan's time and candidate count, read after the pass's
                // last readback has synchronised the stream (no wait here)
                fetch(pinned + 8, st, sizeof(unsigned long long));
                auto read_pass = [&] {
                    float t = 0.f;
                    CK(cudaEventElapsedTime(&t, evs[0], evs[1]));
                    ms_scan += t;
                    if (pass < 16) stats.ms_pass[pass] = t;
                    unsigned long long c;
                    memcpy(&c, pinned + 8, sizeof(c));
                    if (pass < 16) stats.pass_candidates[pass] = (int64_t)c - cand_before;
                    cand_before = (int64_t)c;
                };
                // one readback for the end of the pass: overflowed queries,
                // re-queued queries (moved a level up here under the default
                // policy) and their level range, which the next pass then
                // does not read back again
                bool counts_known = false;
                int64_t m1 = 0;
                if (fast) {
                    uint32_t *summ = small + 8;  // initialised by the pass's k_pass_init
                    k_status_summary<<<grid_for(m, 256, nsm), 256, 0, s>>>(active, status, m, lvl, hp.top_level,
                                                                          policy == 0 ? 1 : 0, summ); ++launches;
                    fetch(pinned, summ, 4 * sizeof(uint32_t));
                    CK(cudaStreamSynchronize(s));
                    const int64_t mo = pinned[0];
                    m1 = pinned[1];
                    next_lmin = pinned[2];
                    next_lmax = pinned[3];
                    counts_known = mo == 0;
                    if (mo > 0) {
                        // queries whose buffer overflowed (massive ties): general kernel
                        int64_t mo2 = select_list(active, m, 2, ovl);
                        CK(cudaMemsetAsync(small + 2, 0, 4, s));  // make_items' largest group
                        a.items = make_items(ovl, mo2, SCAN_WARPS, nitems);
                        a.active = ovl;
                        a.nactive = mo2;
                        a.nitems = nitems;
                        CK(cudaMemsetAsync(small + 3, 0, 4, s));
                        dispatch_scan(*this, d, a, smem1);
                        stats.overflow_queries += mo2;
                        // those it could not certify move up a level too
                        if (policy == 0) {
                            k_bump_levels<<<grid_for(mo2, 256, nsm), 256, 0, s>>>(ovl, status, mo2, lvl, hp.top_level); ++launches;
                        }
                    }
                }
                if (policy == 1) {
                    k_mark_done<<<grid_for(m, 256, nsm), 256, 0, s>>>(active, status, m, qperm, done); ++launches;
                    int64_t left = select_list(active, m, 1, active2);
                    read_pass();
                    if (pass < 16) stats.pass_queries[pass] = m;
                    ++pass;
                    m = left;
                    break;  // next epoch (or done)
                }
                int64_t next = 0;
                if (counts_known) {
                    // the summary counted the re-queued queries: compact without a readback
                    next = m1;
                    if (next > 0) {
                        k_status_flags<<<grid_for(m, 256, nsm), 256, 0, s>>>(active, status, m, 1u, flags); ++launches;
                        scan(flags, rid, m);
                        k_compact<<<grid_for(m, 256, nsm), 256, 0, s>>>(active, flags, rid, m, active2); ++launches;
                        range_known = true;
                    }
                } else {
                    if (!fast) {
                        k_bump_levels<<<grid_for(m, 256, nsm), 256, 0, s>>>(active, status, m, lvl, hp.top_level); ++launches;
                    }
                    next = select_list(active, m, 1, active2);
                }
                read_pass();
                if (pass < 16) stats.pass_queries[pass] = m;
                std::swap(active, active2);
                m = next;
                ++pass;
                if (m > 0 && pass >= 2 && tail_limit >= 0 && m <= tail_limit) {
                    if ((double)m * (double)n <= TAIL_BF_PAIRS) {
                        // few queries left: every (query, point) pair over the
                        // whole GPU (tail.cuh); a query whose band overflows
                        // keeps status 2 and takes the whole-grid pass below
                        TailArgs t{};
                        t.xsort = xsort;
                        t.qxsort = qxsort;
                        t.perm = perm;
                        t.qperm = qperm;
                        t.list = active;
                        t.m = (int)m;
                        t.n = n;
                        t.K = K;
                        t.self = self ? 1 : 0;
                        t.fixed_ok = hp.fixed_ok;
                        t.F = hp.F;
                        t.prefix = sc.get<uint32_t>("tail_prefix", (size_t)m);
                        t.rank = sc.get<uint32_t>("tail_rank", (size_t)m);
                        t.hist = sc.get<uint32_t>("tail_hist", (size_t)m * 256);
                        t.cnt = sc.get<uint32_t>("tail_cnt", (size_t)m);
                        t.band = sc.get<uint32_t>("tail_band", (size_t)m * TAIL_CAP);
                        t.status = status;
                        t.out_ids = ids;
                        t.out_dist = dist;
                        t.row0 = row0;
                        t.out_rows = chunked ? chunk_rows : nrows;
                        t.sorted_rows = shard_sorted ? 1 : 0;
                        CK(cudaMemsetAsync(t.prefix, 0, sizeof(uint32_t) * m, s));
                        CK(cudaMemsetAsync(t.hist, 0, sizeof(uint32_t) * m * 256, s));
                        CK(cudaMemsetAsync(t.cnt, 0, sizeof(uint32_t) * m, s));
                        k_fill_u32<<<grid_for(m, 256, nsm), 256, 0, s>>>(t.rank, m, (uint32_t)K); ++launches;
                        // about 4 blocks per SM in all, chunks of at least 1024 points
                        const int64_t want = std::max<int64_t>(1, (int64_t)4 * nsm / m);
                        const int64_t chunk = std::max<int64_t>(1024, (n + want - 1) / want);
                        const unsigned chunks = (unsigned)((n + chunk - 1) / chunk);
                        CK(cudaEventRecord(evs[0], s));
                        tail_launch(d, t, chunk, chunks, s, launches);
                        CK(cudaEventRecord(evs[1], s));
                        CK(cudaGetLastError());
                        const int64_t left = select_list(active, m, 2, active2);
                        float tms = 0.f;
                        CK(cudaEventElapsedTime(&tms, evs[0], evs[1]));
                        ms_scan += tms;
                        const int64_t pairs = m * (n - (self ? 1 : 0));
                        tail_cand += pairs;
                        if (pass < 16) {
                            stats.ms_pass[pass] = tms;
                            stats.pass_queries[pass] = m;
                            stats.pass_candidates[pass] = pairs;
                        }
                        ++pass;
                        std::swap(active, active2);
                        m = left;
                    }
                    if (m > 0) {
                        // the tail: the rest in one pass over the whole grid
                        k_set_levels<<<grid_for(m, 256, nsm), 256, 0, s>>>(active, m, lvl, (uint32_t)hp.top_level);
                        ++launches;
                        next_lmin = next_lmax = (uint32_t)hp.top_level;
                        range_known = true;
                    }
                }
            }
            if (chunked) {
                const int64_t rows = r1 - r0;
                k_sqrt_rows<<<grid_for(rows * K, 256, nsm, 16), 256, 0, s>>>(dist, rows * K); ++launches;
                CK(cudaMemcpyAsync(ids_in + (r0 - row_b) * K, ids, sizeof(int32_t) * rows * K, cudaMemcpyDefault, s));
                CK(cudaMemcpyAsync(dist_in + (r0 - row_b) * K, dist, sizeof(double) * rows * K, cudaMemcpyDefault, s));
            }
        }
        if (policy != 1 || m == 0) break;
        if (!tail_epoch && tail_limit >= 0 && m <= tail_limit) {
            // the rest in one pass over the whole grid of this epoch
            tail_epoch = true;
            continue;
        }
        tail_epoch = false;
        // re-index: eps += eps_min / 2 (doubling after 256 epochs)
        eps_mult = epoch < 256 ? eps_mult + 0.5f : eps_mult * 2.0f;
        pin.width_mult = eps_mult;
        k_params<<<1, 32, 0, s>>>(red, gp, pin, 3); ++launches;
        hp = read1(gp);
    }
    trace_phase.reset(new NvtxRange("a11 square roots, result copy"));
    stats.start_level = first_level;
    stats.passes = pass;
    if (!chunked) {
        k_sqrt_rows<<<grid_for(nrows * K, 256, nsm, 16), 256, 0, s>>>(dist, nrows * K); ++launches;
    }
    if (shard_sorted && shard_rows_out) {
        // the original row of each output row (sorted position row_b + j)
        const bool rows_dev = device_side(shard_rows_out, device, "out_rows");
        int64_t *rows = rows_dev ? shard_rows_out : sc.get<int64_t>("shard_rows", (size_t)nrows);
        k_rows_of<<<grid_for(nrows, 256, nsm), 256, 0, s>>>(last_perm, row_b, nrows, rows);
        ++launches;
        if (!rows_dev) CK(cudaMemcpyAsync(shard_rows_out, rows, sizeof(int64_t) * nrows, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaEventRecord(ev[2], s));
    if (turn.owns_lock()) {
        CK(cudaEventSynchronize(ev[2]));
        turn.unlock();
    }
    if (!ids_dev && !chunked) CK(cudaMemcpyAsync(ids_in, ids, sizeof(int32_t) * nrows * K, cudaMemcpyDeviceToHost, s));
    if (!dist_dev && !chunked) CK(cudaMemcpyAsync(dist_in, dist, sizeof(double) * nrows * K, cudaMemcpyDeviceToHost, s));
    fetch(pinned, st, 4 * sizeof(unsigned long long));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
#ifdef KNN_CHECKS
    {
        const unsigned w = all_check_words(true);
        if (w) {
            char msg[96];
            snprintf(msg, sizeof(msg), "bounds check failed (sites 0x%x)", w);
            fail(KNN_ERR_CUDA, msg);
        }
    }
#endif
    unsigned long long hs[4];
    memcpy(hs, pinned, sizeof(hs));
    stats.candidates = (int64_t)hs[0] + tail_cand;
    stats.overflow_queries += (int64_t)hs[1];
    stats.band_entries = (int64_t)hs[2];
    float ms = 0.f, ms1 = 0.f;
    CK(cudaEventElapsedTime(&ms, ev[0], ev[2]));
    CK(cudaEventElapsedTime(&ms1, ev[0], ev[1]));
    stats.ms_total = ms;
    stats.ms_index = ms1;
    stats.ms_scan = ms_scan;
    stats.launches = launches;
}

// Cost-balanced shards (Sec. 6, one join split over GPUs).  Queries are
// taken in the index's key order (cells contiguous, neighbouring cells
// mostly nearby).  A query costs the points of its 3^d neighbourhood at its
// start level (the join's own, from the sliding-window cell counts: sparse
// regions start coarser) -- the candidates it evaluates at ring 1 -- plus
// those one and two levels up while that count is below 2K, where it will
// not be certified and is re-queued.  The cut points split the total cost
// evenly between queries.
void Pipeline::shard_bounds(const float *pts, int64_t n, int d, int K, int nshards, int64_t *bounds, double *costs)
{
    // the data's index (steps a1-a5), kept as a resident index would be
    const int saved_mode = res_mode;
    res_mode = 1;
    try {
        run(pts, n, d, K, nullptr, nullptr);
    } catch (...) {
        res_mode = saved_mode;
        throw;
    }
    res_mode = saved_mode;
    const GridParams hp = res_hp;
    // the join's own start levels of the queries
    uint32_t *lvl = sc.get<uint32_t>("lvl", n), *small = sc.get<uint32_t>("small", 16);
    start_levels(res_keys, n, d, K, res_wm, hp, lvl);
    k_fill_u32<<<1, 32, 0, s>>>(small + 4, 1, 0xffffffffu); ++launches;
    k_fill_u32<<<1, 32, 0, s>>>(small + 5, 1, 0u); ++launches;
    k_minmax_u32<<<grid_for(n, 256, nsm), 256, 0, s>>>(lvl, n, small + 4); ++launches;
    fetch(pinned, small + 4, 8);
    CK(cudaStreamSynchronize(s));
    QueryCostArgs qa;
    memset(&qa, 0, sizeof(qa));
    qa.lmin = (int)pinned[0];
    qa.lmax = std::min(std::min(hp.top_level, (int)pinned[1] + 2), qa.lmin + COST_MAX_LEVELS - 1);
    // per level: cells, their table, each cell's neighbourhood points, and the
    // cell of every sorted position
    uint32_t *flags = sc.get<uint32_t>("flags", n), *rid = sc.get<uint32_t>("rid", n);
    uint32_t *cbegin = sc.get<uint32_t>("cbegin", n + 1);
    for (int l = qa.lmin; l <= qa.lmax; ++l) {
        const int j = l - qa.lmin, sh = d * l;
        k_run_flags<<<grid_for(n, 256, nsm), 256, 0, s>>>(res_keys, nullptr, n, sh, flags); ++launches;
        scan(flags, rid, n);
        k_run_begin<<<grid_for(n, 256, nsm), 256, 0, s>>>(flags, rid, n, cbegin, small + 0); ++launches;
        uint32_t *idx = sc.get<uint32_t>("shard_idx" + std::to_string(j), n);
        k_run_index<<<grid_for(n, 256, nsm), 256, 0, s>>>(flags, rid, n, idx); ++launches;
        const uint32_t nc = read1(small + 0);
        DenseDims dd{}, cm{};
        double G = 1.0;
        for (int k = 0; k < d; ++k) {
            dd.stride[k] = (uint32_t)G;
            cm.stride[k] = (uint32_t)(hp.cmax0[k] >> l);
            G *= (double)(cm.stride[k] + 1);
        }
        uint2 *dense = nullptr;
        uint4 *slot = nullptr;
        uint32_t hmask = 0;
        if (G <= std::max(2.0 * (double)n, 65536.0)) {
            dense = sc.get<uint2>("shard_dense", (size_t)G);
            CK(cudaMemsetAsync(dense, 0, sizeof(uint2) * (size_t)G, s));
            k_dense_insert<<<grid_for(n, 256, nsm), 256, 0, s>>>(res_keys, cbegin, small + 0, sh, d, hp.bits - l, dd,
                                                                  dense); ++launches;
        } else {
            uint32_t H = 1;
            while (H < 2 * nc) H <<= 1;
            slot = sc.get<uint4>("shard_hslot", H);
            CK(cudaMemsetAsync(slot, 0xff, sizeof(uint4) * H, s));
            k_hash_insert<<<grid_for(nc, 256, nsm), 256, 0, s>>>(res_keys, cbegin, small + 0, sh, slot, H - 1);
            ++launches;
            hmask = H - 1;
        }
        uint32_t *around = sc.get<uint32_t>("shard_around" + std::to_string(j), nc);
        k_cell_around<<<grid_for(nc, 256, nsm), 256, 0, s>>>(res_keys, cbegin, small + 0, sh, d, hp.bits - l, dd, cm,
                                                              dense, slot, hmask, around); ++launches;
        qa.idx[j] = idx;
        qa.around[j] = around;
    }
    float *qcost = sc.get<float>("shard_qcost", n);
    k_query_costs<<<grid_for(n, 256, nsm), 256, 0, s>>>(lvl, n, K, qa, qcost); ++launches;
    CK(cudaGetLastError());
    std::vector<float> hq(n);
    CK(cudaMemcpyAsync(hq.data(), qcost, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // equal shares of the total cost, cut between queries
    std::vector<double> cum(n + 1, 0.0);
    for (int64_t q = 0; q < n; ++q) cum[q + 1] = cum[q] + (double)hq[q];
    const double total = cum[n];
    bounds[0] = 0;
    bounds[nshards] = n;
    for (int sh = 1; sh < nshards; ++sh) {
        const double target = total * (double)sh / (double)nshards;
        const int64_t p = (int64_t)(std::lower_bound(cum.begin(), cum.end(), target) - cum.begin());
        bounds[sh] = std::max<int64_t>(bounds[sh - 1], std::min<int64_t>(p, n));
    }
    if (costs)
        for (int sh = 0; sh < nshards; ++sh) costs[sh] = cum[bounds[sh + 1]] - cum[bounds[sh]];
}

void validate_sizes(int64_t n, int d, int K);

void validate(const float *points, int64_t n, int d, int K, const int32_t *ids, const double *dist)
{
    if (!points || !ids || !dist) fail(KNN_ERR_INVALID, "NULL pointer argument");
    validate_sizes(n, d, K);
}

void validate_sizes(int64_t n, int d, int K)
{
    if (n < 2) fail(KNN_ERR_INVALID, "n must be >= 2");
    if (n > 2147483647LL) fail(KNN_ERR_INVALID, "n must be <= 2^31 - 1");
    if (d < 1 || d > MAX_DIM) fail(KNN_ERR_INVALID, "d must be in [1, 8]");
    if (K < 1 || K > 256) fail(KNN_ERR_INVALID, "K must be in [1, 256]");
    if ((int64_t)K > n - 1) fail(KNN_ERR_INVALID, "K must be <= n - 1");
}

void validate_join(const float *queries, int64_t nq, const float *points, int64_t n, int d, int K,
                   const int32_t *ids, const double *dist)
{
    if (!queries || !points || !ids || !dist) fail(KNN_ERR_INVALID, "NULL pointer argument");
    if (nq < 1) fail(KNN_ERR_INVALID, "nq must be >= 1");
    if (n < 2) fail(KNN_ERR_INVALID, "n must be >= 2");
    if (n > 2147483647LL || nq > 2147483647LL) fail(KNN_ERR_INVALID, "n and nq must be <= 2^31 - 1");
    if (d < 1 || d > MAX_DIM) fail(KNN_ERR_INVALID, "d must be in [1, 8]");
    if (K < 1 || K > 256) fail(KNN_ERR_INVALID, "K must be in [1, 256]");
    if ((int64_t)K > n) fail(KNN_ERR_INVALID, "K must be <= n");
}

}  // namespace

// ---------------------------------------------------------------------------
// Context and serving queue
// ---------------------------------------------------------------------------
// Job of the serving queue (or one job of a blocking batch).
struct Batch {
    int left = 0;
    knnjoin_status first = KNN_OK;
    std::string err;
};

struct Job {
    uint64_t id = 0;
    knnjoin_job job{};
    std::atomic<int> state{0};  // 0 queued, 1 running, 2 done, 3 cancelled
    knnjoin_status status = KNN_OK;
    std::string err;
    knnjoin_stats stats{};
    size_t footprint = 0;
    std::shared_ptr<Batch> batch;  // set for jobs of a blocking batch
    std::chrono::steady_clock::time_point t_submit, t_start, t_end;
};

// A worker: its own stream, scratch and host thread; workers run jobs
// concurrently so one job's host round trips and small kernels overlap with
// another's scan.
struct Worker {
    Pipeline pipe;
    cudaStream_t stream = nullptr;
    cudaStream_t stream_hi = nullptr;  // highest priority (knnjoin_config.large_first)
    std::thread th;
};

struct knnjoin_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Allocator al;
    Pipeline main;
    std::string err;
    knnjoin_config cfg{};
    // worker pool (batched and served joins)
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Job>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Job>> jobs;
    std::vector<std::unique_ptr<Worker>> workers;
    uint64_t next_id = 1;
    bool stop = false;
    int nworkers = 8;
    int max_jobs = 1024;
    size_t budget = 0, in_use = 0;
    std::mutex big_token;  // see Pipeline::big_token
    TuneTable tune;
    std::vector<knnjoin_index *> indexes;  // live resident indexes (under g_idx_mu)
    std::mutex err_mu;                     // index queries writing err
    // batches scanned together (batch_union): one pipeline (stream, scratch)
    // per join of the largest batch so far, and the coordinator
    std::mutex union_mu;                   // one such batch at a time
    std::vector<std::unique_ptr<Pipeline>> upipes;
    std::unique_ptr<UnionScan> ucoord;
};

// Resident index: one data set indexed once on its own pipeline (stream and
// scratch), answering R x S queries until destroyed.
struct knnjoin_index {
    knnjoin_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    Pipeline pipe;
    std::mutex mu;  // one query at a time
    std::string err;
    int64_t n = 0;
    int d = 0;
    int K = 0;
};

// Every live index of every context, so that destroying an index twice (or
// after its context) is detected without touching freed memory.
static std::mutex g_idx_mu;
static std::set<knnjoin_index *> g_idx_live;

static void index_free(knnjoin_index *ix)
{
    cudaSetDevice(ix->ctx->device);
    if (ix->stream) {
        cudaStreamSynchronize(ix->stream);
        ix->pipe.release();
        cudaStreamSynchronize(ix->stream);
        cudaStreamDestroy(ix->stream);
    }
    delete ix;
}

// Device memory a join of n points holds while it runs (an estimate: the
// scratch of one pipeline, two levels of cell maps, and staging copies of
// host buffers).
static size_t job_footprint(const knnjoin_job &j)
{
    const size_t n = (size_t)std::max<int64_t>(j.n, 0);
    size_t H = 1;
    while (H < 2 * n) H <<= 1;
    size_t b = n * (size_t)(4 * j.d + 4 * pad_dim(std::max(1, std::min(j.d, MAX_DIM))) + 24 + 76) + 2 * H * 16;
    b += 32 * std::min<size_t>(n, 65536) + 8192;  // sampled-distance rows
    if (!is_device_ptr(j.points)) b += n * (size_t)j.d * 4;
    if (!is_device_ptr(j.out_ids)) b += n * (size_t)j.K * 4;
    if (!is_device_ptr(j.out_dist)) b += n * (size_t)j.K * 8;
    return b + ((size_t)1 << 20);
}

static void worker_loop(knnjoin_ctx *ctx, Worker *w)
{
    for (;;) {
        std::shared_ptr<Job> j;
        {
            std::unique_lock<std::mutex> lk(ctx->mu);
            for (;;) {
                if (ctx->stop) return;
                while (!ctx->queue.empty() && ctx->queue.front()->state.load() == 3) ctx->queue.pop_front();
                if (!ctx->queue.empty()) {
                    auto &f = ctx->queue.front();
                    // admission by HBM footprint (the head of the queue waits
                    // until it fits; a job runs alone if it never fits)
                    if (ctx->in_use == 0 || ctx->in_use + f->footprint <= ctx->budget) break;
                }
                ctx->cv.wait(lk);
            }
            j = ctx->queue.front();
            ctx->queue.pop_front();
            j->state.store(1);
            ctx->in_use += j->footprint;
            j->t_start = std::chrono::steady_clock::now();
        }
        knnjoin_status st = KNN_OK;
        std::string msg;
        try {
            // large joins first (optional): their launches go to the worker's
            // high-priority stream; the previous join on this worker has
            // finished (run() ends with a stream synchronisation)
            if (w->stream_hi) {
                const bool large = j->job.n * (int64_t)j->job.K >= Pipeline::BIG_JOB_ENTRIES;
                w->pipe.set_stream(large ? w->stream_hi : w->stream);
            }
            validate(j->job.points, j->job.n, j->job.d, j->job.K, j->job.out_ids, j->job.out_dist);
            w->pipe.run(j->job.points, j->job.n, j->job.d, j->job.K, j->job.out_ids, j->job.out_dist);
        } catch (const KnnError &e) {
            st = e.st;
            msg = e.msg;
        } catch (const std::exception &e) {
            st = KNN_ERR_NOMEM;
            msg = e.what();
        }
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            ctx->in_use -= j->footprint;
            j->t_end = std::chrono::steady_clock::now();
            j->status = st;
            j->err = msg;
            j->stats = w->pipe.stats;
            j->stats.ms_queue = std::chrono::duration<double, std::milli>(j->t_start - j->t_submit).count();
            j->stats.ms_wall = std::chrono::duration<double, std::milli>(j->t_end - j->t_submit).count();
            if (j->batch) {
                if (st != KNN_OK && j->batch->first == KNN_OK) {
                    j->batch->first = st;
                    j->batch->err = msg;
                }
                j->batch->left--;
            }
            j->state.store(2);
        }
        ctx->cv.notify_all();
    }
}

static void start_workers(knnjoin_ctx *ctx)
{
    if (!ctx->workers.empty()) return;
    for (int i = 0; i < ctx->nworkers; ++i) {
        auto w = std::make_unique<Worker>();
        CK(cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking));
        if (ctx->cfg.large_first) {
            int lo = 0, hi = 0;
            CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
            CK(cudaStreamCreateWithPriority(&w->stream_hi, cudaStreamNonBlocking, hi));
        }
        w->pipe.init(ctx->device, w->stream, &ctx->al);
        w->pipe.big_token = &ctx->big_token;
        w->pipe.width_mult = ctx->main.width_mult;
        w->pipe.tune = &ctx->tune;
        w->pipe.policy = ctx->main.policy;
        w->pipe.tail_queries = ctx->main.tail_queries;
        w->pipe.out_chunk_bytes = ctx->main.out_chunk_bytes;
        ctx->workers.push_back(std::move(w));
    }
    for (auto &w : ctx->workers) {
        Worker *wp = w.get();
        w->th = std::thread([ctx, wp] {
            cudaSetDevice(ctx->device);
            worker_loop(ctx, wp);
        });
    }
}

// A batch with its joins scanned together (knnjoin_config.batch_union): T =
// min(jobs, workers or 64) host threads, each with a pipeline of its own,
// take joins in job order and run them, every pass's scan through the
// coordinator (a thread stays a member of the union while it has joins to
// run).  Blocks until every join is done; the first failure (in job order)
// is reported.
static void run_union_batch(knnjoin_ctx *ctx, const knnjoin_job *jobs, int njobs)
{
    std::lock_guard<std::mutex> blk(ctx->union_mu);
    CK(cudaSetDevice(ctx->device));
    if (!ctx->ucoord) {
        std::unique_ptr<UnionScan> u(new UnionScan());
        cudaStream_t us = nullptr;
        CK(cudaStreamCreateWithFlags(&us, cudaStreamNonBlocking));
        u->co.init(ctx->device, us, &ctx->al);
        CK(cudaEventCreateWithFlags(&u->done, cudaEventDisableTiming));
        ctx->ucoord = std::move(u);
    }
    const int T = std::min(njobs, ctx->cfg.workers > 0 ? ctx->cfg.workers : 64);
    while ((int)ctx->upipes.size() < T) {
        std::unique_ptr<Pipeline> P(new Pipeline());
        cudaStream_t ps = nullptr;
        CK(cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking));
        P->init(ctx->device, ps, &ctx->al);
        P->width_mult = ctx->main.width_mult;
        P->tune = &ctx->tune;
        P->policy = ctx->main.policy;
        P->tail_queries = ctx->main.tail_queries;
        P->out_chunk_bytes = ctx->main.out_chunk_bytes;
        ctx->upipes.push_back(std::move(P));
    }
    UnionScan &U = *ctx->ucoord;
    U.members = T;
    U.arrived = 0;
    U.err = KNN_OK;
    U.msg.clear();
    U.entries.clear();
    std::vector<knnjoin_status> st(njobs, KNN_OK);
    std::vector<std::string> ms(njobs);
    std::atomic<int> next{0};
    std::vector<std::thread> th;
    th.reserve(T);
    for (int t = 0; t < T; ++t)
        th.emplace_back([&, t] {
            cudaSetDevice(ctx->device);
            Pipeline &P = *ctx->upipes[t];
            P.uscan = &U;
            for (int j = next++; j < njobs; j = next++) {
                try {
                    P.run(jobs[j].points, jobs[j].n, jobs[j].d, jobs[j].K, jobs[j].out_ids, jobs[j].out_dist);
                } catch (const KnnError &e) {
                    st[j] = e.st;
                    ms[j] = e.msg;
                } catch (const std::exception &e) {
                    st[j] = KNN_ERR_INVALID;
                    ms[j] = e.what();
                }
            }
            P.uscan = nullptr;
            U.leave();
        });
    for (auto &t : th) t.join();
    for (int j = 0; j < njobs; ++j)
        if (st[j] != KNN_OK) fail(st[j], "job " + std::to_string(j) + ": " + ms[j]);
}

// Run f, map its exception to a status and put the message in the
// context's error string (or in *msg when given).
static knnjoin_status guard(knnjoin_ctx *ctx, const std::function<void()> &f, std::string *msg = nullptr)
{
    std::string *err = msg ? msg : (ctx ? &ctx->err : nullptr);
    try {
        f();
        if (err) err->clear();
        return KNN_OK;
    } catch (const KnnError &e) {
        if (err) *err = e.msg;
        return e.st;
    } catch (const std::bad_alloc &) {
        if (err) *err = "host allocation failed";
        return KNN_ERR_NOMEM;
    } catch (const std::exception &e) {
        if (err) *err = e.what();
        return KNN_ERR_INVALID;
    }
}

#ifdef KNN_PHASE_TIMING
// Diagnostic builds only: read (and optionally clear) the scan kernel's
// phase cycles and item figures (out[0..16)) and event counts (out[16..32)),
// summed over the kernel's units (scan2_debug.cuh).
extern "C" int knnjoin_debug_phases(unsigned long long *out, int reset)
{
    for (int i = 0; i < 32; ++i) out[i] = 0;
    const bool r = reset != 0;
    if (scan2_debug_read<1>(out, r) != cudaSuccess || scan2_debug_read<2>(out, r) != cudaSuccess ||
        scan2_debug_read<3>(out, r) != cudaSuccess || scan2_debug_read<4>(out, r) != cudaSuccess ||
        scan2_debug_read<5>(out, r) != cudaSuccess || scan2_debug_read<6>(out, r) != cudaSuccess ||
        scan2_debug_read<7>(out, r) != cudaSuccess || scan2_debug_read<8>(out, r) != cudaSuccess)
        return 1;
    return 0;
}
#endif

extern "C" {

const char *knnjoin_version(void) { return "knnjoin-b300 0.1"; }

knnjoin_status knnjoin_create(const knnjoin_config *cfg, knnjoin_ctx **out)
{
    if (!out) return KNN_ERR_INVALID;
    *out = nullptr;
    knnjoin_ctx *ctx = new (std::nothrow) knnjoin_ctx();
    if (!ctx) return KNN_ERR_NOMEM;
    knnjoin_status st = guard(ctx, [&] {
        if (cfg) ctx->cfg = *cfg;
        int ndev = 0;
        CK(cudaGetDeviceCount(&ndev));
        if (ctx->cfg.device < 0 || ctx->cfg.device >= ndev) fail(KNN_ERR_INVALID, "no such CUDA device");
        ctx->device = ctx->cfg.device;
        CK(cudaSetDevice(ctx->device));
        if (ctx->cfg.stream) {
            ctx->stream = (cudaStream_t)ctx->cfg.stream;
        } else {
            CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
            ctx->own_stream = true;
        }
        ctx->al.alloc = ctx->cfg.alloc;
        ctx->al.free = ctx->cfg.free;
        ctx->al.user = ctx->cfg.user;
        if ((ctx->al.alloc == nullptr) != (ctx->al.free == nullptr))
            fail(KNN_ERR_INVALID, "alloc and free hooks must be given together");
        if (!ctx->al.alloc) {
            cudaMemPoolProps props;
            memset(&props, 0, sizeof(props));
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = ctx->device;
            CK(cudaMemPoolCreate(&ctx->al.pool, &props));
            uint64_t keep = ~0ull;  // keep freed memory in the pool
            CK(cudaMemPoolSetAttribute(ctx->al.pool, cudaMemPoolAttrReleaseThreshold, &keep));
        }
        ctx->main.init(ctx->device, ctx->stream, &ctx->al);
        if (ctx->cfg.width_mult > 0.0f) ctx->main.width_mult = ctx->cfg.width_mult;
        ctx->tune.fixed = ctx->cfg.width_mult > 0.0f ? ctx->cfg.width_mult : 0.0f;
        if (ctx->cfg.tune_cache_path) ctx->tune.path = ctx->cfg.tune_cache_path;
        ctx->tune.load();
        ctx->main.tune = &ctx->tune;
        if (ctx->cfg.policy < 0 || ctx->cfg.policy > 1) fail(KNN_ERR_INVALID, "policy must be 0 or 1");
        ctx->main.policy = ctx->cfg.policy;
        ctx->main.tail_queries = ctx->cfg.tail_queries;
        if (ctx->cfg.out_chunk_mb < 0) fail(KNN_ERR_INVALID, "out_chunk_mb must be >= 0");
        ctx->main.out_chunk_bytes = (size_t)ctx->cfg.out_chunk_mb << 20;
        if (ctx->cfg.max_jobs > 0) ctx->max_jobs = ctx->cfg.max_jobs;
        if (ctx->cfg.workers > 0) ctx->nworkers = std::min(ctx->cfg.workers, 64);
        size_t freeb = 0, totalb = 0;
        CK(cudaMemGetInfo(&freeb, &totalb));
        ctx->budget = ctx->cfg.hbm_budget_bytes ? ctx->cfg.hbm_budget_bytes : (size_t)(0.9 * (double)freeb);
    });
    if (st != KNN_OK) {
        knnjoin_destroy(ctx);
        return st;
    }
    *out = ctx;
    return KNN_OK;
}

void knnjoin_destroy(knnjoin_ctx *ctx)
{
    if (!ctx) return;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->stop = true;
    }
    ctx->cv.notify_all();
    for (auto &w : ctx->workers)
        if (w->th.joinable()) w->th.join();
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    {
        std::lock_guard<std::mutex> lk(g_idx_mu);
        for (knnjoin_index *ix : ctx->indexes) {
            g_idx_live.erase(ix);
            index_free(ix);
        }
        ctx->indexes.clear();
    }
    for (auto &w : ctx->workers) {
        cudaStreamSynchronize(w->stream);
        if (w->stream_hi) cudaStreamSynchronize(w->stream_hi);
        w->pipe.release();
        cudaStreamSynchronize(w->pipe.s);
        cudaStreamDestroy(w->stream);
        if (w->stream_hi) cudaStreamDestroy(w->stream_hi);
    }
    for (auto &P : ctx->upipes) {
        cudaStreamSynchronize(P->s);
        cudaStream_t ps = P->s;
        P->release();
        cudaStreamSynchronize(ps);
        cudaStreamDestroy(ps);
    }
    ctx->upipes.clear();
    if (ctx->ucoord) {
        cudaStream_t us = ctx->ucoord->co.s;
        cudaStreamSynchronize(us);
        ctx->ucoord->co.release();
        if (ctx->ucoord->done) cudaEventDestroy(ctx->ucoord->done);
        cudaStreamSynchronize(us);
        cudaStreamDestroy(us);
        ctx->ucoord.reset();
    }
    ctx->main.release();
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    if (ctx->al.pool) cudaMemPoolDestroy(ctx->al.pool);
    delete ctx;
}

knnjoin_status knnjoin_self_join(knnjoin_ctx *ctx, const float *points, int64_t n, int d, int K,
                                 int32_t *out_ids, double *out_dist)
{
    if (!ctx) return KNN_ERR_INVALID;
    return guard(ctx, [&] {
        validate(points, n, d, K, out_ids, out_dist);
        ctx->main.run(points, n, d, K, out_ids, out_dist);
    });
}

knnjoin_status knnjoin_self_join_rows(knnjoin_ctx *ctx, const float *points, int64_t n, int d, int K,
                                      int64_t row_begin, int64_t row_end, int32_t *out_ids, double *out_dist)
{
    if (!ctx) return KNN_ERR_INVALID;
    return guard(ctx, [&] {
        validate(points, n, d, K, out_ids, out_dist);
        if (row_begin < 0 || row_begin >= row_end || row_end > n)
            fail(KNN_ERR_INVALID, "rows must satisfy 0 <= row_begin < row_end <= n");
        ctx->main.run(points, n, d, K, out_ids, out_dist, nullptr, 0, row_begin, row_end);
    });
}

knnjoin_status knnjoin_shard_bounds(knnjoin_ctx *ctx, const float *points, int64_t n, int d, int K, int nshards,
                                    int64_t *bounds, double *costs)
{
    if (!ctx) return KNN_ERR_INVALID;
    return guard(ctx, [&] {
        if (!points || !bounds) fail(KNN_ERR_INVALID, "NULL pointer argument");
        validate_sizes(n, d, K);
        if (nshards < 1 || nshards > 4096) fail(KNN_ERR_INVALID, "nshards must be in [1, 4096]");
        if (ctx->main.policy != 0) fail(KNN_ERR_INVALID, "cost-balanced shards need the default policy");
        std::vector<int64_t> b(nshards + 1);
        std::vector<double> cs(nshards);
        ctx->main.shard_bounds(points, n, d, K, nshards, b.data(), cs.data());
        memcpy(bounds, b.data(), sizeof(int64_t) * (nshards + 1));
        if (costs) memcpy(costs, cs.data(), sizeof(double) * nshards);
    });
}

knnjoin_status knnjoin_index_dump(knnjoin_ctx *ctx, const float *points, int64_t n, int d, int K, int level,
                                  uint64_t *keys, uint32_t *perm, double *grid, const uint64_t *probe_keys,
                                  int64_t nprobe, uint32_t *probe_runs)
{
    if (!ctx) return KNN_ERR_INVALID;
    return guard(ctx, [&] {
        if (!points) fail(KNN_ERR_INVALID, "NULL pointer argument");
        validate_sizes(n, d, K);
        if (nprobe < 0 || (nprobe > 0 && (!probe_keys || !probe_runs)))
            fail(KNN_ERR_INVALID, "probe keys and runs must be given together (nprobe >= 0)");
        if ((keys && is_device_ptr(keys)) || (perm && is_device_ptr(perm)) || (grid && is_device_ptr(grid)) ||
            (nprobe > 0 && (is_device_ptr(probe_keys) || is_device_ptr(probe_runs))))
            fail(KNN_ERR_INVALID, "the dump's buffers must be host memory");
        ctx->main.index_dump(points, n, d, K, level, keys, perm, grid, probe_keys, nprobe, probe_runs);
    });
}

knnjoin_status knnjoin_self_join_range(knnjoin_ctx *ctx, const float *points, int64_t n, int d, int K,
                                       int64_t pos_begin, int64_t pos_end, int64_t *out_rows, int32_t *out_ids,
                                       double *out_dist)
{
    if (!ctx) return KNN_ERR_INVALID;
    return guard(ctx, [&] {
        validate(points, n, d, K, out_ids, out_dist);
        if (!out_rows) fail(KNN_ERR_INVALID, "NULL pointer argument");
        if (pos_begin < 0 || pos_begin >= pos_end || pos_end > n)
            fail(KNN_ERR_INVALID, "positions must satisfy 0 <= pos_begin < pos_end <= n");
        if (ctx->main.policy != 0) fail(KNN_ERR_INVALID, "cost-balanced shards need the default policy");
        Pipeline &P = ctx->main;
        P.shard_sorted = true;
        P.shard_rows_out = out_rows;
        try {
            P.run(points, n, d, K, out_ids, out_dist, nullptr, 0, pos_begin, pos_end);
        } catch (...) {
            P.shard_sorted = false;
            P.shard_rows_out = nullptr;
            throw;
        }
        P.shard_sorted = false;
        P.shard_rows_out = nullptr;
    });
}

knnjoin_status knnjoin_work_queue(knnjoin_ctx *ctx, const float *points, int64_t n, int d, int K, int64_t *out_sizes,
                                  int64_t cap, int64_t *out_len)
{
    if (!ctx) return KNN_ERR_INVALID;
    return guard(ctx, [&] {
        if (!points || !out_sizes || !out_len) fail(KNN_ERR_INVALID, "NULL pointer argument");
        validate_sizes(n, d, K);
        Pipeline &P = ctx->main;
        CK(cudaSetDevice(P.device));
        int32_t *ids = P.sc.get<int32_t>("queue_ids", (size_t)n * K);
        double *dist = P.sc.get<double>("queue_dist", (size_t)n * K);
        std::vector<int64_t> q;
        P.queue_out = &q;
        try {
            P.run(points, n, d, K, ids, dist);
        } catch (...) {
            P.queue_out = nullptr;
            throw;
        }
        P.queue_out = nullptr;
        *out_len = (int64_t)q.size();
        memcpy(out_sizes, q.data(), sizeof(int64_t) * (size_t)std::min<int64_t>(cap, (int64_t)q.size()));
    });
}

knnjoin_status knnjoin_join(knnjoin_ctx *ctx, const float *queries, int64_t nq, const float *points, int64_t n,
                            int d, int K, int32_t *out_ids, double *out_dist)
{
    if (!ctx) return KNN_ERR_INVALID;
    return guard(ctx, [&] {
        validate_join(queries, nq, points, n, d, K, out_ids, out_dist);
        ctx->main.run(points, n, d, K, out_ids, out_dist, queries, nq);
    });
}

knnjoin_status knnjoin_index_create(knnjoin_ctx *ctx, const float *points, int64_t n, int d, int K,
                                    knnjoin_index **out)
{
    if (!ctx) return KNN_ERR_INVALID;
    if (out) *out = nullptr;
    knnjoin_index *ix = nullptr;
    knnjoin_status st = guard(ctx, [&] {
        if (!points || !out) fail(KNN_ERR_INVALID, "NULL pointer argument");
        validate_sizes(n, d, K);
        CK(cudaSetDevice(ctx->device));
        ix = new knnjoin_index();
        ix->ctx = ctx;
        ix->n = n;
        ix->d = d;
        ix->K = K;
        CK(cudaStreamCreateWithFlags(&ix->stream, cudaStreamNonBlocking));
        ix->pipe.init(ctx->device, ix->stream, &ctx->al);
        ix->pipe.width_mult = ctx->main.width_mult;
        ix->pipe.tune = &ctx->tune;
        ix->pipe.tail_queries = ctx->main.tail_queries;
        // work queued on the context's stream (the points' producer) first
        CK(cudaEventRecord(ctx->main.ev[0], ctx->stream));
        CK(cudaStreamWaitEvent(ix->stream, ctx->main.ev[0], 0));
        ix->pipe.res_mode = 1;
        ix->pipe.run(points, n, d, K, nullptr, nullptr);
        ix->pipe.res_mode = 2;
    });
    if (st != KNN_OK) {
        if (ix) index_free(ix);
        return st;
    }
    {
        std::lock_guard<std::mutex> lk(g_idx_mu);
        ctx->indexes.push_back(ix);
        g_idx_live.insert(ix);
    }
    *out = ix;
    return KNN_OK;
}

knnjoin_status knnjoin_index_query(knnjoin_index *ix, const float *queries, int64_t nq, int K,
                                   int32_t *out_ids, double *out_dist)
{
    if (!ix) return KNN_ERR_INVALID;
    knnjoin_ctx *ctx = ix->ctx;
    std::lock_guard<std::mutex> lk(ix->mu);
    // queries of different indexes may run on several threads: the message
    // of a failure goes to the context under its lock, success leaves it
    knnjoin_status st = guard(nullptr, [&] {
        validate_join(queries, nq, queries, ix->n, ix->d, K, out_ids, out_dist);
        CK(cudaSetDevice(ctx->device));
        CK(cudaEventRecord(ix->pipe.ev[0], ctx->stream));
        CK(cudaStreamWaitEvent(ix->stream, ix->pipe.ev[0], 0));
        ix->pipe.run(nullptr, ix->n, ix->d, K, out_ids, out_dist, queries, nq);
        // results are complete; later work on the context's stream may use them
        CK(cudaEventRecord(ix->pipe.ev[2], ix->stream));
        CK(cudaStreamWaitEvent(ctx->stream, ix->pipe.ev[2], 0));
    }, &ix->err);
    if (st != KNN_OK) {
        std::lock_guard<std::mutex> elk(ctx->err_mu);
        ctx->err = ix->err;
    }
    return st;
}

knnjoin_status knnjoin_index_stats(knnjoin_index *ix, knnjoin_stats *out)
{
    if (!ix || !out) return KNN_ERR_INVALID;
    std::lock_guard<std::mutex> lk(ix->mu);
    *out = ix->pipe.stats;
    return KNN_OK;
}

void knnjoin_index_destroy(knnjoin_index *ix)
{
    std::lock_guard<std::mutex> lk(g_idx_mu);
    if (!g_idx_live.erase(ix)) return;  // not a live index
    auto &v = ix->ctx->indexes;
    v.erase(std::remove(v.begin(), v.end(), ix), v.end());
    {
        std::lock_guard<std::mutex> wait_query(ix->mu);
    }
    index_free(ix);
}

knnjoin_status knnjoin_autotune(knnjoin_ctx *ctx, const float *points, int64_t n, int d, int K,
                                float *best_width_mult)
{
    if (!ctx) return KNN_ERR_INVALID;
    return guard(ctx, [&] {
        if (!best_width_mult || !points) fail(KNN_ERR_INVALID, "NULL pointer argument");
        validate_sizes(n, d, K);
        Pipeline &P = ctx->main;
        int32_t *ids = P.sc.get<int32_t>("tune_ids", (size_t)n * K);
        double *dist = P.sc.get<double>("tune_dist", (size_t)n * K);
        static const float cand[] = {1.0f, 1.0625f, 1.125f, 1.1875f, 1.25f, 1.3125f, 1.4f, 1.5f, 1.625f};
        auto time_join = [&] {
            double ms = 1e300;
            for (int rep = 0; rep < 2; ++rep) {
                P.run(points, n, d, K, ids, dist);
                ms = std::min(ms, (double)P.stats.ms_total);
            }
            return ms;
        };
        // the cell-width multiplier at the default buffer size ...
        const int E0 = K + 32 <= 64 ? 2 : (K + 32 <= 128 ? 4 : 8);
        P.force_E = E0;
        float best = ctx->tune.dflt;
        double best_ms = 1e300;
        for (float c : cand) {
            P.force_wm = c;
            const double ms = time_join();
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        // ... then, at that multiplier, the next larger buffer (half as many
        // queries per work item, more room before a shrink)
        int bestE = E0;
        if (2 * E0 <= 8) {
            P.force_wm = best;
            P.force_E = 2 * E0;
            if (time_join() < best_ms) bestE = 2 * E0;
        }
        P.force_wm = 0.0f;
        P.force_E = 0;
        if (ctx->tune.fixed <= 0.0f) ctx->tune.set(d, K, n, best, bestE);
        *best_width_mult = best;
    });
}

knnjoin_status knnjoin_self_join_batch(knnjoin_ctx *ctx, const knnjoin_job *jobs, int njobs)
{
    if (!ctx) return KNN_ERR_INVALID;
    return guard(ctx, [&] {
        if (njobs < 0 || (njobs > 0 && !jobs)) fail(KNN_ERR_INVALID, "bad job list");
        for (int i = 0; i < njobs; ++i)
            validate(jobs[i].points, jobs[i].n, jobs[i].d, jobs[i].K, jobs[i].out_ids, jobs[i].out_dist);
        if (njobs == 0) return;
        // the caller's stream may hold work producing the inputs
        CK(cudaStreamSynchronize(ctx->stream));
        if (ctx->cfg.batch_union) {
            run_union_batch(ctx, jobs, njobs);
            return;
        }
        auto b = std::make_shared<Batch>();
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            start_workers(ctx);
            b->left = njobs;
            const auto now = std::chrono::steady_clock::now();
            for (int i = 0; i < njobs; ++i) {
                auto j = std::make_shared<Job>();
                j->job = jobs[i];
                j->footprint = job_footprint(jobs[i]);
                j->batch = b;
                j->t_submit = now;
                ctx->queue.push_back(j);
            }
        }
        ctx->cv.notify_all();
        std::unique_lock<std::mutex> lk(ctx->mu);
        ctx->cv.wait(lk, [&] { return b->left == 0; });
        if (b->first != KNN_OK) fail(b->first, b->err);
    });
}

knnjoin_status knnjoin_submit(knnjoin_ctx *ctx, const knnjoin_job *job, uint64_t *job_id)
{
    if (!ctx) return KNN_ERR_INVALID;
    return guard(ctx, [&] {
        if (!job || !job_id) fail(KNN_ERR_INVALID, "NULL job or job_id");
        validate(job->points, job->n, job->d, job->K, job->out_ids, job->out_dist);
        const size_t fp = job_footprint(*job);
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            if ((int)ctx->queue.size() >= ctx->max_jobs) fail(KNN_ERR_QUEUE_FULL, "serving queue is full");
            start_workers(ctx);
            auto j = std::make_shared<Job>();
            j->id = ctx->next_id++;
            j->job = *job;
            j->footprint = fp;
            j->t_submit = std::chrono::steady_clock::now();
            ctx->jobs[j->id] = j;
            ctx->queue.push_back(j);
            *job_id = j->id;
        }
        ctx->cv.notify_all();
    });
}

knnjoin_status knnjoin_poll(knnjoin_ctx *ctx, uint64_t job_id)
{
    if (!ctx) return KNN_ERR_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->jobs.find(job_id);
    if (it == ctx->jobs.end()) {
        ctx->err = "unknown job id";
        return KNN_ERR_INVALID;
    }
    int stt = it->second->state.load();
    if (stt == 0 || stt == 1) return KNN_ERR_NOT_READY;
    knnjoin_status st = stt == 3 ? KNN_ERR_CANCELLED : it->second->status;
    ctx->err = it->second->err;
    ctx->jobs.erase(it);
    return st;
}

knnjoin_status knnjoin_cancel(knnjoin_ctx *ctx, uint64_t job_id)
{
    if (!ctx) return KNN_ERR_INVALID;
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->jobs.find(job_id);
    if (it == ctx->jobs.end()) {
        ctx->err = "unknown job id";
        return KNN_ERR_INVALID;
    }
    int expect = 0;
    if (it->second->state.compare_exchange_strong(expect, 3)) return KNN_OK;
    ctx->err = "job already started";
    return KNN_ERR_INVALID;
}

knnjoin_status knnjoin_get_stats(knnjoin_ctx *ctx, uint64_t job_id, knnjoin_stats *out)
{
    if (!ctx || !out) return KNN_ERR_INVALID;
    if (job_id == 0) {
        *out = ctx->main.stats;
        return KNN_OK;
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->jobs.find(job_id);
    if (it == ctx->jobs.end()) {
        ctx->err = "unknown job id";
        return KNN_ERR_INVALID;
    }
    *out = it->second->stats;
    return KNN_OK;
}

knnjoin_status knnjoin_fp32_mismatch(knnjoin_ctx *ctx, const float *points, int64_t n, int d, int K,
                                     const int32_t *ids, const int64_t *rows, int64_t nrows,
                                     int64_t *out_counts)
{
    if (!ctx) return KNN_ERR_INVALID;
    return guard(ctx, [&] {
        if (!points || !ids || !rows || !out_counts) fail(KNN_ERR_INVALID, "NULL pointer argument");
        validate_sizes(n, d, K);
        if (nrows < 1 || nrows > 2147483647LL) fail(KNN_ERR_INVALID, "nrows must be in [1, 2^31 - 1]");
        if (is_device_ptr(rows)) fail(KNN_ERR_INVALID, "rows must be host memory");
        for (int64_t r = 0; r < nrows; ++r)
            if (rows[r] < 0 || rows[r] >= n) fail(KNN_ERR_INVALID, "row index out of range");
        Pipeline &P = ctx->main;
        CK(cudaSetDevice(P.device));
        const float *pts = points;
        if (!device_side(points, P.device, "points")) {
            float *p = P.sc.get<float>("diag_pts", (size_t)n * d);
            CK(cudaMemcpyAsync(p, points, sizeof(float) * n * d, cudaMemcpyHostToDevice, P.s));
            pts = p;
        }
        const int32_t *idd = ids;
        if (!device_side(ids, P.device, "ids")) {
            int32_t *p = P.sc.get<int32_t>("diag_ids", (size_t)n * K);
            CK(cudaMemcpyAsync(p, ids, sizeof(int32_t) * n * K, cudaMemcpyHostToDevice, P.s));
            idd = p;
        }
        int64_t *rowd = P.sc.get<int64_t>("diag_rows", (size_t)nrows);
        uint32_t *outd = P.sc.get<uint32_t>("diag_out", (size_t)nrows * 2);
        std::vector<uint32_t> outh((size_t)nrows * 2);
        CK(cudaMemcpyAsync(rowd, rows, sizeof(int64_t) * nrows, cudaMemcpyHostToDevice, P.s));
        const unsigned grid = (unsigned)std::min<int64_t>(nrows, (int64_t)P.nsm * 8);
        switch (d) {
#define KNN_RANK_CASE(D) \
    case D: k_fp32_rank<D><<<grid, RANK_CTA, 0, P.s>>>(pts, n, K, idd, rowd, nrows, outd); break;
            KNN_RANK_CASE(1) KNN_RANK_CASE(2) KNN_RANK_CASE(3) KNN_RANK_CASE(4)
            KNN_RANK_CASE(5) KNN_RANK_CASE(6) KNN_RANK_CASE(7) KNN_RANK_CASE(8)
#undef KNN_RANK_CASE
        }
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(outh.data(), outd, sizeof(uint32_t) * nrows * 2, cudaMemcpyDeviceToHost, P.s));
        CK(cudaStreamSynchronize(P.s));
        int64_t rows_wrong = 0, wrong = 0, missing = 0;
        for (int64_t r = 0; r < nrows; ++r) {
            if (outh[2 * r] == 0xffffffffu) fail(KNN_ERR_INVALID, "ids row holds an index outside [0, n) or the row itself");
            rows_wrong += outh[2 * r] != 0;
            wrong += outh[2 * r];
            missing += outh[2 * r + 1];
        }
        out_counts[0] = rows_wrong;
        out_counts[1] = wrong;
        out_counts[2] = missing;
    });
}

const char *knnjoin_last_error(knnjoin_ctx *ctx)
{
    if (!ctx) return "NULL context";
    return ctx->err.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Self-join without any allocation by the library.
//
// For callers that cannot allocate device memory themselves or let a
// library do it -- code running under another framework's memory pool or a
// hard memory cap, or an embedding that owns every allocation and forbids
// cudaMalloc/cudaFree behind its back.  The join's scratch (coordinates in
// SoA and key order, keys, permutation, cell tables, hash map, work items)
// lives in one fixed device array declared below; the caller passes device
// input and output buffers and a stream.
//
// Limits: n <= KNN_NOALLOC_MAX_POINTS (65,536), d <= 8, K <= 256; the array
// is NOALLOC_SCRATCH_BYTES (32 MiB) and every GPU that loads this library
// keeps it until the process exits.  All calls share the array and it keeps
// the previous call's contents (the join initialises everything it reads),
// so calls that overlap on the GPU (other threads, other streams) race and
// must be serialised by the caller.  The first call on a device does a
// one-time set-up there (it looks up the array's device address and creates
// the timing events); make that first call before any stream capture.
// ---------------------------------------------------------------------------
static constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

struct NoallocDevice {
    bool ready = false;
    unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch
    cudaEvent_t ev[5] = {};
    int nsm = 0;
};

std::mutex g_noalloc_mu;
NoallocDevice g_noalloc_dev[64];

struct Bump {
    unsigned char *base;
    size_t cap, off;
};

void *bump_alloc(size_t bytes, void *user)
{
    Bump *b = (Bump *)user;
    size_t o = (b->off + 255) & ~(size_t)255;
    if (o + bytes > b->cap) return nullptr;
    b->off = o + bytes;
    return b->base + o;
}

void bump_free(void *, void *) {}

// Worst-case upper bound of the scratch one join of n points needs.
size_t noalloc_bytes_needed(int64_t n, int d)
{
    size_t H = 1;
    while (H < (size_t)(2 * n)) H <<= 1;
    size_t b = 0;
    b += (size_t)n * d * 4 + (size_t)n * pad_dim(d) * 4;  // xs, xsort
    b += 2 * (size_t)n * 8 + 2 * (size_t)n * 4;  // keys, perm (+ alternates)
    b += 16 * ((size_t)n + 1) * 4;           // active lists, flags, scans, groups, fail
    b += (size_t)n * 8;                      // work items
    b += 4 * std::max(H * 16, std::max<size_t>(2 * (size_t)n, 65536) * 8);  // cell tables of up to four levels
    b += 3 * (size_t)n * 4 + 2 * (size_t)n;  // levels, level sort keys, window minima
    b += 256 * (((size_t)n + RS_TILE - 1) / RS_TILE) * 4 + 64 * 1024;  // histograms, sums, small
    b += sizeof(PrepReduce) + sizeof(GridParams) + 64 * 256;          // alignment slack
    return b;
}

}  // namespace

extern "C" knnjoin_status knnjoin_self_join_noalloc(const float *points, int64_t n, int d, int K,
                                                    int32_t *out_ids, double *out_dist, void *stream,
                                                    char *errbuf, size_t errlen)
{
    std::string msg;
    knnjoin_status st = KNN_OK;
    int prev_dev = -1;
    cudaGetDevice(&prev_dev);
    cudaStream_t joined_stream = nullptr;
    bool started = false;  // kernels may have been queued on the caller's stream
    try {
        validate(points, n, d, K, out_ids, out_dist);
        if (n > KNN_NOALLOC_MAX_POINTS)
            fail(KNN_ERR_INVALID, "n = " + std::to_string(n) + " exceeds the no-allocation limit of " +
                                      std::to_string(KNN_NOALLOC_MAX_POINTS) + " points");
        if (noalloc_bytes_needed(n, d) > NOALLOC_SCRATCH_BYTES)
            fail(KNN_ERR_INVALID, "problem does not fit the fixed scratch array");
        // all three buffers: device memory (not host, not managed) of the
        // GPU that holds the points, which runs the join
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, points) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
            cudaGetLastError();
            fail(KNN_ERR_INVALID, "points must be device memory (this entry point copies nothing)");
        }
        const int dev = at.device;
        if (dev < 0 || dev >= 64) fail(KNN_ERR_INVALID, "device ordinal out of range");
        const void *outs[2] = {out_ids, out_dist};
        for (const void *o : outs) {
            cudaPointerAttributes ao;
            if (cudaPointerGetAttributes(&ao, o) != cudaSuccess || ao.type != cudaMemoryTypeDevice ||
                ao.device != dev) {
                cudaGetLastError();
                fail(KNN_ERR_INVALID, "out_ids and out_dist must be device memory of the points' GPU");
            }
        }
        CK(cudaSetDevice(dev));
        joined_stream = (cudaStream_t)stream;
        NoallocDevice &D = g_noalloc_dev[dev];
        {
            std::lock_guard<std::mutex> lk(g_noalloc_mu);
            if (!D.ready) {
                void *ptr = nullptr;
                CK(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
                D.scratch = (unsigned char *)ptr;
                for (auto &e : D.ev) CK(cudaEventCreate(&e));
                CK(cudaDeviceGetAttribute(&D.nsm, cudaDevAttrMultiProcessorCount, dev));
                D.ready = true;
            }
        }
        Bump bump{D.scratch, NOALLOC_SCRATCH_BYTES, 0};
        Allocator al;
        al.alloc = bump_alloc;
        al.free = bump_free;
        al.user = &bump;
        al.nomem_msg = "fixed scratch array exhausted: this input needs the cell tables of more grid "
                       "levels than the no-allocation array holds (use knnjoin_self_join)";
        alignas(64) static thread_local uint32_t readback[1024];
        Pipeline P;
        P.device = dev;
        P.nsm = D.nsm;
        P.s = (cudaStream_t)stream;
        P.sc.al = &al;
        P.sc.stream = P.s;
        P.pinned = readback;
        for (int i = 0; i < 3; ++i) P.ev[i] = D.ev[i];
        P.evs[0] = D.ev[3];
        P.evs[1] = D.ev[4];
        // Reserve the buffers whose size varies between passes at their
        // largest, so no buffer is carved twice.
        const char *per_point[] = {"gbegin", "skey", "sval", "skey2", "sval2", "nit", "ioff", "fail", "fpos"};
        for (const char *nm : per_point) P.sc.get<uint32_t>(nm, (size_t)n + 1);
        P.sc.get<uint2>("items", (size_t)n + 1);
        P.sc.get<uint32_t>("scan_sums0", (size_t)(n + SCAN_TILE - 1) / SCAN_TILE + 2);
        P.sc.get<uint32_t>("scan_sums1", 4);
        started = true;
        P.run(points, n, d, K, out_ids, out_dist);
    } catch (const KnnError &e) {
        st = e.st;
        msg = e.msg;
    } catch (const std::exception &e) {
        st = KNN_ERR_INVALID;
        msg = e.what();
    }
    // an error part-way through a join leaves kernels queued on the caller's
    // stream that still use the shared array: wait for them, so that every
    // return (success or error) means the GPU has stopped using it
    if (st != KNN_OK && started) {
        cudaStreamSynchronize(joined_stream);
        cudaGetLastError();
    }
    if (prev_dev >= 0) cudaSetDevice(prev_dev);
    if (errbuf && errlen) {
        size_t k = std::min(errlen - 1, msg.size());
        memcpy(errbuf, msg.data(), k);
        errbuf[k] = 0;
    }
    return st;
}
