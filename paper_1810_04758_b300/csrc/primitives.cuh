// primitives.cuh -- prefix sums, stream compaction and LSD radix sort.
//
// Hand-written for the index build (Sec. 4.6, GPU: Indexing: the grid is built on the GPU):
// cell keys are sorted with an LSD radix sort on 8-bit digits (one pass per
// digit of the bits actually used), and cell offsets come from exclusive
// prefix sums over run flags.  Both use the reduce-then-scan pattern (no
// inter-block spin waits).
#pragma once
#include "common.cuh"

namespace knn {

// ----------------------------------------------------------------------------
// Exclusive scan of uint32 (sums must not exceed 2^32 - 1).
// ----------------------------------------------------------------------------
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const uint32_t *in, uint32_t *out,
                                                            uint32_t *sums, int64_t n)
{
    __shared__ uint32_t sm[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + i;
        v[i] = idx < n ? in[idx] : 0;
        s += v[i];
    }
    uint32_t total;
    uint32_t off = block_exclusive_scan(s, total, sm);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = off;
        off += v[i];
    }
    if (threadIdx.x == 0 && sums) sums[blockIdx.x] = total;
}

// Second half of a two-launch scan (nb <= SCAN_TILE tiles): block b adds
// the exclusive prefix of the tile sums, sum of sums[0..b), which it forms
// itself (no separate scan of the sums).
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_add_direct(uint32_t *out, const uint32_t *sums, int64_t n)
{
    __shared__ uint32_t sm[32];
    const int b = (int)blockIdx.x;
    uint32_t part = 0;
    for (int i = threadIdx.x; i < b; i += SCAN_THREADS) part += sums[i];
    uint32_t add;
    block_exclusive_scan(part, add, sm);
    const int64_t base = (int64_t)b * SCAN_TILE;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        const int64_t idx = base + i;
        if (idx < n) out[idx] += add;
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_add(uint32_t *out, const uint32_t *sums, int64_t n)
{
    uint32_t add = sums[blockIdx.x];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t idx = base + i;
        if (idx < n) out[idx] += add;
    }
}

// ----------------------------------------------------------------------------
// LSD radix sort of (key, uint32 value) pairs, 8-bit digits, stable.
// ----------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

template <typename K>
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const K *keys, int64_t n, int shift,
                                                       uint32_t *hist, int nblocks)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
        int64_t idx = base + i;
        if (idx < n) atomicAdd(&h[(uint32_t)(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: items of a tile are ranked in index order, round by round
// (256 consecutive items per round, warp-level match for equal digits).
template <typename K>
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const K *kin, const uint32_t *vin, K *kout,
                                                          uint32_t *vout, int64_t n, int shift,
                                                          const uint32_t *offs, int nblocks)
{
    __shared__ uint32_t base_off[256];
    __shared__ uint32_t wcnt[RS_THREADS / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base_off[tid] = offs[(int64_t)tid * nblocks + blockIdx.x];
    int64_t tile = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
        int64_t idx = tile + (int64_t)r * RS_THREADS + tid;
        bool valid = idx < n;
        K k = valid ? kin[idx] : (K)0;
        uint32_t v = valid ? vin[idx] : 0u;
        uint32_t dg = valid ? ((uint32_t)(k >> shift) & 255u) : (256u + lane);
#pragma unroll
        for (int w = 0; w < RS_THREADS / 32; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        uint32_t peers = __match_any_sync(FULL, dg);
        uint32_t rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) wcnt[warp][dg] = __popc(peers);
        __syncthreads();
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < RS_THREADS / 32; ++w) {
            uint32_t c = wcnt[w][tid];
            wcnt[w][tid] = run;
            run += c;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = base_off[dg] + wcnt[warp][dg] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        base_off[tid] += run;
        __syncthreads();
    }
}

}  // namespace knn
