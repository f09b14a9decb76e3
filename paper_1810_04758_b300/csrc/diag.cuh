// diag.cuh -- FP32-only ranking diagnostic (not on the join's path).
//
// The join filters candidates by an FP32 squared distance and ranks them in
// canonical FP64 (Sec. 4 kernel, with the FP64 re-score of the band).  This
// kernel measures what ranking by the FP32 value alone would have returned:
// for a sampled query row i with the exact neighbour row E (K ids in exact
// order), the FP32-only row is the K smallest j != i under
// (d2_32(i, j), j), with d2_32 the same FP32 expression the scan kernels use
// (dist2_f32).  For every entry e of E the kernel finds its position in that
// FP32-only row,
//     r(e) = #{ j != i : (d2_32(i, j), j) < (d2_32(i, e), e) },
// and reports per row
//     out[2 r + 0] = #{ positions k : FP32-only row[k] != E[k] }
//     out[2 r + 1] = #{ e in E : r(e) >= K }  (ids missing from the FP32 set)
// or 0xffffffff in out[2 r + 0] when the row holds an id outside [0, n).
//
// Work: one CTA per sampled row scans all n points once.  Points whose FP32
// key lies below the largest key of E are rare (about K per row); for those
// outside E the kernel counts how many of E's sorted keys lie below them
// (H[b]), and r(E_sorted[m]) = m + sum_{b <= m} H[b].
#pragma once
#include <stdint.h>

#include "common.cuh"
#include "dist32.cuh"

namespace knn {

constexpr int RANK_CTA = 256;

template <int DIM>
__global__ void __launch_bounds__(RANK_CTA) k_fp32_rank(const float *__restrict__ pts, int64_t n, int K,
                                                        const int32_t *__restrict__ ids,
                                                        const int64_t *__restrict__ rows, int64_t nrows,
                                                        uint32_t *__restrict__ out)
{
    __shared__ uint64_t keys[256];   // FP32 keys of E in exact order
    __shared__ uint64_t S[256];      // the same keys, ascending
    __shared__ int32_t E[256];       // exact ids
    __shared__ uint16_t pos[256];    // exact position of S[m]
    __shared__ uint32_t H[257];
    __shared__ int bad;
    const int t = threadIdx.x;
    for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int64_t i = rows[r];
        float q[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) q[k] = pts[i * DIM + k];
        if (t == 0) bad = 0;
        __syncthreads();
        if (t < K) {
            const int32_t id = ids[i * K + t];
            uint64_t key = ~0ull;
            if (id >= 0 && (int64_t)id < n && (int64_t)id != i) {
                float c[DIM];
#pragma unroll
                for (int k = 0; k < DIM; ++k) c[k] = pts[(int64_t)id * DIM + k];
                key = ((uint64_t)__float_as_uint(dist2_f32<DIM>(q, c)) << 32) | (uint32_t)id;
            } else {
                bad = 1;
            }
            keys[t] = key;
            E[t] = id;
        }
        for (int b = t; b <= K; b += RANK_CTA) H[b] = 0;
        __syncthreads();
        if (t < K) {
            int m = 0;
            for (int u = 0; u < K; ++u) m += keys[u] < keys[t] || (keys[u] == keys[t] && u < t);
            S[m] = keys[t];
            pos[m] = (uint16_t)t;
        }
        __syncthreads();
        const uint64_t top = S[K - 1];
        if (!bad) {
            for (int64_t j = t; j < n; j += RANK_CTA) {
                if (j == i) continue;
                float c[DIM];
#pragma unroll
                for (int k = 0; k < DIM; ++k) c[k] = pts[j * DIM + k];
                const uint64_t key = ((uint64_t)__float_as_uint(dist2_f32<DIM>(q, c)) << 32) | (uint32_t)j;
                if (key >= top) continue;
                bool member = false;
                for (int u = 0; u < K; ++u) member |= E[u] == (int32_t)j;
                if (member) continue;
                int lo = 0, hi = K;  // number of S entries below key
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (S[mid] < key) lo = mid + 1;
                    else hi = mid;
                }
                atomicAdd(&H[lo], 1u);
            }
        }
        __syncthreads();
        if (t == 0) {
            uint32_t wrong = 0, missing = 0, below = 0;
            for (int m = 0; m < K; ++m) {
                below += H[m];
                const uint32_t rank = (uint32_t)m + below;
                wrong += rank != pos[m];
                missing += rank >= (uint32_t)K;
            }
            out[2 * r + 0] = bad ? 0xffffffffu : wrong;
            out[2 * r + 1] = bad ? 0u : missing;
        }
        __syncthreads();
    }
}

}  // namespace knn
