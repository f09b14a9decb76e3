// common.cuh -- shared definitions of the B300 KNN self-join kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "exact.cuh"

namespace knn {

constexpr unsigned FULL = 0xffffffffu;

// Checked build (-DKNN_CHECKS, build.py build_checked): guarded accesses test
// their index first; a failed test sets bit `site` of g_check_word and the
// access is skipped.  The host reads and clears the word after every join.
// In the normal build a guard is the constant true and compiles away.
#ifdef KNN_CHECKS
__device__ unsigned int g_check_word;
__device__ __forceinline__ bool knn_guard(bool ok, int site)
{
    if (!ok) atomicOr(&g_check_word, 1u << site);
    return ok;
}
#define KNN_GUARD(cond, site) (::knn::knn_guard((cond), (site)))
#else
#define KNN_GUARD(cond, site) (true)
#endif
constexpr int MAX_DIM = 8;
constexpr int MAX_LEVELS = 26;  // grid levels 0 .. 25 (at most 24 key bits per dimension)

// Coordinates in key order are stored AoS, each point padded to 2, 4 or 8
// floats (8, 16 or 32 bytes: one or two aligned vector loads per point).
__host__ __device__ constexpr int pad_dim(int d) { return d <= 2 ? 2 : (d <= 4 ? 4 : 8); }

// Per-join parameters computed on the device (steps a1-a2) and read back.
struct GridParams {
    int n, d, K;
    float lo[MAX_DIM], hi[MAX_DIM];  // bounding box (face origin = lo)
    int fixed_ok;                    // every coordinate is X * 2^-F, |X| < 2^30
    int F;
    float eps_mean, eps_min;         // Sec. 4.4 search distance
    float w0, inv_w0;                // level-0 cell side
    int cmax0[MAX_DIM];              // largest level-0 cell index per dimension
    int bits;                        // bits per dimension of the Morton key
    int key_bits;                    // d * bits
    int top_level;                   // level at which the grid is one cell
    int start_level;                 // level of the first pass
    int finer;                       // levels below the search-distance width
    int nonfinite;                   // input holds NaN / Inf
};

// Reductions of step a1 (atomics targets).
struct PrepReduce {
    unsigned lo_enc[MAX_DIM], hi_enc[MAX_DIM];
    int min_lsb, max_msb;
    int nonfinite;
    int pad;
    double eps_sum;
    unsigned long long eps_pairs;
    unsigned hist[2][1024];
    unsigned scount[256];            // sampled points' neighbours within eps_min
};

// Order-preserving float <-> uint32 encodings (for atomicMin/Max on floats).
__device__ __forceinline__ unsigned fenc(float f)
{
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ __forceinline__ float fdec(unsigned u)
{
    unsigned v = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
#ifdef __CUDA_ARCH__
    return __uint_as_float(v);
#else
    return bitsf(v);
#endif
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Level-0 cell of coordinate x: the largest c in [0, limit] whose lower face
// fmaf(c, w, o) is <= x.  Faces are exact float values, strictly increasing in
// c (the cell side is at least 2^-21 of the largest face magnitude), so the
// assignment is exact and the certificate can use the very same faces.
__device__ __forceinline__ int cell_of(float x, float o, float w, float invw, int limit)
{
    float f = floorf((x - o) * invw);
    f = fminf(fmaxf(f, 0.0f), (float)limit);
    int c = (int)f;
    while (c > 0 && fmaf((float)c, w, o) > x) --c;
    while (c < limit && fmaf((float)(c + 1), w, o) <= x) ++c;
    return c;
}

__device__ __forceinline__ float face_of(int c, float o, float w)
{
    return fmaf((float)c, w, o);
}

// Morton interleave of d coordinates with `nb` bits each (bit b of
// coordinate j goes to key bit b*d + j).
__device__ __forceinline__ uint64_t morton_encode(const int *c, int d, int nb)
{
    uint64_t key = 0;
    for (int b = 0; b < nb; ++b)
        for (int j = 0; j < d; ++j)
            key |= (uint64_t)((c[j] >> b) & 1) << (b * d + j);
    return key;
}

__device__ __forceinline__ void morton_decode(uint64_t key, int d, int nb, int *c)
{
    for (int j = 0; j < d; ++j) c[j] = 0;
    for (int b = 0; b < nb; ++b)
        for (int j = 0; j < d; ++j)
            c[j] |= (int)((key >> (b * d + j)) & 1) << b;
}

// Positive normal float -> IEEE double bit pattern; subnormals and zero map
// to +0 (callers use this as a lower bound).
__device__ __forceinline__ uint64_t f32_to_f64_bits_floor(float f)
{
    uint32_t b = __float_as_uint(f);
    uint32_t e8 = b >> 23;
    if (e8 == 0 || (b >> 31)) return 0;
    return ((uint64_t)(e8 - 127 + 1023) << 52) | ((uint64_t)(b & 0x7fffffu) << 29);
}

// Hash map (open addressing, linear probing) from level cell key to its run
// [begin, end) in key order.  One 16-byte slot per entry -- key (x, y),
// begin (z), end (w) -- so a probe is a single vector load.  Capacity is a
// power of two >= 2 x cells.  Built by k_hash_insert (grid.cuh).
constexpr uint64_t HASH_EMPTY = ~0ull;

__device__ __forceinline__ uint2 hash_lookup(const uint4 *__restrict__ slot, uint32_t hmask, uint64_t P)
{
    uint32_t h = (uint32_t)mix64(P) & hmask;
    for (uint32_t probe = 0; probe <= hmask; ++probe) {
        const uint4 v = __ldg(&slot[h]);
        const uint64_t k = (uint64_t)v.x | ((uint64_t)v.y << 32);
        if (k == P) return make_uint2(v.z, v.w);
        if (k == HASH_EMPTY) break;
        h = (h + 1) & hmask;
    }
    return make_uint2(0, 0);
}

// Block-wide exclusive scan of one value per thread; `sm` holds >= 32 words.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t &total, uint32_t *sm)
{
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? sm[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        sm[lane] = w;
    }
    __syncthreads();
    uint32_t off = warp ? sm[warp - 1] : 0;
    total = sm[nw - 1];
    __syncthreads();
    return off + x - v;
}

// Dense cell table of one grid level (used instead of the hash map when the
// level's grid is small): entry c = (begin, end) of the run of the cell whose
// level coordinates are c_0..c_{d-1}, index sum_k c_k * stride_k with
// stride_0 = 1 and stride_k = stride_{k-1} * (cells in dimension k - 1);
// cells without points hold (0, 0).
__device__ __forceinline__ bool xless(uint64_t da, uint32_t ia, uint64_t db, uint32_t ib)
{
    return da < db || (da == db && ia < ib);
}

// Bitonic sort, ascending by (D, I), of 32*E entries held E per lane in
// blocked order (entry g = lane*E + e).
template <int E>
__device__ __forceinline__ void warp_bitonic(uint64_t (&D)[E], uint32_t (&I)[E], int lane)
{
    constexpr int N = 32 * E;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j < E) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int p = e ^ j;
                    if (p > e) {
                        const int g = lane * E + e;
                        const bool up = (g & k) == 0;
                        const bool sw = up ? xless(D[p], I[p], D[e], I[e]) : xless(D[e], I[e], D[p], I[p]);
                        if (sw) {
                            uint64_t td = D[e]; D[e] = D[p]; D[p] = td;
                            uint32_t ti = I[e]; I[e] = I[p]; I[p] = ti;
                        }
                    }
                }
            } else {
                const int lm = j / E;
                const bool lower = (lane & lm) == 0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    uint64_t od = __shfl_xor_sync(FULL, D[e], lm);
                    uint32_t oi = __shfl_xor_sync(FULL, I[e], lm);
                    const int g = lane * E + e;
                    const bool up = (g & k) == 0;
                    const bool take = (lower == up) ? xless(od, oi, D[e], I[e]) : xless(D[e], I[e], od, oi);
                    if (take) {
                        D[e] = od;
                        I[e] = oi;
                    }
                }
            }
        }
    }
}

struct DenseDims {
    uint32_t stride[MAX_DIM];
};

}  // namespace knn
