// grid.cuh -- index construction on the GPU (paper Sec. 3.1, 4.3, 4.4, 4.5).
//
//  a1  k_prep        AoS -> SoA, bounding box, fixed-point frame, finiteness.
//  a2  k_eps_pairs   mean distance among ~0.1% sampled points (eps_mean).
//      k_eps_hist    histogram of sampled distances below eps_mean (n_bins
//                    bins), twice: over [0, eps_mean), then refined over
//                    [0, 2 x the first estimate).
//      k_params      eps_min = middle of the first bin whose cumulative count
//                    reaches K per sampled point; cell side, grid, key bits.
//  a3  k_keys        exact level-0 cell of every point, Morton key.
//  a4  radix sort (primitives.cuh).
//  a5  k_gather      coordinates permuted to key order (padded AoS rows).
//      k_run_flags / k_run_begin / k_dense_insert / k_hash_insert: the
//                    non-empty cells of a level (a level-l cell is a run of
//                    equal key >> (d*l)) and a dense table or a hash map from
//                    cell to its run.
//  a6  k_group_*     density-ordered work queue: groups of queries sharing a
//                    cell, sorted by count descending (Fig. 4), split into
//                    work items.
#pragma once
#include "common.cuh"

namespace knn {

// ---------------------------------------------------------------------------
// a1
// ---------------------------------------------------------------------------
__global__ void k_prep(const float *__restrict__ pts, int64_t n, int d, float *__restrict__ xs,
                       PrepReduce *red)
{
    float lmin[MAX_DIM], lmax[MAX_DIM];
    for (int k = 0; k < MAX_DIM; ++k) {
        lmin[k] = __int_as_float(0x7f800000);
        lmax[k] = -__int_as_float(0x7f800000);
    }
    int lsb = 1 << 30, msb = -(1 << 30), bad = 0;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        for (int k = 0; k < d; ++k) {
            float x = pts[i * d + k];
            xs[(int64_t)k * n + i] = x;
            if (!isfinite(x)) {
                bad = 1;
                continue;
            }
            lmin[k] = fminf(lmin[k], x);
            lmax[k] = fmaxf(lmax[k], x);
            if (x != 0.0f) {
                uint32_t M;
                int E;
                fdecode(x, M, E);
                lsb = min(lsb, E + (__ffs(M) - 1));
                msb = max(msb, E + 31 - __clz(M));
            }
        }
    }
    for (int k = 0; k < d; ++k) {
        float a = lmin[k], b = lmax[k];
        for (int o = 16; o; o >>= 1) {
            a = fminf(a, __shfl_xor_sync(FULL, a, o));
            b = fmaxf(b, __shfl_xor_sync(FULL, b, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&red->lo_enc[k], fenc(a));
            atomicMax(&red->hi_enc[k], fenc(b));
        }
    }
    for (int o = 16; o; o >>= 1) {
        lsb = min(lsb, __shfl_xor_sync(FULL, lsb, o));
        msb = max(msb, __shfl_xor_sync(FULL, msb, o));
        bad |= __shfl_xor_sync(FULL, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&red->min_lsb, lsb);
        atomicMax(&red->max_msb, msb);
        if (bad) atomicOr(&red->nonfinite, 1);
    }
}

// ---------------------------------------------------------------------------
// a2: search distance.  Samples are taken at fixed strides (deterministic).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dist_f32(const float *xs, int64_t n, int d, int64_t i, int64_t j)
{
    float s = 0.0f;
    for (int k = 0; k < d; ++k) {
        float t = xs[(int64_t)k * n + i] - xs[(int64_t)k * n + j];
        s = fmaf(t, t, s);
    }
    return sqrtf(s);
}

// Mean distance over all pairs of `sm` points at stride n / sm.
__global__ void k_eps_pairs(const float *xs, int64_t n, int d, int64_t sm, PrepReduce *red)
{
    int64_t stride = n / sm;
    float acc = 0.0f;
    unsigned long long cnt = 0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < sm * sm;
         p += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = p / sm, b = p % sm;
        if (b >= a) continue;
        acc += dist_f32(xs, n, d, a * stride, b * stride);
        ++cnt;
    }
    for (int o = 16; o; o >>= 1) {
        acc += __shfl_xor_sync(FULL, acc, o);
        cnt += __shfl_xor_sync(FULL, cnt, o);
    }
    if ((threadIdx.x & 31) == 0 && cnt) {
        atomicAdd(&red->eps_sum, (double)acc);
        atomicAdd(&red->eps_pairs, cnt);
    }
}

// Rows of the S sample points (stride n / S) and of the m subset points
// (stride n / m), 8 floats each (zero padded), for the sampled-distance
// kernels below.
__global__ void k_eps_rows(const float *__restrict__ xs, int64_t n, int d, int64_t S, int64_t m,
                           float *__restrict__ srow, float *__restrict__ mrow)
{
    const int64_t sstride = n / S, mstride = n / m;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < S + m;
         t += (int64_t)gridDim.x * blockDim.x) {
        const bool smp = t < S;
        const int64_t i = smp ? t * sstride : (t - S) * mstride;
        float *row = smp ? srow + t * 8 : mrow + (t - S) * 8;
        for (int k = 0; k < 8; ++k) row[k] = k < d ? xs[(int64_t)k * n + i] : 0.0f;
    }
}

// Squared distance of two sampled rows over their first P floats (P = 4
// for d <= 4, else 8).  The rows are zero beyond d, and fmaf(0, 0, s) = s,
// so this is the d-term sum exactly.
template <int P>
__device__ __forceinline__ float row_d2(const float4 *a, const float (&b)[P])
{
    float s = 0.0f;
#pragma unroll
    for (int v = 0; v < P / 4; ++v) {
        const float4 t = a[v];
        const float x[4] = {t.x - b[4 * v], t.y - b[4 * v + 1], t.z - b[4 * v + 2], t.w - b[4 * v + 3]};
#pragma unroll
        for (int k = 0; k < 4; ++k) s = fmaf(x[k], x[k], s);
    }
    return s;
}

// A bound every s with sqrtf(s) < r lies below: sqrtf rounds correctly and r
// is a float, so sqrtf(s) < r means sqrt(s) < r, i.e. s < r^2 <= this bound
// (r^2 (1 + 2^-20), rounded up).  Larger s skip the square root.
__device__ __forceinline__ float below_bound(float r) { return __fmul_ru(__fmul_ru(r, r), 1.0f + 0x1p-20f); }

// The sample index of subset point j's own point (-1 if it is not a sample).
__device__ __forceinline__ int64_t self_sample(int64_t j, int64_t mstride, int64_t sstride)
{
    const int64_t p = j * mstride;
    return p % sstride == 0 ? p / sstride : -1;
}

// Samples [i0, i1) of slice blockIdx.y (gridDim.y slices of the S samples).
__device__ __forceinline__ void sample_slice(int64_t S, int64_t &i0, int64_t &i1)
{
    const int64_t per = (S + gridDim.y - 1) / gridDim.y;
    i0 = (int64_t)blockIdx.y * per;
    i1 = min(S, i0 + per);
}

struct ParamsIn {
    int64_t n;
    int d, K;
    int64_t S, m;        // histogram samples / subset size
    float width_mult;    // cell side = width_mult * eps_min
    int start_level;
    int max_finer;       // cap on levels finer than the search-distance width
};

__device__ __forceinline__ float eps_mean_of(const PrepReduce *red)
{
    return red->eps_pairs ? (float)(red->eps_sum / (double)red->eps_pairs) : 0.0f;
}

// Stage 0 of the grid parameters (written by one thread): the grid-independent
// fields, from the reductions of k_prep and k_eps_pairs.
__device__ void params_stage0(const PrepReduce *red, const ParamsIn &in, GridParams *gp)
{
    const int d = in.d;
    gp->n = (int)in.n;
    gp->d = d;
    gp->K = in.K;
    gp->nonfinite = red->nonfinite;
    for (int k = 0; k < d; ++k) {
        gp->lo[k] = fdec(red->lo_enc[k]);
        gp->hi[k] = fdec(red->hi_enc[k]);
    }
    if (red->max_msb < red->min_lsb) {  // every coordinate is zero
        gp->fixed_ok = 1;
        gp->F = 0;
    } else {
        int F = -red->min_lsb;
        gp->F = F;
        gp->fixed_ok = (red->max_msb + F <= 29) ? 1 : 0;
    }
    gp->eps_mean = eps_mean_of(red);
    gp->eps_min = 0.0f;
}

// The search distance of a histogram h of bins range / 1024 (one warp, every
// lane returns it): the middle of the first bin at which the cumulative count
// per sampled point reaches K (scaled to the subset), or range if none.  Lane
// l sums bins [32 l, 32 l + 32), a warp prefix sum finds the lane whose chunk
// crosses the target, that lane finds the bin (integer sums: exact).
__device__ float params_pick(const unsigned *h, float range, const ParamsIn &in, int lane)
{
    const double target = (double)in.K * (double)in.S * (double)in.m / (double)(in.n - 1);
    unsigned long long own = 0;
    for (int b = 0; b < 32; ++b) own += h[lane * 32 + b];
    unsigned long long inc = own;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    const unsigned cross = __ballot_sync(FULL, (double)inc >= target);
    int pick = -1;
    if (cross) {
        const int src = __ffs(cross) - 1;
        if (lane == src) {
            unsigned long long cum = inc - own;
            for (int b = 0; b < 32; ++b) {
                cum += h[lane * 32 + b];
                if ((double)cum >= target) {
                    pick = lane * 32 + b;
                    break;
                }
            }
        }
        pick = __shfl_sync(FULL, pick, src);
    }
    return pick >= 0 ? (pick + 0.5f) * (range / 1024.0f) : range;
}

// Histogram of distances from the S sample points to the m subset points,
// bins of width range / 1024 over [0, range), where range = eps_mean (stage
// 0) or twice the stage-0 estimate (stage 1).  A thread holds one subset
// point and walks its block's slice of the samples (staged in shared
// memory); the block's histogram is added to the global one.
template <int P>
__global__ void k_eps_hist(const float *__restrict__ srow, const float *__restrict__ mrow, int64_t n,
                           int64_t S, int64_t m, GridParams *gp, PrepReduce *red, int stage, const ParamsIn in)
{
    __shared__ unsigned h[1024];
    __shared__ float4 sp[256 * 2];
    __shared__ float s_range;
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) h[i] = 0;
    for (int i = threadIdx.x; i < (int)S * 2; i += blockDim.x) sp[i] = ((const float4 *)srow)[i];
    // the grid parameters this stage needs, formed by every block (block
    // (0, 0) also stores them for the kernels after): stage 0, the
    // grid-independent fields and eps_mean; stage 1, the first eps_min
    // estimate from the stage-0 histogram
    const bool first = blockIdx.x == 0 && blockIdx.y == 0;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        float range;
        if (stage == 0) {
            range = eps_mean_of(red);
            if (first && lane == 0) params_stage0(red, in, gp);
        } else {
            const float e = params_pick(red->hist[0], gp->eps_mean, in, lane);
            if (first && lane == 0) gp->eps_min = e;
            range = 2.0f * e;
        }
        if (lane == 0) s_range = range;
    }
    __syncthreads();
    const float range = s_range;
    if (range > 0.0f) {
        const float inv_bw = 1024.0f / range, r2 = below_bound(range);
        const int64_t sstride = n / S, mstride = n / m;
        int64_t i0, i1;
        sample_slice(S, i0, i1);
        for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m;
             j += (int64_t)gridDim.x * blockDim.x) {
            float p[P];
#pragma unroll
            for (int k = 0; k < P; ++k) p[k] = mrow[j * 8 + k];
            const int64_t own = self_sample(j, mstride, sstride);
            for (int64_t i = i0; i < i1; ++i) {
                const float s2 = row_d2<P>(sp + i * 2, p);
                if (s2 < r2 && i != own) {
                    const float dd = sqrtf(s2);
                    if (dd < range) atomicAdd(&h[min((int)(dd * inv_bw), 1023)], 1u);
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 1024; i += blockDim.x)
        if (h[i]) atomicAdd(&red->hist[stage][i], h[i]);
}


// Density skew: neighbours of each sampled point among the subset within
// the radius where about K are expected (eps_min scaled by (n/m)^(1/d)).
// A thread holds one subset point and walks its block's slice of the
// samples; per sample, a warp ballot counts its lanes within the radius.
template <int P>
__global__ void k_eps_count(const float *__restrict__ srow, const float *__restrict__ mrow, int64_t n, int d,
                            int64_t S, int64_t m, GridParams *gp, PrepReduce *red, const ParamsIn in)
{
    __shared__ unsigned cnt[256];
    __shared__ float4 sp[256 * 2];
    __shared__ float s_eps;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) cnt[i] = 0;
    for (int i = threadIdx.x; i < (int)S * 2; i += blockDim.x) sp[i] = ((const float4 *)srow)[i];
    // stage 2 of the grid parameters, formed by every block (block 0 also
    // stores it): eps_min refined from the stage-1 histogram over [0, 2 x
    // the first estimate), or eps_mean when that estimate is 0.  The first
    // estimate is formed again here from the stage-0 histogram, since block
    // 0 overwrites gp->eps_min
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const float range = 2.0f * params_pick(red->hist[0], gp->eps_mean, in, lane);
        float e = params_pick(red->hist[1], range, in, lane);
        if (!(range > 0.0f)) e = gp->eps_mean;
        if (blockIdx.x == 0 && blockIdx.y == 0 && lane == 0) gp->eps_min = e;
        if (lane == 0) s_eps = e;
    }
    __syncthreads();
    const float e = s_eps * powf((float)n / (float)m, 1.0f / (float)d);
    if (e > 0.0f && isfinite(e)) {
        const float e2 = below_bound(e);
        const int64_t sstride = n / S, mstride = n / m;
        int64_t i0, i1;
        sample_slice(S, i0, i1);
        // every lane of a warp runs the same number of rounds (ballots)
        const int64_t span = (int64_t)gridDim.x * blockDim.x;
        const int64_t first = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
        for (int64_t base = first; base < m; base += span) {
            const int64_t j = base + (threadIdx.x & 31);
            const bool valid = j < m;
            float p[P];
#pragma unroll
            for (int k = 0; k < P; ++k) p[k] = valid ? mrow[j * 8 + k] : 0.0f;
            const int64_t own = valid ? self_sample(j, mstride, sstride) : -1;
            for (int64_t i = i0; i < i1; ++i) {
                const float s2 = row_d2<P>(sp + i * 2, p);
                const bool in = valid && i != own && s2 < e2 && sqrtf(s2) < e;
                const unsigned b = __ballot_sync(FULL, in);
                if ((threadIdx.x & 31) == 0 && b) atomicAdd(&cnt[i], (unsigned)__popc(b));
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (int)S; i += blockDim.x)
        if (cnt[i]) atomicAdd(&red->scount[i], cnt[i]);
}

__device__ void k_params_grid(const PrepReduce *red, GridParams *gp, const ParamsIn &in, double csum,
                              unsigned cmaxs);

// stage 0: eps_mean and the grid-independent fields; stage 1: eps_min
// estimate from hist[0]; stage 2: refined eps_min from hist[1]; stage 3:
// density skew, cell side, grid and key bits.  One warp: the bin search and
// the sample sums are spread over the lanes (integer sums, exact in any
// order), the rest runs on lane 0.
__global__ void k_params(const PrepReduce *red, GridParams *gp, ParamsIn in, int stage)
{
    const int lane = threadIdx.x & 31;
    if (blockIdx.x || threadIdx.x >= 32) return;
    if (stage == 0) {
        if (lane == 0) params_stage0(red, in, gp);
        return;
    }
    if (stage == 3) {
        // sampled points' neighbour counts: their sum and maximum
        unsigned long long cs = 0;
        unsigned cm = 0;
        for (int i = lane; i < (int)in.S && i < 256; i += 32) {
            cs += red->scount[i];
            cm = max(cm, red->scount[i]);
        }
        for (int o = 16; o; o >>= 1) {
            cs += __shfl_xor_sync(FULL, cs, o);
            cm = max(cm, __shfl_xor_sync(FULL, cm, o));
        }
        if (lane == 0) k_params_grid(red, gp, in, (double)cs, cm);
        return;
    }
    const float range = stage == 1 ? gp->eps_mean : 2.0f * gp->eps_min;
    float eps = params_pick(red->hist[stage - 1], range, in, lane);
    if (lane) return;
    if (stage == 2 && !(range > 0.0f)) eps = gp->eps_mean;
    gp->eps_min = eps;
}

__device__ void k_params_grid(const PrepReduce *red, GridParams *gp, const ParamsIn &in, double csum,
                              unsigned cmaxs)
{
    const int d = in.d;
    const float eps = gp->eps_min;
    // cell side and grid
    float ext = 0.0f, mag = 0.0f;
    for (int k = 0; k < d; ++k) {
        ext = fmaxf(ext, gp->hi[k] - gp->lo[k]);
        mag = fmaxf(mag, fmaxf(fabsf(gp->lo[k]), fabsf(gp->hi[k])));
    }
    int bmax = min(24, 63 / d);
    // levels finer than the search-distance width, from the density skew of
    // the sampled points: the densest sample over the mean, per dimension
    int finer = 0;
    if (csum > 0.0) {
        double ratio = (double)cmaxs * (double)min((int64_t)256, in.S) / csum;
        finer = (int)floor(log2(fmax(ratio, 1.0)) / d + 0.5);
        finer = max(0, min(finer, in.max_finer));
    }
    gp->finer = finer;
    float w = in.width_mult * eps;
    if (!(w > 0.0f) || !isfinite(w)) w = ext > 0.0f ? ext : 1.0f;
    w = ldexpf(w, -finer);
    float wf1 = ldexpf(mag, -21);                            // faces strictly increasing
    float wf2 = ext / (float)((1 << bmax) - 4);              // grid fits the key bits
    w = fmaxf(w, fmaxf(wf1, wf2));
    if (!(w > 0.0f)) w = 1.0f;
    if (!isfinite(w)) w = 3.0e38f;
    gp->w0 = w;
    gp->inv_w0 = 1.0f / w;
    int cmax = 0;
    for (int k = 0; k < d; ++k) {
        int c = cell_of(gp->hi[k], gp->lo[k], w, gp->inv_w0, (1 << bmax) - 1);
        gp->cmax0[k] = c;
        cmax = max(cmax, c);
    }
    int bits = cmax ? 32 - __clz(cmax) : 0;
    gp->bits = bits;
    gp->key_bits = bits * d;
    gp->top_level = bits;
    gp->start_level = min(in.start_level, bits);
}

// ---------------------------------------------------------------------------
// Start level of every query (density adaptivity).  L(p) = the smallest level
// at which the cell of sorted point p holds at least H points; equivalently
// the minimum, over the windows of H consecutive sorted points that contain
// p, of the level at which the window's first and last keys share a prefix
// (a level-l cell is a run of equal key >> d*l).  Sliding-window minimum by
// the van Herk / Gil-Werman method: per block of H windows a prefix and a
// suffix minimum.  The query starts one level below: lvl[p] = max(0, L - 1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t window_level(const uint64_t *keys, int64_t a, int64_t H, int d)
{
    uint64_t x = keys[a] ^ keys[a + H - 1];
    int nb = x ? 64 - __clzll((long long)x) : 0;
    return (uint32_t)((nb + d - 1) / d);
}

__global__ void k_window_blocks(const uint64_t *__restrict__ keys, int64_t nw, int64_t H, int d,
                                uint8_t *__restrict__ pm, uint8_t *__restrict__ sm)
{
    const int64_t nblk = (nw + H - 1) / H;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nblk;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lo = b * H, hi = min(nw, lo + H);
        uint32_t m = 255;
        for (int64_t a = lo; a < hi; ++a) {
            m = min(m, window_level(keys, a, H, d));
            pm[a] = (uint8_t)m;
        }
        m = 255;
        for (int64_t a = hi - 1; a >= lo; --a) {
            m = min(m, window_level(keys, a, H, d));
            sm[a] = (uint8_t)m;
        }
    }
}

__global__ void k_start_levels(const uint8_t *__restrict__ pm, const uint8_t *__restrict__ sm, int64_t n,
                               int64_t H, uint32_t top, uint32_t base, uint32_t *__restrict__ lvl)
{
    const int64_t nw = n - H + 1;  // number of windows (> 0 here)
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lo = max((int64_t)0, p - H + 1), hi = min(p, nw - 1);
        uint32_t L;
        if (lo / H == hi / H) L = (lo % H == 0) ? pm[hi] : sm[lo];
        else L = min((uint32_t)sm[lo], (uint32_t)pm[hi]);
        uint32_t l = L > 0 ? L - 1 : 0;
        l = max(l, base);
        lvl[p] = min(l, top);
    }
}

__global__ void k_fill_u32(uint32_t *out, int64_t m, uint32_t v)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < m;
         a += (int64_t)gridDim.x * blockDim.x)
        out[a] = v;
}

// Sort keys (the level) of the active list, and the level range present.
__global__ void k_level_keys(const uint32_t *__restrict__ list, const uint32_t *__restrict__ lvl, int64_t m,
                             uint32_t *__restrict__ key, uint32_t *range)
{
    uint32_t lmin = 0xffffffffu, lmax = 0;
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < m;
         a += (int64_t)gridDim.x * blockDim.x) {
        uint32_t l = lvl[list[a]];
        key[a] = l;
        lmin = min(lmin, l);
        lmax = max(lmax, l);
    }
    for (int o = 16; o; o >>= 1) {
        lmin = min(lmin, __shfl_xor_sync(FULL, lmin, o));
        lmax = max(lmax, __shfl_xor_sync(FULL, lmax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&range[0], lmin);
        atomicMax(&range[1], lmax);
    }
}

// Group boundaries of a level-sorted list: a new group where the level or
// the cell at that level changes.
__global__ void k_run_flags_lv(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ list,
                               const uint32_t *__restrict__ lvl, int64_t m, int d,
                               uint32_t *__restrict__ flags)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < m;
         a += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = list[a], l = lvl[s];
        uint32_t f = 1;
        if (a > 0) {
            const uint32_t s0 = list[a - 1], l0 = lvl[s0];
            f = (l != l0) || ((keys[s] >> (d * l)) != (keys[s0] >> (d * l0)));
        }
        flags[a] = f;
    }
}

// Uncertified queries move one level up (a ring of cells twice as wide).
__global__ void k_bump_levels(const uint32_t *__restrict__ list, const uint32_t *__restrict__ status, int64_t m,
                              uint32_t *__restrict__ lvl, uint32_t top)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < m;
         a += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = list[a];
        if (status[s] == 1) lvl[s] = min(lvl[s] + 1, top);
    }
}

// End of a pass, one readback: out[0] = entries of `list` with status 2
// (buffer overflow), out[1] = entries with status 1 (re-queued), out[2] /
// out[3] = the smallest / largest level of the status-1 entries, after
// moving them one level up when `bump` is set (k_bump_levels's rule).
// out must hold {0, 0, 0xffffffff, 0} on entry (k_summary_init).
// Start of a pass: the device words its kernels accumulate into -- [2] the
// largest group (work queue), [3] the scan's queue head, [4..5] the active
// queries' level range (min, max), [8..11] the end-of-pass summary (as
// k_summary_init) -- in one launch.
__global__ void k_pass_init(uint32_t *small)
{
    if (threadIdx.x == 0) {
        small[2] = 0u;
        small[3] = 0u;
        small[4] = 0xffffffffu;
        small[5] = 0u;
        small[8] = 0u;
        small[9] = 0u;
        small[10] = 0xffffffffu;
        small[11] = 0u;
    }
}

__global__ void k_summary_init(uint32_t *out)
{
    if (threadIdx.x == 0) {
        out[0] = 0u;
        out[1] = 0u;
        out[2] = 0xffffffffu;
        out[3] = 0u;
    }
}

__global__ void k_status_summary(const uint32_t *__restrict__ list, const uint32_t *__restrict__ status, int64_t m,
                                 uint32_t *__restrict__ lvl, uint32_t top, int bump, uint32_t *out)
{
    uint32_t c2 = 0, c1 = 0, lmin = 0xffffffffu, lmax = 0;
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < m;
         a += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = list[a];
        const uint32_t st = status[s];
        if (st == 2) {
            ++c2;
        } else if (st == 1) {
            ++c1;
            uint32_t l = lvl[s];
            if (bump) {
                l = min(l + 1, top);
                lvl[s] = l;
            }
            lmin = min(lmin, l);
            lmax = max(lmax, l);
        }
    }
    for (int o = 16; o; o >>= 1) {
        c2 += __shfl_xor_sync(FULL, c2, o);
        c1 += __shfl_xor_sync(FULL, c1, o);
        lmin = min(lmin, __shfl_xor_sync(FULL, lmin, o));
        lmax = max(lmax, __shfl_xor_sync(FULL, lmax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (c2) atomicAdd(&out[0], c2);
        if (c1) {
            atomicAdd(&out[1], c1);
            atomicMin(&out[2], lmin);
            atomicMax(&out[3], lmax);
        }
    }
}

// The queries of a list go to level `l` (the tail strategy: the whole grid).
__global__ void k_set_levels(const uint32_t *__restrict__ list, int64_t m, uint32_t *__restrict__ lvl, uint32_t l)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < m; a += (int64_t)gridDim.x * blockDim.x)
        lvl[list[a]] = l;
}

// ---------------------------------------------------------------------------
// a3 / a5
// ---------------------------------------------------------------------------
__global__ void k_keys(const float *__restrict__ xs, int64_t n, const GridParams *__restrict__ gp,
                       uint64_t *__restrict__ keys, uint32_t *__restrict__ vals)
{
    const int d = gp->d, bits = gp->bits;
    const float w = gp->w0, iw = gp->inv_w0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int c[MAX_DIM];
        for (int k = 0; k < d; ++k)
            c[k] = cell_of(xs[(int64_t)k * n + i], gp->lo[k], w, iw, gp->cmax0[k]);
        keys[i] = morton_encode(c, d, bits);
        vals[i] = (uint32_t)i;
    }
}

__global__ void k_gather(const float *__restrict__ xs, int64_t n, int d, const uint32_t *__restrict__ perm,
                         float *__restrict__ xsort)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        uint32_t i = perm[s];
        const int P = pad_dim(d);
        for (int k = 0; k < P; ++k) xsort[(int64_t)s * P + k] = k < d ? xs[(int64_t)k * n + i] : 0.0f;
    }
}

// ---------------------------------------------------------------------------
// Runs of equal key >> shift over keys[idx[a]] (idx == nullptr: identity).
// ---------------------------------------------------------------------------
__global__ void k_run_flags(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ idx,
                            int64_t m, int shift, uint32_t *__restrict__ flags)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < m;
         a += (int64_t)gridDim.x * blockDim.x) {
        uint64_t ka = keys[idx ? idx[a] : a] >> shift;
        uint32_t f = 1;
        if (a > 0) f = ka != (keys[idx ? idx[a - 1] : a - 1] >> shift);
        flags[a] = f;
    }
}

// Run starts: begin[rid[a]] = a where flags[a]; also the run count.
__global__ void k_run_begin(const uint32_t *__restrict__ flags, const uint32_t *__restrict__ rid,
                            int64_t m, uint32_t *__restrict__ begin, uint32_t *count)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < m;
         a += (int64_t)gridDim.x * blockDim.x) {
        if (flags[a]) begin[rid[a]] = (uint32_t)a;
        if (a == m - 1) {
            uint32_t c = rid[a] + flags[a];
            *count = c;
            begin[c] = (uint32_t)m;
        }
    }
}

// Dense cell table of a level (common.cuh, DenseDims): each run of the
// level writes its (begin, end) at its cell's index; the table was zeroed.
__global__ void k_dense_insert(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ begin,
                               const uint32_t *ncells_p, int shift, int d, int nbits, DenseDims dims,
                               uint2 *__restrict__ tab)
{
    const uint32_t ncells = *ncells_p;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
        const uint32_t b = begin[c], e = begin[c + 1];
        int cell[MAX_DIM];
        morton_decode(keys[b] >> shift, d, nbits, cell);
        uint32_t idx = 0;
        for (int k = 0; k < d; ++k) idx += (uint32_t)cell[k] * dims.stride[k];
        tab[idx] = make_uint2(b, e);
    }
}

// Insertion into the level hash map (common.cuh: layout and lookup).
__global__ void k_hash_insert(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ begin,
                              const uint32_t *ncells_p, int shift, uint4 *slot, uint32_t hmask)
{
    uint32_t ncells = *ncells_p;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
        uint32_t b = begin[c], e = begin[c + 1];
        uint64_t P = keys[b] >> shift;
        uint32_t h = (uint32_t)mix64(P) & hmask;
        for (uint32_t probe = 0; probe <= hmask; ++probe) {
            unsigned long long prev = atomicCAS((unsigned long long *)&slot[h], HASH_EMPTY, P);
            if (prev == HASH_EMPTY || prev == P) {
                ((uint2 *)&slot[h])[1] = make_uint2(b, e);
                break;
            }
            h = (h + 1) & hmask;
        }
    }
}

// ---------------------------------------------------------------------------
// a6: groups (queries of the active list sharing a level cell), ordered by
// size descending (the paper's density order), split into work items of at
// most `qpi` queries.
// ---------------------------------------------------------------------------
__global__ void k_group_sizes(const uint32_t *__restrict__ gbegin, const uint32_t *ng_p,
                              uint32_t *__restrict__ sortkey, uint32_t *__restrict__ gid,
                              uint32_t *maxsize)
{
    uint32_t ng = *ng_p;
    uint32_t lmax = 0;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        uint32_t sz = gbegin[g + 1] - gbegin[g];
        sortkey[g] = sz;
        gid[g] = g;
        lmax = max(lmax, sz);
    }
    for (int o = 16; o; o >>= 1) lmax = max(lmax, __shfl_xor_sync(FULL, lmax, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxsize, lmax);
}

// sortkey = maxsize - size (ascending sort => size descending, stable)
// The order of at most GROUP_SORT_SMALL groups by size descending, ties by
// group index (what the radix sort of the size keys gives, it being stable),
// in one block: a bitonic sort in shared memory of (max - size) << 12 | g.
constexpr int GROUP_SORT_SMALL = 4096;
__global__ void __launch_bounds__(1024) k_group_sort_small(const uint32_t *__restrict__ sizes, const uint32_t *ng_p,
                                                         const uint32_t *maxsize, uint32_t *__restrict__ order)
{
    __shared__ uint32_t v[GROUP_SORT_SMALL];
    const uint32_t ng = *ng_p, mx = *maxsize;
    uint32_t N = 64;
    while (N < ng) N <<= 1;
    for (uint32_t g = threadIdx.x; g < N; g += blockDim.x)
        v[g] = g < ng ? ((mx - sizes[g]) << 12) | g : 0xffffffffu;
    __syncthreads();
    for (uint32_t k = 2; k <= N; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t t = threadIdx.x; t < N / 2; t += blockDim.x) {
                const uint32_t i = 2 * t - (t & (j - 1)), p = i + j;  // i has bit j clear
                const bool up = (i & k) == 0;
                const uint32_t a = v[i], b = v[p];
                if ((a > b) == up) {
                    v[i] = b;
                    v[p] = a;
                }
            }
            __syncthreads();
        }
    }
    for (uint32_t g = threadIdx.x; g < ng; g += blockDim.x) order[g] = v[g] & 4095u;
}

__global__ void k_group_sortkey(uint32_t *__restrict__ sortkey, const uint32_t *ng_p, const uint32_t *maxsize)
{
    uint32_t ng = *ng_p, mx = *maxsize;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x)
        sortkey[g] = mx - sortkey[g];
}

__global__ void k_group_nitems(const uint32_t *__restrict__ gbegin, const uint32_t *__restrict__ order,
                               const uint32_t *ng_p, int qpi, uint32_t *__restrict__ nitems)
{
    uint32_t ng = *ng_p;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        uint32_t og = order[g];
        uint32_t sz = gbegin[og + 1] - gbegin[og];
        nitems[g] = (sz + qpi - 1) / qpi;
    }
}

// Item = (first list index, count | level << 16).
__global__ void k_group_items(const uint32_t *__restrict__ gbegin, const uint32_t *__restrict__ order,
                              const uint32_t *ng_p, int qpi, const uint32_t *__restrict__ ioff,
                              const uint32_t *__restrict__ list, const uint32_t *__restrict__ lvl,
                              uint2 *__restrict__ items)
{
    uint32_t ng = *ng_p;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        uint32_t og = order[g];
        uint32_t b = gbegin[og], e = gbegin[og + 1];
        uint32_t o = ioff[g];
        uint32_t l = lvl[list[b]];
        for (uint32_t a = b; a < e; a += qpi) items[o++] = make_uint2(a, min((uint32_t)qpi, e - a) | (l << 16));
    }
}

// Next active list: active entries whose query was not certified.
__global__ void k_compact(const uint32_t *__restrict__ active, const uint32_t *__restrict__ flags,
                          const uint32_t *__restrict__ pos, int64_t m, uint32_t *__restrict__ out)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < m;
         a += (int64_t)gridDim.x * blockDim.x)
        if (flags[a]) out[pos[a]] = active ? active[a] : (uint32_t)a;
}

// flags[a] = (status[list[a]] == value)
__global__ void k_status_flags(const uint32_t *__restrict__ list, const uint32_t *__restrict__ status,
                               int64_t m, uint32_t value, uint32_t *__restrict__ flags)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < m;
         a += (int64_t)gridDim.x * blockDim.x)
        flags[a] = status[list[a]] == value;
}

// a11: every output distance holds the bit pattern of its canonical squared
// distance D; replace it by the correctly rounded sqrt(D) (exact.cuh).
// Streaming pass: with 16-byte aligned data each thread keeps two 16-byte
// vectors (four values) in flight per iteration, enough to run near HBM
// bandwidth; otherwise one value at a time.
__global__ void k_sqrt_rows(double *__restrict__ dist, int64_t count)
{
    unsigned long long *u = (unsigned long long *)dist;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    if (((uintptr_t)dist & 15) == 0) {
        ulonglong2 *v = (ulonglong2 *)dist;
        const int64_t nv = count / 2;
        int64_t i = tid;
        for (; i + nth < nv; i += 2 * nth) {
            ulonglong2 a = v[i], b = v[i + nth];
            a.x = sqrt_bits(a.x);
            a.y = sqrt_bits(a.y);
            b.x = sqrt_bits(b.x);
            b.y = sqrt_bits(b.y);
            v[i] = a;
            v[i + nth] = b;
        }
        for (; i < nv; i += nth) {
            ulonglong2 a = v[i];
            a.x = sqrt_bits(a.x);
            a.y = sqrt_bits(a.y);
            v[i] = a;
        }
        if (tid == 0 && (count & 1)) u[count - 1] = sqrt_bits(u[count - 1]);
    } else {
        for (int64_t i = tid; i < count; i += nth) u[i] = sqrt_bits(u[i]);
    }
}

// The paper's policy (epochs): flag the sorted positions whose query is not
// done yet, and mark the queries certified by a pass as done.
__global__ void k_undone_flags(const uint32_t *__restrict__ qperm, const uint32_t *__restrict__ done, int64_t nq,
                               uint32_t *__restrict__ flags)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nq; a += (int64_t)gridDim.x * blockDim.x)
        flags[a] = done[qperm[a]] == 0u;
}

__global__ void k_mark_done(const uint32_t *__restrict__ list, const uint32_t *__restrict__ status, int64_t m,
                            const uint32_t *__restrict__ qperm, uint32_t *__restrict__ done)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < m; a += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = list[a];
        if (status[s] == 0u) done[qperm[s]] = 1u;
    }
}

// Chunked or sharded output: flags[a] = (the original row of sorted query
// position list[a] lies in [r0, r1)).
// Sorted-position shard (cost-balanced shards): flags[a] = list[a] in [r0, r1).
__global__ void k_pos_flags(const uint32_t *__restrict__ list, int64_t m, uint32_t r0, uint32_t r1,
                            uint32_t *__restrict__ flags)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < m; a += (int64_t)gridDim.x * blockDim.x)
        flags[a] = list[a] >= r0 && list[a] < r1;
}

// Original rows of the sorted positions [p0, p0 + m) (int64).
__global__ void k_rows_of(const uint32_t *__restrict__ perm, int64_t p0, int64_t m, int64_t *__restrict__ rows)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < m; a += (int64_t)gridDim.x * blockDim.x)
        rows[a] = perm[p0 + a];
}

// Shard cost model, per level: the points of each non-empty cell's 3^d
// neighbourhood (Alg. 1, ring 1), cells found in the level's dense table or
// hash map.
__global__ void k_cell_around(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ begin,
                              const uint32_t *ncells_p, int shift, int d, int nbits, DenseDims dims, DenseDims cmax,
                              const uint2 *__restrict__ dense, const uint4 *__restrict__ hslot, uint32_t hmask,
                              uint32_t *__restrict__ around)
{
    int noff = 1;
    for (int k = 0; k < d; ++k) noff *= 3;
    const uint32_t ncells = *ncells_p;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
        int cell[MAX_DIM], nb[MAX_DIM];
        morton_decode(keys[begin[c]] >> shift, d, nbits, cell);
        uint32_t sum = 0;
        for (int o = 0; o < noff; ++o) {
            int r = o;
            bool ok = true;
            uint32_t idx = 0;
            for (int k = 0; k < d; ++k) {
                nb[k] = cell[k] + r % 3 - 1;
                r /= 3;
                ok = ok && nb[k] >= 0 && nb[k] <= (int)cmax.stride[k];
                idx += (uint32_t)nb[k] * dims.stride[k];
            }
            if (!ok) continue;
            const uint2 rg = dense ? dense[idx] : hash_lookup(hslot, hmask, morton_encode(nb, d, nbits));
            sum += rg.y - rg.x;
        }
        around[c] = sum;
    }
}

// Cell (run) index of every sorted position at a level: inclusive count of
// run starts - 1.
__global__ void k_run_index(const uint32_t *__restrict__ flags, const uint32_t *__restrict__ rid, int64_t n,
                            uint32_t *__restrict__ idx)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n; a += (int64_t)gridDim.x * blockDim.x)
        idx[a] = rid[a] + flags[a] - 1u;
}

// Per-level arrays of the shard cost model, levels [lmin, lmax].
constexpr int COST_MAX_LEVELS = 12;
struct QueryCostArgs {
    const uint32_t *idx[COST_MAX_LEVELS];     // cell index of each sorted position
    const uint32_t *around[COST_MAX_LEVELS];  // neighbourhood points of each cell
    int lmin, lmax;
};

// Cost of each query: the neighbourhood points at its start level, and at
// the levels above while that count is below 2K (where it would fail and be
// re-queued), as the candidates it is expected to evaluate.
__global__ void k_query_costs(const uint32_t *__restrict__ lvl, int64_t n, int K, const QueryCostArgs c,
                              float *__restrict__ cost)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        int l = max((int)lvl[s], c.lmin);
        float sum = 0.0f;
        for (; l <= c.lmax; ++l) {
            const uint32_t a = c.around[l - c.lmin][c.idx[l - c.lmin][s]];
            sum += (float)a;
            if (a >= 2u * (uint32_t)K) break;
        }
        cost[s] = sum;
    }
}

// Diagnostic (knnjoin_index_dump): the run [begin, end) of sorted positions
// that a level's cell table gives for each probe key (the Morton bits of a
// level cell's coordinates, nbits per dimension), as the scan looks cells up:
// the dense table at index sum_k c_k stride_k, or the hash map at the key;
// (0, 0) for a key beyond the level's grid or a cell without points.
__global__ void k_probe_cells(const uint64_t *__restrict__ probe, int64_t m, int d, int nbits, DenseDims stride,
                              DenseDims cmaxL, const uint2 *__restrict__ dense, const uint4 *__restrict__ slot,
                              uint32_t hmask, uint2 *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = probe[i];
        int c[MAX_DIM];
        morton_decode(key, d, nbits, c);
        bool in = nbits * d >= 64 || (key >> (nbits * d)) == 0;
        uint32_t idx = 0;
        for (int k = 0; k < d; ++k) {
            in = in && (uint32_t)c[k] <= cmaxL.stride[k];
            idx += (uint32_t)c[k] * stride.stride[k];
        }
        uint2 r = make_uint2(0, 0);
        if (in) r = dense ? dense[idx] : hash_lookup(slot, hmask, key);
        out[i] = r;
    }
}

// Smallest and largest value of a uint32 array (out[0] min, out[1] max,
// initialised to ~0 and 0).
__global__ void k_minmax_u32(const uint32_t *__restrict__ v, int64_t n, uint32_t *out)
{
    uint32_t lo = 0xffffffffu, hi = 0;
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n; a += (int64_t)gridDim.x * blockDim.x) {
        lo = min(lo, v[a]);
        hi = max(hi, v[a]);
    }
    for (int o = 16; o; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(FULL, lo, o));
        hi = max(hi, __shfl_xor_sync(FULL, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&out[0], lo);
        atomicMax(&out[1], hi);
    }
}

__global__ void k_row_flags(const uint32_t *__restrict__ list, const uint32_t *__restrict__ qperm, int64_t m,
                            uint32_t r0, uint32_t r1, uint32_t *__restrict__ flags)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < m; a += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = qperm[list[a]];
        flags[a] = r >= r0 && r < r1;
    }
}

// Small readback: copy `words` 32-bit words (to mapped host memory).
__global__ void k_fetch(uint32_t *dst, const uint32_t *__restrict__ src, int words)
{
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}

// dst[0] = *a + *b (a list's length: the last exclusive prefix plus the last flag).
__global__ void k_fetch_sum2(uint32_t *dst, const uint32_t *__restrict__ a, const uint32_t *__restrict__ b)
{
    if (threadIdx.x == 0) dst[0] = *a + *b;
}

__global__ void k_iota(uint32_t *out, int64_t m)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < m;
         a += (int64_t)gridDim.x * blockDim.x)
        out[a] = (uint32_t)a;
}

}  // namespace knn
