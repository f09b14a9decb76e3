// scan2.cuh -- register-reuse neighbour-cell scan with top-K selection
// (paper Alg. 1 GPUJoinKernel, Sec. 4.6 task granularity), the fast path.
//
// Each warp works alone (no block barriers) on work items of up to QM
// queries that share a level-l grid cell:
//   a7  lanes look up the 3^d neighbouring cells, 32 at a time, in the
//       level's hash map, and a warp prefix sum flattens their point runs;
//   a8  lane t takes candidate t of the flattened runs, loads its
//       coordinates once (one or two aligned vector loads through L1/L2) and
//       scores it against every query of the item (query coordinates are
//       broadcast from shared memory), so a candidate read serves QM queries.
//       A candidate is kept only if its FP32 squared distance is at most the
//       query's threshold, which starts at R^2 (1 + 2^-14) -- R the distance
//       from the query to the faces of the scanned box, the certificate
//       radius: a point farther than R cannot belong to a certified answer
//       -- and drops to T (1 + 2^-15) + 2^-120 when the per-query buffer of B
//       entries fills (T = its K-th value, found by a warp radix select);
//   a9  per query, the warp selects T32 (the K-th FP32 value), keeps the band
//       d2_32 <= T32 (1 + 2^-15) + 2^-120, scores the band with the bit-exact
//       canonical FP64 distance (exact.cuh), sorts it by (D, original id)
//       with a warp bitonic network and certifies the K-th against R;
//   a10 writes the per-point status: 0 certified, 1 not certified (fewer
//       than K points within R, or D_K >= R^2: retry one level up), 2 buffer
//       overflow (massive ties: redone by the general kernel of scan.cuh);
//   a11 writes certified rows: original ids and the bit patterns of D (the
//       correctly rounded square roots are taken afterwards, k_sqrt_rows).
#pragma once
#include "common.cuh"
#include "grid.cuh"
#include "scan.cuh"

namespace knn {

// Phase timing (diagnostics): built with -DKNN_PHASE_TIMING, lane 0 of every
// warp adds clock64() deltas per phase of k_scan2 to g_phase; otherwise the
// markers compile to nothing.
#ifdef KNN_PHASE_TIMING
__device__ unsigned long long g_phase[8];
#define KNN_PT_DECL unsigned long long ph_[8] = {0, 0, 0, 0, 0, 0, 0, 0}, pt_ = clock64()
#define KNN_PT(i)                                          \
    do {                                                   \
        unsigned long long t_ = clock64();                 \
        ph_[i] += t_ - pt_;                                \
        pt_ = t_;                                          \
    } while (0)
#define KNN_PT_FLUSH                                       \
    do {                                                   \
        if ((threadIdx.x & 31) == 0)                       \
            for (int q_ = 0; q_ < 8; ++q_) atomicAdd(&g_phase[q_], ph_[q_]); \
    } while (0)
#else
#define KNN_PT_DECL
#define KNN_PT(i) \
    do {          \
    } while (0)
#define KNN_PT_FLUSH \
    do {             \
    } while (0)
#endif

constexpr int S2_WARPS = 4;

// Neighbour offsets of the 3^d box, nearest first: for each d the offset
// codes (base-3 digits, digit 1 = no move) ordered by how many dimensions
// move (0, then faces, edges, ...).  Filled once per device by the host.
constexpr int NB_ORDER_TOTAL = 3 + 9 + 27 + 81 + 243 + 729 + 2187 + 6561;
__constant__ uint16_t c_nb_order[NB_ORDER_TOTAL];
__host__ __device__ constexpr int nb_order_offset(int d)
{
    return d <= 1 ? 0 : nb_order_offset(d - 1) + (d == 2 ? 3 : d == 3 ? 9 : d == 4 ? 27 : d == 5 ? 81 : d == 6 ? 243 : d == 7 ? 729 : 2187);
}
constexpr int S2_CTA = S2_WARPS * 32;

template <int DIM>
__device__ __forceinline__ void load_point(const float *__restrict__ xs, uint32_t s, float (&c)[DIM])
{
    constexpr int P = pad_dim(DIM);
    const float *p = xs + (size_t)s * P;
    if (P == 2) {
        float2 v = __ldg((const float2 *)p);
        c[0] = v.x;
        if (DIM > 1) c[DIM > 1 ? 1 : 0] = v.y;
    } else if (P == 4) {
        float4 v = __ldg((const float4 *)p);
        float t[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < DIM; ++k) c[k] = t[k];
    } else {
        float4 v0 = __ldg((const float4 *)p), v1 = __ldg((const float4 *)(p + 4));
        float t[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
        for (int k = 0; k < DIM; ++k) c[k] = t[k];
    }
}

// K-th smallest (1 <= k <= cnt) of the high 32 bits (non-negative float bit
// patterns) of buf[0..cnt).
__device__ uint32_t warp_select_hi(const uint64_t *buf, int cnt, int k, uint32_t *hist, int lane)
{
    uint32_t prefix = 0, mask = 0;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int i = lane; i < 256; i += 32) hist[i] = 0;
        __syncwarp();
        for (int i = lane; i < cnt; i += 32) {
            uint32_t v = (uint32_t)(buf[i] >> 32);
            if ((v & mask) == prefix) atomicAdd(&hist[(v >> shift) & 255u], 1u);
        }
        __syncwarp();
        uint32_t h[8], s = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            h[j] = hist[lane * 8 + j];
            s += h[j];
        }
        uint32_t inc = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        uint32_t ball = __ballot_sync(FULL, inc >= (uint32_t)k);
        int src = __ffs(ball) - 1;
        uint32_t digit = 0, below = 0;
        if (lane == src) {
            uint32_t run = inc - s;
            bool found = false;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (!found && run + h[j] >= (uint32_t)k) {
                    digit = lane * 8 + j;
                    below = run;
                    found = true;
                }
                run += h[j];
            }
        }
        digit = __shfl_sync(FULL, digit, src);
        below = __shfl_sync(FULL, below, src);
        prefix |= digit << shift;
        mask |= 255u << shift;
        k -= (int)below;
        __syncwarp();
    }
    return prefix;
}

// Keep entries whose high 32 bits are <= thr (in place); returns the count.
__device__ int warp_compact_hi(uint64_t *buf, int cnt, uint32_t thr, int lane)
{
    int out = 0;
    for (int base = 0; base < cnt; base += 32) {
        int i = base + lane;
        bool v = i < cnt;
        uint64_t e = v ? buf[i] : 0ull;
        bool keep = v && (uint32_t)(e >> 32) <= thr;
        uint32_t bal = __ballot_sync(FULL, keep);
        __syncwarp();
        if (keep) buf[out + __popc(bal & lanemask_lt())] = e;
        out += __popc(bal);
        __syncwarp();
    }
    return out;
}

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

// Bitonic sort, ascending, of 32*E 64-bit values held E per lane in blocked
// order (entry g = lane*E + e).
template <int E>
__device__ __forceinline__ void warp_bitonic_u64(uint64_t (&V)[E], int lane)
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
                        const bool up = ((lane * E + e) & k) == 0;
                        const uint64_t lo = V[e] < V[p] ? V[e] : V[p];
                        const uint64_t hi = V[e] < V[p] ? V[p] : V[e];
                        V[e] = up ? lo : hi;
                        V[p] = up ? hi : lo;
                    }
                }
            } else {
                const int lm = j / E;
                const bool lower = (lane & lm) == 0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const uint64_t o = __shfl_xor_sync(FULL, V[e], lm);
                    const bool up = ((lane * E + e) & k) == 0;
                    const bool keep_min = lower == up;
                    V[e] = keep_min ? (o < V[e] ? o : V[e]) : (o < V[e] ? V[e] : o);
                }
            }
        }
    }
}

// Row of a query in shared memory: coordinates, current threshold, sorted
// position (as float bits), padded to a multiple of 4 floats (vector loads).
__host__ __device__ constexpr int query_row_floats(int d) { return (d + 2 + 3) & ~3; }

template <int DIM>
__device__ __forceinline__ void load_query_row(const float *qc, int i, float (&q)[DIM], float &thr, uint32_t &qs)
{
    constexpr int QP = query_row_floats(DIM);
    float r[QP];
    const float4 *row = (const float4 *)(qc + i * QP);
#pragma unroll
    for (int v = 0; v < QP / 4; ++v) {
        const float4 t = row[v];
        r[4 * v] = t.x;
        r[4 * v + 1] = t.y;
        r[4 * v + 2] = t.z;
        r[4 * v + 3] = t.w;
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) q[k] = r[k];
    thr = r[DIM];
    qs = __float_as_uint(r[DIM + 1]);
}

// FP32 squared distance; for d >= 4 even and odd dimensions accumulate in two
// chains (shorter latency).  Either way the value is within (d + 2) 2^-24
// relative of the exact squared distance (plus underflow terms far below
// 2^-120), which the band factor 2^-15 covers.
template <int DIM>
__device__ __forceinline__ float dist2_f32(const float (&q)[DIM], const float (&c)[DIM])
{
    if (DIM < 4) {
        float d2 = 0.0f;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const float df = q[k] - c[k];
            d2 = fmaf(df, df, d2);
        }
        return d2;
    }
    float e = 0.0f, o = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const float df = q[k] - c[k];
        if (k & 1) o = fmaf(df, df, o);
        else e = fmaf(df, df, e);
    }
    return e + o;
}

// Bitonic sort, ascending, of 32*E 32-bit values held E per lane in blocked
// order (entry g = lane*E + e).
template <int E>
__device__ __forceinline__ void warp_bitonic_u32(uint32_t (&V)[E], int lane)
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
                        const bool up = ((lane * E + e) & k) == 0;
                        const uint32_t lo = min(V[e], V[p]), hi = max(V[e], V[p]);
                        V[e] = up ? lo : hi;
                        V[p] = up ? hi : lo;
                    }
                }
            } else {
                const int lm = j / E;
                const bool lower = (lane & lm) == 0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const uint32_t o = __shfl_xor_sync(FULL, V[e], lm);
                    const bool up = ((lane * E + e) & k) == 0;
                    V[e] = (lower == up) ? min(o, V[e]) : max(o, V[e]);
                }
            }
        }
    }
}

// Certificate radius of a query at level `level` in cell `cell` (rounded
// down): distance to the nearest face of the 3^d box beyond which points exist.
template <int DIM>
__device__ __forceinline__ float cert_radius(const float *q, const int *cell, const int *cmaxL,
                                             const ScanArgs &a, int level)
{
    float R = __int_as_float(0x7f800000);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const int cL = cell[k];
        if (cL >= 2) R = fminf(R, __fsub_rd(q[k], face_of((cL - 1) << level, a.lo[k], a.w0)));
        if (cL + 1 < cmaxL[k]) R = fminf(R, __fsub_rd(face_of((cL + 2) << level, a.lo[k], a.w0), q[k]));
    }
    return R;
}

// Buffer full: find its K-th value T, lower the threshold to the band of T
// and keep only the entries within it.  Returns (new count, new threshold
// bits).  Kept out of line: it runs rarely.
__device__ __noinline__ int2 shrink_buffer(uint64_t *bi, int c0, int K, uint32_t *hist, int lane, float thr)
{
    __syncwarp();
    uint32_t T = warp_select_hi(bi, c0, K, hist, lane);
    float nt = fminf(thr, band_thr(T));
    int c1 = warp_compact_hi(bi, c0, __float_as_uint(nt), lane);
    __syncwarp();
    return make_int2(c1, __float_as_int(nt));
}

template <int DIM, int QM, int E>
__global__ void __launch_bounds__(S2_CTA, 5) k_scan2(ScanArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int P = pad_dim(DIM);
    constexpr int QP = query_row_floats(DIM);
    constexpr int B = 32 * E;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int K = a.K, NOFF = a.noff;

    // per-warp shared memory
    constexpr int BS = B;
    const size_t wbytes = (size_t)QM * BS * 8 + (size_t)QM * QP * 4 + (size_t)QM * 8 + 256 * 4 +
                          (size_t)QM * 2 * DIM * 4;
    unsigned char *wb = smem + warp * ((wbytes + 15) & ~(size_t)15);
    uint64_t *buf = (uint64_t *)wb;            // [QM][BS]  (d2_32 bits << 32 | sorted index)
    float *qc = (float *)(buf + QM * BS);      // [QM][QP] coords, threshold, sorted position
    int *cnt = (int *)(qc + QM * QP);          // [QM]
    uint32_t *qsv = (uint32_t *)(cnt + QM);    // [QM]
    uint32_t *hist = qsv + QM;                 // [256]
    float *gaps = (float *)(hist + 256);       // [QM][2*DIM] distance to own cell's faces (rounded down)

    unsigned long long st_cand = 0, st_band = 0;
    KNN_PT_DECL;

    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(a.counter, 1u);
        item = __shfl_sync(FULL, item, 0);
        if (item >= a.nitems) break;
        const uint2 it = a.items[item];
        const int Q = (int)(it.y & 0xffffu);
        const int level = (int)(it.y >> 16);
        const int shift = DIM * level;
        const int nbits = a.bits - level;
        int cmaxL[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) cmaxL[k] = a.cmax0[k] >> level;
        const uint64_t *hkey = a.hkeyL[level];
        const uint2 *hval = a.hvalL[level];
        const uint32_t hmask = a.hmaskL[level];

        if (lane < Q) {
            uint32_t s = a.active[it.x + lane];
            float c[DIM];
            load_point<DIM>(a.xsort, s, c);
            qsv[lane] = s;
#pragma unroll
            for (int k = 0; k < DIM; ++k) qc[lane * QP + k] = c[k];
        }
        __syncwarp();
        int cell[DIM];
        morton_decode(a.keys[qsv[0]] >> shift, DIM, nbits, cell);
        // query state: threshold and sorted position sit in the query's row
        // (one broadcast vector load gives a pair everything it needs); the
        // buffer count lives in lane i's register for query i
        int my_cnt = 0;
        if (lane < Q) {
            float q[DIM];
#pragma unroll
            for (int k = 0; k < DIM; ++k) q[k] = qc[lane * QP + k];
            const float R = cert_radius<DIM>(q, cell, cmaxL, a, level);
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                gaps[lane * 2 * DIM + 2 * k] = __fsub_rd(q[k], face_of(cell[k] << level, a.lo[k], a.w0));
                gaps[lane * 2 * DIM + 2 * k + 1] = __fsub_rd(face_of((cell[k] + 1) << level, a.lo[k], a.w0), q[k]);
            }
            qc[lane * QP + DIM] = isinf(R) ? __int_as_float(0x7f800000)
                                           : __fmul_ru(__fmul_ru(R, R), 1.0f + 0x1p-14f);
            qc[lane * QP + DIM + 1] = __uint_as_float(qsv[lane]);
        }
        __syncwarp();

        KNN_PT(0);
        // a7 + a8
        for (int ob = 0; ob < NOFF; ob += 32) {
            const int o = ob + lane;
            uint32_t rb = 0, re = 0;
            int code = 0;
            if (o < NOFF) {
                int nb[DIM];
                int r = c_nb_order[nb_order_offset(DIM) + o];
                code = r;
                bool ok = true;
#pragma unroll
                for (int k = 0; k < DIM; ++k) {
                    nb[k] = cell[k] + (r % 3) - 1;
                    r /= 3;
                    ok = ok && nb[k] >= 0 && nb[k] <= cmaxL[k];
                }
                if (ok) {
                    uint2 rg = hash_lookup(hkey, hval, hmask, morton_encode(nb, DIM, nbits));
                    rb = rg.x;
                    re = rg.y;
                }
            }
            const uint32_t len = re - rb;
            // queries this cell can still serve: rounded-down squared distance
            // from the query to the cell's box, against the query's threshold
            // with a 2^-19 margin for FP32 rounding of candidate distances
            uint32_t cmask = 0;
            if (len) {
                for (int i = 0; i < Q; ++i) {
                    float lb = 0.0f;
                    int r = code;
#pragma unroll
                    for (int k = 0; k < DIM; ++k) {
                        const int dg = r % 3;
                        r /= 3;
                        if (dg != 1) {
                            const float g = gaps[i * 2 * DIM + 2 * k + (dg == 2 ? 1 : 0)];
                            lb = __fmaf_rd(g, g, lb);
                        }
                    }
                    if (!(lb > qc[i * QP + DIM] * (1.0f + 0x1p-19f))) cmask |= 1u << i;
                }
            }
            uint32_t inc = len;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                uint32_t y = __shfl_up_sync(FULL, inc, d);
                if (lane >= d) inc += y;
            }
            const uint32_t exc = inc - len;
            const uint32_t total = __shfl_sync(FULL, inc, 31);
            KNN_PT(1);
            for (uint32_t t0 = 0; t0 < total; t0 += 32) {
                const uint32_t t = t0 + lane;
                const bool valid = t < total;
                int src = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    uint32_t ex = __shfl_sync(FULL, exc, src + step);
                    if (ex <= t) src += step;
                }
                const uint32_t sb = __shfl_sync(FULL, rb, src);
                const uint32_t se = __shfl_sync(FULL, exc, src);
                const uint32_t s = valid ? sb + (t - se) : 0u;
                const uint32_t cm = __shfl_sync(FULL, cmask, src);  // every lane takes part
                const uint32_t tmask = __reduce_or_sync(FULL, valid ? cm : 0u);
                float c[DIM];
                if (valid) {
                    load_point<DIM>(a.xsort, s, c);
                    st_cand += (unsigned long long)Q;
                } else {
#pragma unroll
                    for (int k = 0; k < DIM; ++k) c[k] = 0.0f;
                }
#pragma unroll 2
                for (int i = 0; i < Q; ++i) {
                    if (!((tmask >> i) & 1u)) continue;
                    float qv[DIM], ti;
                    uint32_t qi_s;
                    load_query_row<DIM>(qc, i, qv, ti, qi_s);
                    const float d2 = dist2_f32<DIM>(qv, c);
                    bool acc = valid && d2 <= ti && s != qi_s;
                    uint32_t bal = __ballot_sync(FULL, acc);
                    if (bal) {
                        uint64_t *bi = buf + i * BS;
                        int c0 = __shfl_sync(FULL, my_cnt, i);
                        int nnew = __popc(bal);
                        if (c0 + nnew > B) {
                            // buffer full: drop to the K-th value's band (rare)
                            int2 r2 = shrink_buffer(bi, c0, K, hist, lane, ti);
                            c0 = r2.x;
                            const float nt = __int_as_float(r2.y);
                            acc = acc && d2 <= nt;
                            bal = __ballot_sync(FULL, acc);
                            nnew = __popc(bal);
                            float tnew = nt;
                            if (c0 + nnew > B) {  // too many ties: general kernel
                                c0 = -1;
                                tnew = -1.0f;
                                acc = false;
                                nnew = 0;
                            }
                            if (lane == 0) qc[i * QP + DIM] = tnew;
                            __syncwarp();
                        }
                        if (acc) bi[c0 + __popc(bal & lanemask_lt())] = ((uint64_t)__float_as_uint(d2) << 32) | s;
                        if (lane == i) my_cnt = c0 < 0 ? -1 : c0 + nnew;
                    }
                }
            }
            KNN_PT(2);
        }
        __syncwarp();

        if (lane < Q) cnt[lane] = my_cnt;
        __syncwarp();

        // a9 - a11, one query at a time, whole warp
        for (int i = 0; i < Q; ++i) {
            const int c0 = cnt[i];
            uint32_t flag = 1;
            if (c0 < 0) {
                flag = 2;
            } else if (c0 >= K) {
                const uint64_t *bi = buf + i * BS;
                // whole buffer in registers (blocked: entry g = lane*E + e) as
                // 32-bit words: the FP32 key with its low bits replaced by the
                // buffer slot.  Sorted, entry K-1 bounds T32 from above by at
                // most the dropped bits, and the band (a prefix) stays a
                // superset of every entry within T32 (1 + 2^-15) + 2^-120.
                constexpr uint32_t SLOT = (uint32_t)B - 1;
                uint32_t v[E];
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int g = lane * E + e;
                    v[e] = g < c0 ? (((uint32_t)(bi[g] >> 32) & ~SLOT) | (uint32_t)g) : 0xffffffffu;
                }
                warp_bitonic_u32<E>(v, lane);
                KNN_PT(3);
                uint32_t vk = 0;
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (e == (K - 1) % E) vk = v[e];
                vk = __shfl_sync(FULL, vk, (K - 1) / E);
                const uint32_t tb = __float_as_uint(band_thr(vk | SLOT)) & ~SLOT;
                int mine = 0;
#pragma unroll
                for (int e = 0; e < E; ++e) mine += (lane * E + e < c0 && (v[e] & ~SLOT) <= tb) ? 1 : 0;
                int m = mine;
#pragma unroll
                for (int o = 16; o; o >>= 1) m += __shfl_xor_sync(FULL, m, o);
                KNN_PT(4);
                // exact canonical distances and original ids of the band
                float q[DIM];
                int32_t qi[DIM];
#pragma unroll
                for (int k = 0; k < DIM; ++k) {
                    q[k] = qc[i * QP + k];
                    qi[k] = a.fixed_ok ? to_fixed(q[k], a.F) : 0;
                }
                uint64_t D[E];
                uint32_t I[E];
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int g = lane * E + e;
                    D[e] = ~0ull;
                    I[e] = ~0u;
                    if (g < m) {
                        const uint32_t s = (uint32_t)bi[v[e] & SLOT];
                        float c[DIM];
                        load_point<DIM>(a.xsort, s, c);
                        uint64_t bits = 0;
                        bool done = false;
                        if (a.fixed_ok) {
                            int32_t ci[DIM];
#pragma unroll
                            for (int k = 0; k < DIM; ++k) ci[k] = to_fixed(c[k], a.F);
                            done = canon_d2_fixed<DIM>(qi, ci, a.F, bits);
                        }
                        if (!done) bits = canon_d2_fp64<DIM>(q, c);
                        D[e] = bits;
                        I[e] = a.perm[s];
                    }
                }
                if (lane == 0) st_band += (unsigned long long)m;
                KNN_PT(5);
                // the FP32 order is the exact order unless two near-equal
                // values swap; check neighbours, re-sort by (D, id) if needed
                bool inv = false;
#pragma unroll
                for (int e = 0; e + 1 < E; ++e)
                    inv = inv || (lane * E + e + 1 < m && xless(D[e + 1], I[e + 1], D[e], I[e]));
                const uint64_t nd = __shfl_down_sync(FULL, D[0], 1);
                const uint32_t ni = __shfl_down_sync(FULL, I[0], 1);
                inv = inv || (lane < 31 && (lane + 1) * E < m && xless(nd, ni, D[E - 1], I[E - 1]));
                if (__any_sync(FULL, inv)) warp_bitonic<E>(D, I, lane);
                uint64_t dk = 0;
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (e == (K - 1) % E) dk = D[e];
                dk = __shfl_sync(FULL, dk, (K - 1) / E);
                const float R = cert_radius<DIM>(q, cell, cmaxL, a, level);
                bool certified = isinf(R);
                if (!certified) {
                    const float R2 = __fmul_rd(__fmul_rd(R, R), 1.0f - 0x1p-20f);
                    certified = dk < f32_to_f64_bits_floor(R2);
                }
                KNN_PT(6);
                if (certified) {
                    flag = 0;
                    const int64_t row = (int64_t)a.perm[qsv[i]] * K;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int g = lane * E + e;
                        if (g < K) {
                            a.out_ids[row + g] = (int32_t)I[e];
                            a.out_dist[row + g] = __longlong_as_double((long long)D[e]);  // D; k_sqrt_rows converts
                        }
                    }
                }
            }
            if (lane == 0) a.fail[qsv[i]] = flag;
            KNN_PT(7);
        }
        __syncwarp();
    }
    KNN_PT_FLUSH;
    for (int o = 16; o; o >>= 1) {
        st_cand += __shfl_xor_sync(FULL, st_cand, o);
        st_band += __shfl_xor_sync(FULL, st_band, o);
    }
    if (lane == 0) {
        atomicAdd(&a.stats[0], st_cand);
        if (st_band) atomicAdd(&a.stats[2], st_band);
    }
}

}  // namespace knn
