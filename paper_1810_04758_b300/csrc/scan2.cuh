// scan2.cuh -- register-reuse neighbour-cell scan with top-K selection
// (paper Alg. 1 GPUJoinKernel, Sec. 4.7, GPU: Optimizing Task Granularity), the fast path.
//
// Each warp works alone (no block barriers) on work items of up to QM
// queries that share a level-l grid cell.  Per batch of 32 neighbour cells,
// nearest first:
//   a7  each lane forms its cell's key (or dense-table index) from the
//       item's table of coordinate parts, reads the level's cell table (one
//       load per probe) and, for every query of the item, tests the cell's
//       box against the query's threshold with a rounded-down squared
//       distance (a bit per query: the cell mask); a warp prefix sum
//       flattens the runs;
//   a8  runs of at least S2_BIG points go first, in super-tiles of S2_SUPER
//       consecutive sorted points, each tested per query against the box of
//       its Morton prefix (on skewed data S2_MEGA super-tiles at once, one
//       per lane); the other runs are scanned two tiles at a time:
//       lane t holds candidates t and t + 32, loads their coordinates once
//       and scores them against every query in the tiles' masks (query rows
//       broadcast from shared memory), so a candidate read serves up to QM
//       queries.  A candidate is kept when its FP32 squared distance is at
//       most the query's threshold: R^2 (1 + 2^-14) to start -- R the
//       distance to the faces of the scanned box, beyond which no point can
//       belong to a certified answer -- or the band of the K-th value an
//       earlier pass found, and T (1 + 2^-15) + 2^-120 once the per-query
//       buffer of B entries has filled (T = its K-th value, by a warp sort
//       or radix select);
//   a9  per query, the warp sorts the buffer as 32-bit keys, takes T32 (the
//       K-th FP32 value), keeps the band d2_32 <= T32 (1 + 2^-15) + 2^-120,
//       scores it with the bit-exact canonical FP64 distance (exact.cuh),
//       orders it by (D, original id) and certifies the K-th against R;
//   a10 writes the per-point status: 0 certified, 1 not certified (fewer
//       than K points within R, or D_K >= R^2: retry one level up, starting
//       from the band of this K-th value), 2 buffer overflow (massive ties:
//       redone by the general kernel of scan.cuh);
//   a11 writes certified rows: original ids and the bit patterns of D (the
//       correctly rounded square roots are taken afterwards, k_sqrt_rows).
#pragma once
#include "common.cuh"
#include "scan.cuh"
#include "dist32.cuh"
#include "scan2_launch.h"
// diagnostic phase timing and event counts (compiled away unless built with
// -DKNN_PHASE_TIMING): the KNN_PT / KNN_CNT / KNN_ITEM markers below
#include "scan2_debug.cuh"

namespace knn {


// Runs of at least S2_BIG points are scanned in super-tiles of S2_SUPER
// consecutive points, each skipped by the queries it cannot serve.
#ifndef S2_BIG
#define S2_BIG 256
#endif
#ifndef S2_SUPER
#define S2_SUPER 128
#endif
// Super-tiles are visited in groups of S2_MEGA (a mega-tile): a group whose
// key-range box no query of the item can use is skipped whole, so a query
// whose neighbourhood holds long runs far from it pays one box test per
// S2_MEGA * S2_SUPER points instead of one per S2_SUPER.
#ifndef S2_MEGA
#define S2_MEGA 32
#endif

// Smallest d whose tiles score two queries at a time.
#ifndef S2_PAIR_DIM
#define S2_PAIR_DIM 5
#endif

// Smallest d scanned two tiles (64 candidates) at a time.
#ifndef S2_WIDE_DIM
#define S2_WIDE_DIM 2
#endif

// Resident CTAs per SM the register allocation is sized for (5: 96
// registers a thread).  At d <= 2 the shared memory of 64-entry buffers
// leaves room for 6 (80 registers), measured 5% faster on 2M-point 2-D sets.
#ifndef S2_MIN_CTAS
#define S2_MIN_CTAS 5
#endif
#ifndef S2_MIN_CTAS_2D
#define S2_MIN_CTAS_2D 6
#endif
// The same for the instances with 128- or 256-entry buffers.  5 spills a
// few registers there; 4 (no spills) was measured 4-9% slower on the 2M
// exponential sets: the fifth CTA's warps hide more latency.
#ifndef S2_MIN_CTAS_BIG
#define S2_MIN_CTAS_BIG 5
#endif

// Start-threshold prefilter of a pass, in units of the squared certificate
// radius (0: none).
#ifndef KNN_PREFILTER_R2
#define KNN_PREFILTER_R2 1.0f
#endif

// Neighbour offsets of the 3^d box, nearest first: for each d the offset
// codes (base-3 digits, digit 1 = no move) ordered by how many dimensions
// move (0, then faces, edges, ...).  Filled once per device by the host; read
// through the read-only data cache (lanes read different entries, which the
// constant cache would serialise).
constexpr int NB_ORDER_TOTAL = 3 + 9 + 27 + 81 + 243 + 729 + 2187 + 6561;
__device__ uint16_t g_nb_order[NB_ORDER_TOTAL];
__host__ __device__ constexpr int nb_order_offset(int d)
{
    return d <= 1 ? 0 : nb_order_offset(d - 1) + (d == 2 ? 3 : d == 3 ? 9 : d == 4 ? 27 : d == 5 ? 81 : d == 6 ? 243 : d == 7 ? 729 : 2187);
}

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
static __device__ uint32_t warp_select_hi(const uint64_t *buf, int cnt, int k, uint32_t *hist, int lane)
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
static __device__ int warp_compact_hi(uint64_t *buf, int cnt, uint32_t thr, int lane)
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
    return a.rcap > 0.0f ? fminf(R, a.rcap) : R;  // the paper's policy: K within eps
}

// K-th smallest (1 <= k <= cnt <= 32*E) of the high 32 bits of
// buf[0..cnt), by a warp bitonic sort of the words (E per lane); for small
// buffers this takes about half the instructions of the radix select.
template <int E>
__device__ __forceinline__ uint32_t warp_kth_hi_sort(const uint64_t *buf, int cnt, int k, int lane)
{
    uint32_t v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int g = lane * E + e;
        v[e] = g < cnt ? (uint32_t)(buf[g] >> 32) : 0xffffffffu;
    }
    warp_bitonic_u32<E>(v, lane);
    uint32_t r = 0;
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (e == (k - 1) % E) r = v[e];
    return __shfl_sync(FULL, r, (k - 1) / E);
}

// Buffer full: find its K-th value T, lower the threshold to the band of T
// and keep only the entries within it.  Returns (new count, new threshold
// bits).  Kept out of line: it runs rarely.
template <int E>
static __device__ __noinline__ int2 shrink_buffer(uint64_t *bi, int c0, int K, uint32_t *hist, int lane, float thr)
{
    __syncwarp();
    const uint32_t T = E <= 2 ? warp_kth_hi_sort<E>(bi, c0, K, lane) : warp_select_hi(bi, c0, K, hist, lane);
    float nt = fminf(thr, band_thr(T));
    int c1 = warp_compact_hi(bi, c0, __float_as_uint(nt), lane);
    __syncwarp();
    return make_int2(c1, __float_as_int(nt));
}

// The query-pair rows and the contiguous thresholds follow the query rows
// in a warp's shared memory (Scan2Warp).
template <int DIM, int E>
__device__ __forceinline__ float *scan2_qq(float *qc)
{
    return qc + scan2_queries_per_item(E) * query_row_floats(DIM);
}
template <int DIM, int E>
__device__ __forceinline__ float *scan2_thrv(float *qc)
{
    return scan2_qq<DIM, E>(qc) + qpair_floats(DIM, scan2_queries_per_item(E), E);
}
// The bound a neighbour cell's rounded-down squared distance must not
// exceed for a query of threshold t: t with a 2^-19 margin for the FP32
// rounding of candidate distances.
__device__ __forceinline__ float cell_test_thr(float t) { return t * (1.0f + 0x1p-19f); }

// Query i's threshold, in every copy (its row, its query pair's row) and
// its cell-test bound (contiguous, for vector loads).
template <int DIM, int E>
__device__ __forceinline__ void scan2_set_thr(float *qc, int i, float t)
{
    qc[i * query_row_floats(DIM) + DIM] = t;
    scan2_thrv<DIM, E>(qc)[i] = cell_test_thr(t);
    if (scan2_qpair(DIM, E)) scan2_qq<DIM, E>(qc)[(i >> 1) * qpair_row_floats(DIM) + 2 * DIM + (i & 1)] = t;
}

// Append this tile's accepted candidates (ballot `bal`) to query i's buffer;
// on overflow shrink it to the band of its K-th value first, and mark the
// query for the general kernel (count -1, threshold -1) if even that does
// not make room.  The count of query i lives in lane i's `my_cnt`.
template <int DIM, int E>
__device__ __forceinline__ void scan2_insert(uint64_t *buf, float *qc, uint32_t *hist, int &my_cnt, int i,
                                             bool acc, uint32_t bal, float d2, uint32_t s, int K, float ti,
                                             int lane KNN_CNT_PARAM)
{
    KNN_CNT(9, 1);
    constexpr int B = 32 * E;
    uint64_t *bi = buf + i * B;
    int c0 = __shfl_sync(FULL, my_cnt, i);
    int nnew = __popc(bal);
    if (c0 + nnew > B) {
        KNN_CNT(10, 1);
        // buffer full: drop to the K-th value's band (rare)
        int2 r2 = shrink_buffer<E>(bi, c0, K, hist, lane, ti);
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
        if (lane == 0) scan2_set_thr<DIM, E>(qc, i, tnew);
        __syncwarp();
    }
    if (acc && KNN_GUARD(c0 >= 0 && c0 + __popc(bal & lanemask_lt()) < B, 4))
        bi[c0 + __popc(bal & lanemask_lt())] = ((uint64_t)__float_as_uint(d2) << 32) | s;
    if (lane == i) my_cnt = c0 < 0 ? -1 : c0 + nnew;
}

// Queries (bit i = query i) that points [sb, se) of the sorted order can
// serve.  Those keys share their bits above the highest bit in which the
// first and last differ, so the points lie in the box of that key prefix:
// in dimension k the level-0 cells whose low fb_k bits are free, fb_k = the
// number of key bits of dimension k below that bit.  A query is dropped when
// the rounded-down squared distance to the box exceeds its threshold (with
// the 2^-19 margin of the cell test).
template <int DIM>
__device__ __forceinline__ uint32_t super_tile_mask(const ScanArgs &a, uint32_t sb, uint32_t se, const float *qc,
                                                    int Q, int lane)
{
    constexpr int QP = query_row_floats(DIM);
    const uint64_t k0 = KNN_GUARD(se <= (uint64_t)a.n && sb < se, 3) ? a.keys[sb] : 0,
                   k1 = KNN_GUARD(se <= (uint64_t)a.n && sb < se, 3) ? a.keys[se - 1] : ~0ull;
    const uint64_t x = k0 ^ k1;
    const int hb = x ? 64 - __clzll((long long)x) : 0;  // free low key bits
    float blo = 0.0f, bhi = 0.0f;
    if (lane < DIM) {
        const int fb = hb > lane ? (hb - lane + DIM - 1) / DIM : 0;
        if (fb >= 30) {
            blo = -__int_as_float(0x7f800000);
            bhi = __int_as_float(0x7f800000);
        } else {
            int cc = 0;
            for (int b = fb; b < a.bits; ++b) cc |= (int)((k0 >> (b * DIM + lane)) & 1u) << b;
            blo = face_of(cc, a.lo[lane], a.w0);
            bhi = face_of(cc + (1 << fb), a.lo[lane], a.w0);
        }
    }
    float lb = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const float lo = __shfl_sync(FULL, blo, k), hi = __shfl_sync(FULL, bhi, k);
        if (lane < Q) {
            const float q = qc[lane * QP + k];
            const float g = fmaxf(fmaxf(__fsub_rd(lo, q), __fsub_rd(q, hi)), 0.0f);
            lb = __fadd_rd(lb, __fmul_rd(g, g));
        }
    }
    const bool keep = lane < Q && !(lb > qc[lane * QP + DIM] * (1.0f + 0x1p-19f));
    return __ballot_sync(FULL, keep);
}

// The same test for 32 ranges at once: each lane tests its own range [sb,
// se) (valid lanes) against every query of the item -- one round of key
// loads for 32 super-tiles instead of 32 dependent rounds.  Same box, same
// rounding (the squared gaps summed in dimension order, rounded down) and
// margin as super_tile_mask.
template <int DIM>
__device__ __forceinline__ uint32_t tile_mask_lane(const ScanArgs &a, uint32_t sb, uint32_t se, bool valid,
                                                   const float *qc, int Q)
{
    valid = valid && KNN_GUARD(se <= (uint64_t)a.n && sb < se, 3);
    const uint64_t k0 = valid ? a.keys[sb] : 0, k1 = valid ? a.keys[se - 1] : 0;
    const uint64_t x = k0 ^ k1;
    const int hb = x ? 64 - __clzll((long long)x) : 0;  // free low key bits
    float blo[DIM], bhi[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const int fb = hb > k ? (hb - k + DIM - 1) / DIM : 0;
        if (fb >= 30) {
            blo[k] = -__int_as_float(0x7f800000);
            bhi[k] = __int_as_float(0x7f800000);
        } else {
            int cc = 0;
            for (int b = fb; b < a.bits; ++b) cc |= (int)((k0 >> (b * DIM + k)) & 1u) << b;
            blo[k] = face_of(cc, a.lo[k], a.w0);
            bhi[k] = face_of(cc + (1 << fb), a.lo[k], a.w0);
        }
    }
    uint32_t m = 0;
    for (int i = 0; i < Q; ++i) {
        float q[DIM], thr;
        uint32_t qs;
        load_query_row<DIM>(qc, i, q, thr, qs);
        float lb = 0.0f;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const float g = fmaxf(fmaxf(__fsub_rd(blo[k], q[k]), __fsub_rd(q[k], bhi[k])), 0.0f);
            lb = __fadd_rd(lb, __fmul_rd(g, g));
        }
        if (!(lb > thr * (1.0f + 0x1p-19f))) m |= 1u << i;
    }
    return valid ? m : 0u;
}

// Score one tile (lane = candidate s with coordinates c, `valid` lanes only)
// against the queries in `tmask` and append the accepted ones to their buffers.
template <int DIM, int E>
__device__ __forceinline__ void scan2_tile(const float (&c)[DIM], uint32_t s, bool valid, uint32_t tmask,
                                           uint64_t *buf, float *qc, uint32_t *hist, int &my_cnt, int K, int lane
                                           KNN_CNT_PARAM)
{
    // the queries this tile can serve; for d >= S2_PAIR_DIM, two at a time
    // (independent dependency chains: a query's threshold only
    // changes in its own insert, so both use current thresholds)
    if (DIM >= S2_PAIR_DIM) {
        for (uint32_t m = tmask; m;) {
            const int i0 = __ffs(m) - 1;
            m &= m - 1;
            const int i1 = m ? __ffs(m) - 1 : i0;
            const bool two = m != 0;
            m &= m - 1;
            float q0[DIM], q1[DIM], t0v, t1v;
            uint32_t s0, s1;
            load_query_row<DIM>(qc, i0, q0, t0v, s0);
            load_query_row<DIM>(qc, i1, q1, t1v, s1);
            const float d0 = dist2_f32<DIM>(q0, c);
            const float d1 = dist2_f32<DIM>(q1, c);
            const bool acc0 = valid && d0 <= t0v && s != s0;
            const bool acc1 = two && valid && d1 <= t1v && s != s1;
            const uint32_t bal0 = __ballot_sync(FULL, acc0);
            const uint32_t bal1 = __ballot_sync(FULL, acc1);
            if (bal0) scan2_insert<DIM, E>(buf, qc, hist, my_cnt, i0, acc0, bal0, d0, s, K, t0v, lane KNN_CNT_ARG);
            if (bal1) scan2_insert<DIM, E>(buf, qc, hist, my_cnt, i1, acc1, bal1, d1, s, K, t1v, lane KNN_CNT_ARG);
        }
    } else {
        for (uint32_t m = tmask; m; m &= m - 1) {
            const int i = __ffs(m) - 1;
            float qv[DIM], ti;
            uint32_t qi_s;
            load_query_row<DIM>(qc, i, qv, ti, qi_s);
            const float d2 = dist2_f32<DIM>(qv, c);
            const bool acc = valid && d2 <= ti && s != qi_s;
            const uint32_t bal = __ballot_sync(FULL, acc);
            if (bal) scan2_insert<DIM, E>(buf, qc, hist, my_cnt, i, acc, bal, d2, s, K, ti, lane KNN_CNT_ARG);
        }
    }
}

// Two tiles at once (lane = candidates sA and sB, NaN coordinates past the
// end of the list): each query's row is read
// once for 64 candidates and its two distances are independent chains.  The
// second batch may be tested against a threshold the first batch's insert
// has since lowered; that only keeps extra entries (the buffer holds a
// superset of what its threshold admits).
// The acceptances of one query in a two-tile step (ballots accA / accB over
// the lanes) go to its buffer.  The first tile's insert may have shrunk the
// buffer and lowered the threshold, or marked the query for the general
// kernel (threshold -1, count -1): the second tile is tested again, so that
// nothing is appended to a marked query's buffer.
template <int DIM, int E>
__device__ __forceinline__ void scan2_insert_pair(uint64_t *buf, float *qc, uint32_t *hist, int &my_cnt, int i,
                                                  bool accA, bool accB, float dA, float dB, uint32_t sA,
                                                  uint32_t sB, float ti, int K, int lane KNN_CNT_PARAM)
{
    KNN_CNT(11, 1);
    KNN_CYC_BEGIN(ins);
    const uint32_t balA = __ballot_sync(FULL, accA);
    uint32_t balB = __ballot_sync(FULL, accB);
    if (!(balA | balB)) return;
    {
        // common case: both tiles' acceptances fit in the buffer -- one read
        // of the count, both appended, no threshold change in between
        constexpr int B = 32 * E;
        const int c0 = __shfl_sync(FULL, my_cnt, i);
        const int nA = __popc(balA), nB = __popc(balB);
        if (c0 >= 0 && c0 + nA + nB <= B) {
            uint64_t *bi = buf + i * B;
            const uint32_t lt = lanemask_lt();
            const int pA = c0 + __popc(balA & lt), pB = c0 + nA + __popc(balB & lt);
            if (accA && KNN_GUARD(pA < B, 4)) bi[pA] = ((uint64_t)__float_as_uint(dA) << 32) | sA;
            if (accB && KNN_GUARD(pB < B, 4)) bi[pB] = ((uint64_t)__float_as_uint(dB) << 32) | sB;
            if (lane == i) my_cnt = c0 + nA + nB;
            KNN_CYC_END(ins, 15);
            return;
        }
    }
    // the buffer fills: tile A first (its insert may shrink the buffer)
    float tB = ti;
    if (balA) {
        scan2_insert<DIM, E>(buf, qc, hist, my_cnt, i, accA, balA, dA, sA, K, ti, lane KNN_CNT_ARG);
        tB = qc[i * query_row_floats(DIM) + DIM];
        balB = __ballot_sync(FULL, accB && dB <= tB);
    }
    if (balB) scan2_insert<DIM, E>(buf, qc, hist, my_cnt, i, accB && dB <= tB, balB, dB, sB, K, tB, lane KNN_CNT_ARG);
    KNN_CYC_END(ins, 15);
}

// Two tiles at once (lane = candidates sA and sB, NaN coordinates past the
// end of the list): each query's row is read once for 64 candidates and its
// two distances are computed together (packed FP32).  The second batch may
// be tested against a threshold the first batch's insert has since lowered;
// that only keeps extra entries (the buffer holds a superset of what its
// threshold admits).  (Scoring two queries per iteration was measured
// slower on every workload.)
template <int DIM, int E>
__device__ __forceinline__ void scan2_tile_wide(const float (&cA)[DIM], const float (&cB)[DIM], uint32_t sA,
                                                uint32_t sB, uint32_t tmask, uint64_t *buf, float *qc,
                                                uint32_t *hist, int &my_cnt, int K, int lane KNN_CNT_PARAM)
{
    if constexpr (scan2_qpair(DIM, E)) {
        // queries two at a time: the pair's row holds each coordinate of
        // queries 2p and 2p + 1 in one 64-bit word, and each candidate's
        // coordinate is duplicated into both halves once per step, so one
        // packed chain gives the candidate's distances to both queries.
        // Pairs with either query in the mask are scored; the other query
        // of such a pair is scored too (its cell test is a pruning bound
        // only, and accepting what its threshold admits keeps its buffer
        // a superset of that set); a missing query (odd count) has NaN
        // coordinates and accepts nothing.
        constexpr int QQ = qpair_row_floats(DIM);
        const float *qq = scan2_qq<DIM, E>(qc);
        unsigned long long ca[DIM], cb[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            ca[k] = f32x2_pack(cA[k], cA[k]);
            cb[k] = f32x2_pack(cB[k], cB[k]);
        }
        for (uint32_t pm = (tmask | (tmask >> 1)) & 0x55555555u; pm; pm &= pm - 1) {
            const int i0 = __ffs(pm) - 1;  // even
            unsigned long long r[QQ / 2];
            const ulonglong2 *row = (const ulonglong2 *)(qq + (i0 >> 1) * QQ);
#pragma unroll
            for (int v = 0; v < QQ / 4; ++v) {
                const ulonglong2 t = row[v];
                r[2 * v] = t.x;
                r[2 * v + 1] = t.y;
            }
            unsigned long long qp[DIM];
#pragma unroll
            for (int k = 0; k < DIM; ++k) qp[k] = r[k];
            float t0, t1, u0f, u1f, dA0, dA1, dB0, dB1;
            f32x2_unpack(r[DIM], t0, t1);
            f32x2_unpack(r[DIM + 1], u0f, u1f);
            const uint32_t u0 = __float_as_uint(u0f), u1 = __float_as_uint(u1f);
            dist2_f32_x2q<DIM>(qp, ca, dA0, dA1);
            dist2_f32_x2q<DIM>(qp, cb, dB0, dB1);
            const bool aA0 = dA0 <= t0 && sA != u0, aB0 = dB0 <= t0 && sB != u0;  // NaN past the end
            const bool aA1 = dA1 <= t1 && sA != u1, aB1 = dB1 <= t1 && sB != u1;
            if (DIM < 5 || __any_sync(FULL, aA0 || aB0 || aA1 || aB1)) {
                scan2_insert_pair<DIM, E>(buf, qc, hist, my_cnt, i0, aA0, aB0, dA0, dB0, sA, sB, t0, K, lane KNN_CNT_ARG);
                scan2_insert_pair<DIM, E>(buf, qc, hist, my_cnt, i0 + 1, aA1, aB1, dA1, dB1, sA, sB, t1, K, lane KNN_CNT_ARG);
            }
        }
    } else {
        // the two candidates' coordinates packed per dimension (once per step)
        unsigned long long cp[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) cp[k] = f32x2_pack(cA[k], cB[k]);
        for (uint32_t m = tmask; m; m &= m - 1) {
            const int i = __ffs(m) - 1;
            float qv[DIM], ti;
            uint32_t qi_s;
            load_query_row<DIM>(qc, i, qv, ti, qi_s);
            float dA, dB;
            dist2_f32_x2<DIM>(qv, cp, dA, dB);
            const bool accA = dA <= ti && sA != qi_s;  // NaN past the end
            const bool accB = dB <= ti && sB != qi_s;
            // one vote first for d >= 5, where a step usually accepts nothing
            if (DIM < 5 || __any_sync(FULL, accA || accB))
                scan2_insert_pair<DIM, E>(buf, qc, hist, my_cnt, i, accA, accB, dA, dB, sA, sB, ti, K, lane KNN_CNT_ARG);
        }
    }
}

// One super-tile [sb, se), one tile of 32 candidates per step.
template <int DIM, int E>
__device__ __forceinline__ void scan2_super_tile(const ScanArgs &a, uint32_t sb, uint32_t se, uint32_t smask,
                                                 uint64_t *buf, float *qc, uint32_t *hist, int &my_cnt, int K,
                                                 int lane, unsigned long long &st_cand KNN_CNT_PARAM)
{
    for (uint32_t t0 = sb; t0 < se; t0 += 32) {
        const bool valid = t0 + lane < se;
        const uint32_t s = valid ? t0 + lane : 0u;
        float c[DIM];
        if (valid) {
            load_point<DIM>(a.xsort, s, c);
            st_cand += (unsigned long long)__popc(smask);
        } else {
#pragma unroll
            for (int k = 0; k < DIM; ++k) c[k] = 0.0f;
        }
        scan2_tile<DIM, E>(c, s, valid, smask, buf, qc, hist, my_cnt, K, lane KNN_CNT_ARG);
    }
}

// Slices of one warp's shared memory in k_scan2 (sizes: scan2_warp_bytes).
template <int DIM, int QM, int E>
struct Scan2Warp {
    uint64_t *buf;   // [QM][32E]  (d2_32 bits << 32 | sorted index)
    uint64_t *dil;   // [3d] key parts (or dense index terms) of neighbour coordinates
    float *qc;       // [QM][QP] coords, threshold, sorted position
    float *qq;       // [QM/2][QQ] query pairs (scan2_qpair): coords, thresholds, positions
    float *thrv;     // [QM] cell-test bounds of the thresholds, contiguous (vector loads)
    int *cnt;        // [QM]
    uint32_t *qsv;   // [QM]
    uint32_t *hist;  // [hist_entries] (or the face-gap table: hist_aliased)
    // [3d][QM]: per dimension, the squared distance (rounded down) from each
    // query to the lower neighbour cell, 0 (same slab), to the upper one --
    // row 3k + g for the base-3 digit g of a neighbour offset in dimension k,
    // queries contiguous (a lane reads every query's gap with vector loads)
    float *gsq;
    float *rcert;    // [QM] certificate radius of each query
    int *cellv;      // [2d] the item's cell and the level's extent
    static_assert(QM == scan2_queries_per_item(E), "queries per item follow the buffer size");
    __device__ __forceinline__ explicit Scan2Warp(unsigned char *wb)
    {
        buf = (uint64_t *)wb;
        dil = buf + QM * 32 * E;
        qc = (float *)(dil + dil_entries(DIM));
        qq = qc + QM * query_row_floats(DIM);
        thrv = qq + qpair_floats(DIM, QM, E);
        cnt = (int *)(thrv + QM);
        qsv = (uint32_t *)(cnt + QM);
        uint32_t *own_hist = qsv + QM;
        gsq = (float *)(own_hist + hist_entries(DIM, QM, E));
        hist = hist_aliased(DIM, QM, E) ? (uint32_t *)gsq : own_hist;
        rcert = gsq + 3 * DIM * QM;
        cellv = (int *)(rcert + QM);
    }
};

// 2^F as a float for the fixed-point distance from FP32 differences (0: F
// outside the normal exponent range, that path unused).
__device__ __forceinline__ float scan2_fixed_scale(const ScanArgs &a)
{
    return (a.fixed_ok && a.F >= -126 && a.F <= 127) ? __int_as_float((a.F + 127) << 23) : 0.0f;
}

// A warp's candidate and band counts into the join's statistics.
__device__ __forceinline__ void scan2_flush_stats(const ScanArgs &a, unsigned long long st_cand,
                                                  unsigned long long st_band, int lane)
{
    for (int o = 16; o; o >>= 1) {
        st_cand += __shfl_xor_sync(FULL, st_cand, o);
        st_band += __shfl_xor_sync(FULL, st_band, o);
    }
    if (lane == 0) {
        if (st_cand) atomicAdd(&a.stats[0], st_cand);
        if (st_band) atomicAdd(&a.stats[2], st_band);
    }
}

// MEGA selects the long-run walk: false, every super-tile tested in turn
// (uniform data: the code of the hot loop stays as compiled without it);
// true, mega-tiles tested first and skipped whole, two tiles per step
// (density skew and re-queued passes, where one query's box can hold long
// runs far from it).
// One work item (a7-a11): its queries against their neighbour cells.
template <int DIM, int QM, int E, bool MEGA>
__device__ __forceinline__ void scan2_item(const ScanArgs &a, uint32_t item, const Scan2Warp<DIM, QM, E> &w,
                                           int lane, float fsc, unsigned long long &st_cand,
                                           unsigned long long &st_band KNN_CNT_PARAM)
{
    constexpr int P = pad_dim(DIM);
    constexpr int QP = query_row_floats(DIM);
    constexpr int B = 32 * E;
    constexpr int BS = B;
    constexpr int GQ = 3 * DIM;
    (void)P;
    (void)GQ;
    const int K = a.K, NOFF = a.noff;
    uint64_t *const buf = w.buf;
    uint64_t *const dil = w.dil;
    float *const qc = w.qc;
    float *const thrv = w.thrv;
    int *const cnt = w.cnt;
    uint32_t *const qsv = w.qsv;
    uint32_t *const hist = w.hist;
    float *const gsq = w.gsq;
    float *const rcert = w.rcert;
    int *const cellv = w.cellv;
    KNN_ITEM_BEGIN;
    const uint2 it = a.items[item];
    const int Q = (int)(it.y & 0xffffu);
    const int level = (int)(it.y >> 16);
    const int shift = DIM * level;
    const int nbits = a.bits - level;
    const LevelRef lr = a.levels[level];
    const uint4 *hslot = lr.hslot;
    const uint32_t hmask = lr.hmask;
    const uint2 *dtab = lr.dense;  // dense cell table, or null: the hash map

    if (lane < Q && KNN_GUARD(it.x + lane < (uint64_t)a.nactive, 0)) {
        uint32_t s = a.active[it.x + lane];
        if (!KNN_GUARD(s < (uint64_t)a.nq, 1)) s = 0;
        float c[DIM];
        load_point<DIM>(a.qxsort, s, c);
        qsv[lane] = s;
#pragma unroll
        for (int k = 0; k < DIM; ++k) qc[lane * QP + k] = c[k];
    }
    __syncwarp();
    // the item's cell at its level and the level's last cell index, kept
    // in shared memory (cellv) rather than registers across the scan
    {
        int cell[DIM];
        morton_decode(a.qkeys[qsv[0]] >> shift, DIM, nbits, cell);
        if (lane < DIM) {
#pragma unroll
            for (int k = 0; k < DIM; ++k)
                if (k == lane) {
                    cellv[k] = cell[k];
                    cellv[DIM + k] = a.cmax0[k] >> level;
                }
        }
    }
    __syncwarp();
    const int *cell = cellv, *cmaxL = cellv + DIM;
    // neighbour keys by parts: dil[3k + g] holds the part of coordinate k
    // of the neighbour at digit g (cell[k] + g - 1) -- its level-key
    // bits, or with a dense cell table its term c * stride_k of the
    // table index -- so a neighbour's key or index is the sum of d table
    // entries (the key parts occupy disjoint bits: sum = OR); bit 3k + g
    // of nbad marks a coordinate outside the level's grid
    uint32_t nbad;
    {
        bool bad = false;
        if (lane < 3 * DIM) {
            const int k = lane / 3;
            const int c = cell[k] + lane % 3 - 1;
            bad = c < 0 || c > cmaxL[k];
            uint64_t v = 0;
            if (dtab) {
                uint32_t st = 1;
                for (int j = 0; j < k; ++j) st *= (uint32_t)cmaxL[j] + 1u;
                v = bad ? 0 : (uint64_t)((uint32_t)c * st);
            } else {
                for (int b = 0; b < nbits; ++b) v |= (uint64_t)((c >> b) & 1) << (b * DIM + k);
            }
            dil[lane] = v;
        }
        nbad = __ballot_sync(FULL, bad);
    }
    __syncwarp();
    // query state: threshold and sorted position sit in the query's row
    // (one broadcast vector load gives a pair everything it needs); the
    // buffer count lives in lane i's register for query i
    int my_cnt = 0;
    if (lane < Q) {
        float q[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) q[k] = qc[lane * QP + k];
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            // q lies in [face(c), face(c+1)) exactly, so both gaps are >= 0
            const float gl = __fsub_rd(q[k], face_of(cell[k] << level, a.lo[k], a.w0));
            const float gh = __fsub_rd(face_of((cell[k] + 1) << level, a.lo[k], a.w0), q[k]);
            gsq[(3 * k) * QM + lane] = __fmul_rd(gl, gl);
            gsq[(3 * k + 1) * QM + lane] = 0.0f;
            gsq[(3 * k + 2) * QM + lane] = __fmul_rd(gh, gh);
        }
        // start threshold: the certificate prefilter KNN_PREFILTER_R2 x R^2
        // (points beyond R cannot be in a certified answer), or the band
        // of the K-th value an earlier pass found in a smaller box
        // (contained in this one), whichever is lower
        const float R = cert_radius<DIM>(q, cell, cmaxL, a, level);
        rcert[lane] = R;
        const float thr0 = (KNN_PREFILTER_R2 <= 0.0f || isinf(R))
                               ? __int_as_float(0x7f800000)
                               : __fmul_ru(__fmul_ru(R, R), KNN_PREFILTER_R2 * (1.0f + 0x1p-14f));
        const float t0 = fminf(thr0, a.seed[qsv[lane]]);
        qc[lane * QP + DIM] = t0;
        thrv[lane] = cell_test_thr(t0);
        // the data position a candidate must not equal (none for R x S)
        qc[lane * QP + DIM + 1] = __uint_as_float(a.self ? qsv[lane] : 0xffffffffu);
    }
    if constexpr (scan2_qpair(DIM, E)) {
        // the query-pair rows; the partner of the last query of an odd
        // count has NaN coordinates and threshold -1 (accepts nothing)
        if (lane < ((Q + 1) & ~1)) {
            float *pr = w.qq + (lane >> 1) * qpair_row_floats(DIM) + (lane & 1);
            const bool real = lane < Q;
#pragma unroll
            for (int k = 0; k < DIM; ++k) pr[2 * k] = real ? qc[lane * QP + k] : __int_as_float(0x7fc00000);
            pr[2 * DIM] = real ? qc[lane * QP + DIM] : -1.0f;
            pr[2 * DIM + 2] = real ? qc[lane * QP + DIM + 1] : __uint_as_float(0xffffffffu);
        }
    }
    __syncwarp();

    KNN_PT(0);
    const uint32_t qmask = Q >= 32 ? ~0u : (1u << Q) - 1u;  // the item's queries
    // a7 + a8
    for (int ob = 0; ob < NOFF; ob += 32) {
        const int o = ob + lane;
        uint32_t rb = 0, re = 0;
        int goff[DIM];  // offset of this cell's squared gap, per dimension
#pragma unroll
        for (int k = 0; k < DIM; ++k) goff[k] = 3 * k + 1;
        if (o < NOFF) {
            int r = __ldg(&g_nb_order[nb_order_offset(DIM) + o]);
            uint64_t key = 0;
            uint32_t hit = 0;
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                goff[k] = 3 * k + r % 3;
                r /= 3;
                key += dil[goff[k]];
                hit |= nbad >> goff[k];
            }
            if (!(hit & 1u)) {
                const uint2 rg = dtab ? __ldg(&dtab[(uint32_t)key]) : hash_lookup(hslot, hmask, key);
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
            // lower bounds of all QM queries at once: the rows of this
            // cell's digits, read as vectors, summed rounding down, two
            // queries per packed add (each half rounds as __fadd_rd)
            unsigned long long lb2[QM / 2];
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                const ulonglong2 *row = (const ulonglong2 *)(gsq + goff[k] * QM);
#pragma unroll
                for (int v = 0; v < QM / 4; ++v) {
                    const ulonglong2 t = row[v];
                    lb2[2 * v] = k == 0 ? t.x : f32x2_add_rd(lb2[2 * v], t.x);
                    lb2[2 * v + 1] = k == 0 ? t.y : f32x2_add_rd(lb2[2 * v + 1], t.y);
                }
            }
            // against the cell-test bounds (lanes past the item's queries
            // hold stale values: masked off below)
#pragma unroll
            for (int v = 0; v < QM / 4; ++v) {
                const float4 t = ((const float4 *)thrv)[v];
                float l0, l1, l2, l3;
                f32x2_unpack(lb2[2 * v], l0, l1);
                f32x2_unpack(lb2[2 * v + 1], l2, l3);
                if (!(l0 > t.x)) cmask |= 1u << (4 * v);
                if (!(l1 > t.y)) cmask |= 1u << (4 * v + 1);
                if (!(l2 > t.z)) cmask |= 1u << (4 * v + 2);
                if (!(l3 > t.w)) cmask |= 1u << (4 * v + 3);
            }
            cmask &= qmask;
        }
        KNN_CNT(3, __popc(__ballot_sync(FULL, len != 0)));
        KNN_CNT(4, __popc(__ballot_sync(FULL, cmask != 0)));
        // long runs first, outside the flattened scan
        const bool bigcell = len >= S2_BIG;
        const uint32_t bigmask = __ballot_sync(FULL, bigcell && cmask != 0);
        // long runs: super-tiles, starting at the one that holds the
        // item's first query when it lies in the run (nearby in key order
        // is mostly nearby in space) and alternating outwards
        for (uint32_t bm = bigmask; bm; bm &= bm - 1) {
            const int src = __ffs(bm) - 1;
            const uint32_t cb = __shfl_sync(FULL, rb, src), ce = __shfl_sync(FULL, re, src);
            const uint32_t cmk = __shfl_sync(FULL, cmask, src);
            const int nst = (int)((ce - cb + S2_SUPER - 1) / S2_SUPER);
            const uint32_t sq = qsv[0];
            const int u0 = (a.self && sq >= cb && sq < ce) ? (int)((sq - cb) / S2_SUPER) : 0;
            if constexpr (MEGA) {
                // super-tiles visited outwards from u0 (u0, u0 + 1, u0 - 1,
                // u0 + 2, ...) in rounds of 32: each lane tests the box of one
                // super-tile of the round against every query of the item,
                // and the tiles some query can use are scanned in walk order
                // (a tile's mask is from the round's start: thresholds only
                // fall, so it keeps every query that can still use it)
                const int above = nst - 1 - u0, below = u0;
                const int mlo = min(above, below);
                for (int base = 0; base < nst; base += 32) {
                    const int w = base + lane;
                    const bool valid = w < nst;
                    int u = 0;
                    if (valid) {
                        if (w <= 2 * mlo) u = (w & 1) ? u0 + (w + 1) / 2 : u0 - w / 2;
                        else u = above > below ? u0 + (w - mlo) : u0 - (w - mlo);
                    }
                    const uint32_t lsb = cb + (uint32_t)u * S2_SUPER;
                    const uint32_t lse = min(lsb + (uint32_t)S2_SUPER, ce);
                    const uint32_t lm = tile_mask_lane<DIM>(a, lsb, lse, valid, qc, Q) & cmk;
                    KNN_CNT(7, __popc(__ballot_sync(FULL, valid)));
                    for (uint32_t todo = __ballot_sync(FULL, lm != 0); todo; todo &= todo - 1) {
                        const int src = __ffs(todo) - 1;
                        const uint32_t smask = __shfl_sync(FULL, lm, src);
                        const uint32_t sb = __shfl_sync(FULL, lsb, src), se = __shfl_sync(FULL, lse, src);
                        KNN_CNT(6, 1);
                        if (DIM >= S2_WIDE_DIM) {
                            // two tiles per step, as for the flattened runs
                            for (uint32_t t0 = sb; t0 < se; t0 += 64) {
                                const bool vA = t0 + lane < se, vB = t0 + 32 + lane < se;
                                const uint32_t sA = vA ? t0 + lane : 0u, sB = vB ? t0 + 32 + lane : 0u;
                                float cA[DIM], cB[DIM];
#pragma unroll
                                for (int k = 0; k < DIM; ++k) cA[k] = cB[k] = __int_as_float(0x7fc00000);
                                if (vA) load_point<DIM>(a.xsort, sA, cA);
                                if (vB) load_point<DIM>(a.xsort, sB, cB);
                                st_cand += (unsigned long long)__popc(smask) * ((vA ? 1u : 0u) + (vB ? 1u : 0u));
                                KNN_ITEM_TILE(__popc(smask) * 2);
                                scan2_tile_wide<DIM, E>(cA, cB, sA, sB, smask, buf, qc, hist, my_cnt, K, lane KNN_CNT_ARG);
                            }
                        } else {
                            scan2_super_tile<DIM, E>(a, sb, se, smask, buf, qc, hist, my_cnt, K, lane, st_cand KNN_CNT_ARG);
                        }
                    }
                }
            } else {
                // super-tiles alternating outwards from u0, one tile per step
                for (int j = 0, left = nst; left > 0; ++j) {
                    const int u = (j & 1) ? u0 + (j + 1) / 2 : u0 - j / 2;
                    if (u < 0 || u >= nst) continue;
                    --left;
                    const uint32_t sb = cb + (uint32_t)u * S2_SUPER;
                    const uint32_t se = min(sb + (uint32_t)S2_SUPER, ce);
                    const uint32_t smask = super_tile_mask<DIM>(a, sb, se, qc, Q, lane) & cmk;
                    if (!smask) continue;
                    scan2_super_tile<DIM, E>(a, sb, se, smask, buf, qc, hist, my_cnt, K, lane, st_cand KNN_CNT_ARG);
                }
            }
        }
        // (cells that no query of the item can use stay out of the
        // flattened list)
        const uint32_t flen = (bigcell || cmask == 0) ? 0u : len;
        uint32_t inc = flen;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, inc, d);
            if (lane >= d) inc += y;
        }
        const uint32_t exc = inc - flen;
        const uint32_t total = __shfl_sync(FULL, inc, 31);
        KNN_CNT(5, total);
        KNN_PT(1);
        // flattened position t -> (sorted position, cell's query mask)
        auto locate = [&](uint32_t t, bool valid, uint32_t &sp, uint32_t &cmo) {
            int src = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                uint32_t ex = __shfl_sync(FULL, exc, src + step);
                if (ex <= t) src += step;
            }
            const uint32_t sb = __shfl_sync(FULL, rb, src);
            const uint32_t se = __shfl_sync(FULL, exc, src);
            sp = valid ? sb + (t - se) : 0u;
            const uint32_t cm = __shfl_sync(FULL, cmask, src);  // every lane takes part
            cmo = valid ? cm : 0u;
        };
        if (DIM >= S2_WIDE_DIM) {
            for (uint32_t t0 = 0; t0 < total; t0 += 64) {
                KNN_CYC_BEGIN(stp);
                const bool vA = t0 + lane < total, vB = t0 + 32 + lane < total;
                uint32_t sA, sB, cmA, cmB;
                locate(t0 + lane, vA, sA, cmA);
                locate(t0 + 32 + lane, vB, sB, cmB);
                const uint32_t tmask = __reduce_or_sync(FULL, cmA | cmB);
                KNN_CNT(0, 1);
                KNN_CNT(1, __popc(tmask));
                KNN_CNT(2, tmask == 0);
                // lanes past the end get NaN coordinates: every distance
                // comparison with them is false
                float cA[DIM], cB[DIM];
#pragma unroll
                for (int k = 0; k < DIM; ++k) cA[k] = cB[k] = __int_as_float(0x7fc00000);
                if (vA && KNN_GUARD(sA < (uint64_t)a.n, 2)) load_point<DIM>(a.xsort, sA, cA);
                if (vB && KNN_GUARD(sB < (uint64_t)a.n, 2)) load_point<DIM>(a.xsort, sB, cB);
                st_cand += (unsigned long long)__popc(tmask) * ((vA ? 1u : 0u) + (vB ? 1u : 0u));
                KNN_ITEM_TILE(__popc(tmask) * 2);
                KNN_CYC_END(stp, 8);
                scan2_tile_wide<DIM, E>(cA, cB, sA, sB, tmask, buf, qc, hist, my_cnt, K, lane KNN_CNT_ARG);
            }
        } else {
            for (uint32_t t0 = 0; t0 < total; t0 += 32) {
                const bool valid = t0 + lane < total;
                uint32_t s, cmo;
                locate(t0 + lane, valid, s, cmo);
                const uint32_t tmask = __reduce_or_sync(FULL, cmo);
                float c[DIM];
                if (valid) {
                    load_point<DIM>(a.xsort, s, c);
                    st_cand += (unsigned long long)__popc(tmask);  // distances evaluated
                    KNN_ITEM_TILE(__popc(tmask));
                } else {
#pragma unroll
                    for (int k = 0; k < DIM; ++k) c[k] = 0.0f;
                }
                scan2_tile<DIM, E>(c, s, valid, tmask, buf, qc, hist, my_cnt, K, lane KNN_CNT_ARG);
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
            // this lane's own (unsorted) entries g = lane*E + e: their FP32
            // keys, and -- issued now, so that the sort below hides the
            // latency -- the coordinates and original ids of their points
            constexpr bool PREFETCH = E * (DIM + 1) <= 28;
            uint32_t v[E], kr[E], sp[E];
            float pc[PREFETCH ? E : 1][DIM];
            uint32_t pid[PREFETCH ? E : 1];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int g = lane * E + e;
                const uint64_t ent = g < c0 ? bi[g] : ~0ull;
                kr[e] = (uint32_t)(ent >> 32) & ~SLOT;
                sp[e] = (uint32_t)ent;
                v[e] = g < c0 ? (kr[e] | (uint32_t)g) : 0xffffffffu;
                if constexpr (PREFETCH) {
                    const bool ok = g < c0 && KNN_GUARD(sp[e] < (uint64_t)a.n, 7);
                    if (ok) {
                        load_point<DIM>(a.xsort, sp[e], pc[e]);
                        pid[e] = __ldg(&a.perm[sp[e]]);
                    } else {
#pragma unroll
                        for (int k = 0; k < DIM; ++k) pc[e][k] = 0.0f;
                        pid[e] = 0;
                    }
                }
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
            // exact canonical distances and original ids of the band: each
            // lane scores its own unsorted entries that lie in the band (the
            // band is the set of keys <= tb, the same test as above) and
            // parks them by buffer slot -- D over the buffer entry, the id in
            // the histogram area -- where the sorted positions pick them up
            float q[DIM];
            int32_t qi[DIM];
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                q[k] = qc[i * QP + k];
                qi[k] = a.fixed_ok ? to_fixed(q[k], a.F) : 0;
            }
            uint64_t *bw = buf + i * BS;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int g = lane * E + e;
                if (g < c0 && kr[e] <= tb) {
                    float c[DIM];
                    uint32_t id;
                    if constexpr (PREFETCH) {
#pragma unroll
                        for (int k = 0; k < DIM; ++k) c[k] = pc[e][k];
                        id = pid[e];
                    } else {
                        if (KNN_GUARD(sp[e] < (uint64_t)a.n, 7)) {
                            load_point<DIM>(a.xsort, sp[e], c);
                            id = a.perm[sp[e]];
                        } else {
#pragma unroll
                            for (int k = 0; k < DIM; ++k) c[k] = 0.0f;
                            id = 0;
                        }
                    }
                    uint64_t bits = 0;
                    bool done = false;
                    if (a.fixed_ok) {
                        done = fsc != 0.0f && canon_d2_fixed_f32<DIM>(q, c, fsc, a.F, bits);
                        if (!done) {
                            int32_t ci[DIM];
#pragma unroll
                            for (int k = 0; k < DIM; ++k) ci[k] = to_fixed(c[k], a.F);
                            done = canon_d2_fixed<DIM>(qi, ci, a.F, bits);
                        }
                    }
                    if (!done) bits = canon_d2_fp64<DIM>(q, c);
                    bw[g] = bits;
                    hist[g] = id;
                }
            }
            __syncwarp();
            uint64_t D[E];
            uint32_t I[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int g = lane * E + e;
                D[e] = ~0ull;
                I[e] = ~0u;
                if (g < m) {
                    const uint32_t slot = v[e] & SLOT;
                    D[e] = bw[slot];
                    I[e] = hist[slot];
                }
            }
            __syncwarp();
            if (lane == 0) st_band += (unsigned long long)m;
            KNN_CNT(12, c0);
            KNN_CNT(13, m);
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
            if (__any_sync(FULL, inv)) {
                KNN_CNT(14, 1);
                warp_bitonic<E>(D, I, lane);
            }
            uint64_t dk = 0;
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (e == (K - 1) % E) dk = D[e];
            dk = __shfl_sync(FULL, dk, (K - 1) / E);
            const float R = rcert[i];
            bool certified = isinf(R);
            if (!certified) {
                const float R2 = __fmul_rd(__fmul_rd(R, R), 1.0f - 0x1p-20f);
                certified = dk < f32_to_f64_bits_floor(R2);
            }
            KNN_PT(6);
            // not certified: the K-th value bounds the next pass's threshold
            if (!certified && lane == 0) a.seed[qsv[i]] = band_thr(vk | SLOT);
            if (certified) {
                flag = 0;
                const int64_t rowq = (int64_t)(a.sorted_rows ? qsv[i] : a.qperm[qsv[i]]) - a.row0;
                const bool rowin = rowq >= 0 && rowq < a.out_rows;  // checked in every build
                const bool rowok = KNN_GUARD(rowin, 5) && rowin;
                const int64_t row = rowq * K;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int g = lane * E + e;
                    if (g < K && rowok) {
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
    KNN_ITEM_END(Q);
}

// The scan of one join: warps take work items from the join's queue.
template <int DIM, int QM, int E, bool MEGA>
__global__ void __launch_bounds__(S2_CTA, E <= 2 ? (DIM <= 2 ? S2_MIN_CTAS_2D : S2_MIN_CTAS) : S2_MIN_CTAS_BIG)
k_scan2(const __grid_constant__ ScanArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Scan2Warp<DIM, QM, E> w(smem + warp * scan2_warp_bytes(DIM, QM, E));
    unsigned long long st_cand = 0, st_band = 0;
    const float fsc = scan2_fixed_scale(a);
    KNN_PT_DECL;
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(a.counter, 1u);
        item = __shfl_sync(FULL, item, 0);
        if (item >= a.nitems) break;
        scan2_item<DIM, QM, E, MEGA>(a, item, w, lane, fsc, st_cand, st_band KNN_CNT_ARG);
    }
    KNN_PT_FLUSH;
    scan2_flush_stats(a, st_cand, st_band, lane);
}

// The scan of several joins in one launch (batched joins): the work items of
// all of them form one queue, ordered dense first across joins (entry = job
// << 24 | item), and the joins' arguments sit in the launch's parameter space
// (indexed by job; a warp reads the arguments of the job it works on).
template <int DIM, int QM, int E, bool MEGA>
__global__ void __launch_bounds__(S2_CTA, E <= 2 ? (DIM <= 2 ? S2_MIN_CTAS_2D : S2_MIN_CTAS) : S2_MIN_CTAS_BIG)
k_scan2_multi(const __grid_constant__ MultiScanArgs p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Scan2Warp<DIM, QM, E> w(smem + warp * scan2_warp_bytes(DIM, QM, E));
    unsigned long long st_cand = 0, st_band = 0;
    int cur = -1;
    KNN_PT_DECL;
    for (;;) {
        uint32_t u = 0;
        if (lane == 0) u = atomicAdd(p.counter, 1u);
        u = __shfl_sync(FULL, u, 0);
        if (u >= p.nuitems) break;
        const uint32_t e = p.uitems[u];
        const int job = (int)(e >> 24);
        if (job != cur) {
            if (cur >= 0) scan2_flush_stats(p.jobs[cur], st_cand, st_band, lane);
            st_cand = st_band = 0;
            cur = job;
        }
        const ScanArgs &a = p.jobs[job];
        scan2_item<DIM, QM, E, MEGA>(a, e & 0xffffffu, w, lane, scan2_fixed_scale(a), st_cand, st_band KNN_CNT_ARG);
    }
    KNN_PT_FLUSH;
    if (cur >= 0) scan2_flush_stats(p.jobs[cur], st_cand, st_band, lane);
}


}  // namespace knn
