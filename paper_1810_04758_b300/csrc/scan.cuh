// scan.cuh -- the per-query neighbour-cell scan with top-K selection
// (paper Alg. 1, GPUJoinKernel; Sec. 4.7 for several threads per query),
// made exact and self-certifying.
//
// One work item = up to WARPS queries that share a level-l grid cell (a slice
// of one group of the density-ordered queue).  The CTA
//   a7  looks up the 3^d neighbouring cells of that cell in the level's hash
//       map and prefix-sums their sizes;
//   a8  stages the candidate coordinates chunk by chunk in shared memory,
//       where every warp (one query each, 32 lanes over the candidates)
//       evaluates FP32 squared distances and appends those at or below its
//       acceptance threshold to a per-query buffer; when the buffer fills, a
//       warp radix select finds the current K-th value T and the threshold
//       becomes T * (1 + 2^-15) + 2^-120, so every candidate that can still
//       rank in the top K is kept;
//   a9  selects T32, the K-th FP32 value, keeps the band d2_32 <= T32 *
//       (1 + 2^-15) + 2^-120 (a superset of the exact top K: FP32 squared
//       distances are within (d + 2) 2^-24 relative of the exact ones), scores
//       it with the bit-exact canonical FP64 distance (exact.cuh), ranks it by
//       (D, original id) and certifies the K-th: D_K < R^2, R the distance
//       from the query to the faces of the scanned box (rounded down), or the
//       box covers every cell;
//   a10 flags queries that are not certified (they go to the next level:
//       a ring of cells twice as wide);
//   a11 writes certified rows: original ids and the bit patterns of D (their
//       correctly rounded square roots are taken by k_sqrt_rows).
// A query whose band overflows its buffer (massive ties) is redone in an
// exact round in which every candidate carries its exact (D, id) key.
#pragma once
#include "common.cuh"

namespace knn {

constexpr int SCAN_WARPS = 8;
constexpr int SCAN_CTA = SCAN_WARPS * 32;

// Cell table of one grid level: a dense table (small grids) or the hash map.
struct LevelRef {
    const uint4 *hslot;  // hash map slots (cell key -> run), or null
    const uint2 *dense;  // dense table (cell index -> run), or null
    uint32_t hmask;      // hash map capacity - 1
    uint32_t pad;
};

struct ScanArgs {
    const float *xsort;        // [n][pad(d)] coordinates in key order (pad = 2, 4 or 8)
    const uint32_t *perm;      // key order -> original id
    const uint64_t *keys;      // sorted Morton keys
    const uint32_t *active;    // active list (sorted positions)
    const uint2 *items;        // (first active index, count | level << 16)
    uint32_t nitems;
    uint32_t *counter;         // work-queue head
    const LevelRef *levels;    // [MAX_LEVELS] cell tables of the grid levels (device memory)
    uint32_t *fail;            // [n] per sorted position: 0 certified, 1 not, 2 overflow
    float *seed;               // [n] per sorted position: FP32-filter threshold carried to the next pass
    int32_t *out_ids;          // [n][K]
    double *out_dist;          // [n][K]
    unsigned long long *stats; // [0] candidates, [1] overflow rounds, [2] band entries
    int64_t n;
    int K;
    int bits;
    int cmax0[MAX_DIM];
    float lo[MAX_DIM];
    float w0;
    int fixed_ok, F;
    int B;                     // buffer entries per query (power of two, >= max(128, 2K))
    // queries: their own sorted arrays (the data arrays above for a self-join)
    const float *qxsort;       // query coordinates in query-key order, padded rows
    const uint64_t *qkeys;     // sorted query keys on the data grid
    const uint32_t *qperm;     // query key order -> original query row
    int self;                  // 1: self-join (a query's own point is not its neighbour)
    float rcap;                // > 0: certificate radius capped at this (the paper's policy)
    int64_t row0;              // first output row held by out_ids/out_dist (chunked output)
    int sorted_rows;           // 1: output rows by sorted query position (cost-balanced shards)
    int64_t out_rows;          // output rows held (bounds of the checked build)
    int64_t nq;                // queries (sorted query positions < nq)
    int64_t nactive;           // entries of `active`
    int CH;                    // staged candidates per chunk
    int noff;                  // 3^d
};

// Arguments of one scan launch over several joins (k_scan2_multi): their
// work items in one queue, entry = job << 24 | item, and each join's
// arguments, in the launch's parameter space.
constexpr int S2_MULTI_JOBS = 64;
struct MultiScanArgs {
    uint32_t *counter;         // queue head
    const uint32_t *uitems;    // [nuitems] queue entries
    uint32_t nuitems;
    int njobs;
    ScanArgs jobs[S2_MULTI_JOBS];
};

__device__ __forceinline__ float band_thr(uint32_t tbits)
{
    float t = __uint_as_float(tbits);
    return fmaf(t, 0x1p-15f, t) + 0x1p-120f;
}

// K-th smallest (1-based k, 1 <= k <= cnt) of non-negative float bit patterns.
static __device__ uint32_t warp_select(const uint32_t *keys, int cnt, int k, uint32_t *hist, int lane)
{
    uint32_t prefix = 0, mask = 0;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int i = lane; i < 256; i += 32) hist[i] = 0;
        __syncwarp();
        for (int i = lane; i < cnt; i += 32) {
            uint32_t v = keys[i];
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
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (digit == 0 && below == 0 && run + h[j] >= (uint32_t)k) {
                    digit = lane * 8 + j + 1;  // +1 marks "found"
                    below = run;
                }
                run += h[j];
            }
            digit -= 1;
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

// Keep entries with key <= thr (in place, any order); returns the new count.
static __device__ int warp_compact(uint32_t *key, uint32_t *idx, int cnt, uint32_t thr_bits, int lane)
{
    int out = 0;
    for (int base = 0; base < cnt; base += 32) {
        int i = base + lane;
        bool v = i < cnt;
        uint32_t k = v ? key[i] : 0, x = v ? idx[i] : 0;
        bool keep = v && k <= thr_bits;
        uint32_t bal = __ballot_sync(FULL, keep);
        __syncwarp();
        if (keep) {
            int p = out + __popc(bal & lanemask_lt());
            key[p] = k;
            idx[p] = x;
        }
        out += __popc(bal);
        __syncwarp();
    }
    return out;
}

template <int DIM>
__device__ __forceinline__ uint64_t exact_d2(const float *q, const int32_t *qi, const ScanArgs &a,
                                             uint32_t s)
{
    float c[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) c[k] = a.xsort[(int64_t)s * pad_dim(DIM) + k];
    if (a.fixed_ok) {
        int32_t ci[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) ci[k] = to_fixed(c[k], a.F);
        uint64_t bits;
        if (canon_d2_fixed<DIM>(qi, ci, a.F, bits)) return bits;
    }
    return canon_d2_fp64<DIM>(q, c);
}

__device__ __forceinline__ bool key_less(uint64_t da, uint32_t ia, uint64_t db, uint32_t ib)
{
    return da < db || (da == db && ia < ib);
}

template <int DIM>
__global__ void __launch_bounds__(SCAN_CTA) k_scan(ScanArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = a.K, B = a.B, CH = a.CH, NOFF = a.noff;

    // shared memory layout
    uint2 *nb_range = (uint2 *)smem;                                // [NOFF]
    uint32_t *nb_cum = (uint32_t *)(nb_range + NOFF);               // [NOFF + 1]
    float *cx = (float *)(nb_cum + ((NOFF + 1 + 3) & ~3));          // [DIM][CH]
    uint32_t *cs = (uint32_t *)(cx + DIM * CH);                     // [CH]
    uint32_t *bkey = cs + CH;                                       // [WARPS][B]
    uint32_t *bidx = bkey + SCAN_WARPS * B;                         // [WARPS][B]
    uint32_t *hist = bidx + SCAN_WARPS * B;                         // [WARPS][256]
    uint64_t *xkey = (uint64_t *)(hist + SCAN_WARPS * 256);         // [WARPS][B] exact keys
    uint32_t *xid = (uint32_t *)(xkey + SCAN_WARPS * B);            // [WARPS][B] original ids
    uint32_t *xs_ = xid + SCAN_WARPS * B;                           // [WARPS][B] sorted idx

    __shared__ int s_item;
    __shared__ int s_cell[MAX_DIM];
    __shared__ int s_exact;
    __shared__ uint32_t s_scan[32];
    __shared__ uint64_t s_dk[SCAN_WARPS];

    uint32_t *wkey = bkey + warp * B, *widx = bidx + warp * B, *whist = hist + warp * 256;
    uint64_t *wxk = xkey + warp * B;
    uint32_t *wxi = xid + warp * B, *wxs = xs_ + warp * B;

    unsigned long long st_cand = 0, st_ovf = 0, st_band = 0;

    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int item = s_item;
        if ((uint32_t)item >= a.nitems) break;
        const uint2 it = a.items[item];
        const int level = (int)(it.y >> 16);
        const int shift = DIM * level;
        const int nbits = a.bits - level;
        int cmaxL[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) cmaxL[k] = a.cmax0[k] >> level;
        const bool has_q = (uint32_t)warp < (it.y & 0xffffu);
        const uint32_t qa = it.x + warp;
        const uint32_t qs = has_q ? a.active[qa] : 0u;
        const uint32_t qself = a.self ? qs : 0xffffffffu;  // data position excluded

        if (tid == 0) {
            int c[MAX_DIM];
            morton_decode(a.qkeys[a.active[it.x]] >> shift, DIM, nbits, c);
#pragma unroll
            for (int k = 0; k < DIM; ++k) s_cell[k] = c[k];
            s_exact = 0;
        }
        __syncthreads();

        // a7: neighbour cells
        for (int t = tid; t < NOFF; t += SCAN_CTA) {
            int nb[DIM];
            int r = t;
            bool ok = true;
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                nb[k] = s_cell[k] + (r % 3) - 1;
                r /= 3;
                ok = ok && nb[k] >= 0 && nb[k] <= cmaxL[k];
            }
            uint2 rg = make_uint2(0, 0);
            if (ok) {
                const LevelRef lr = a.levels[level];
                if (const uint2 *dt = lr.dense) {
                    uint32_t idx = 0, st = 1;
#pragma unroll
                    for (int k = 0; k < DIM; ++k) {
                        idx += (uint32_t)nb[k] * st;
                        st *= (uint32_t)cmaxL[k] + 1u;
                    }
                    rg = __ldg(&dt[idx]);
                } else {
                    rg = hash_lookup(lr.hslot, lr.hmask, morton_encode(nb, DIM, nbits));
                }
            }
            nb_range[t] = rg;
        }
        __syncthreads();
        {
            uint32_t carry = 0;
            for (int base = 0; base < NOFF; base += SCAN_CTA) {
                int t = base + tid;
                uint32_t len = t < NOFF ? nb_range[t].y - nb_range[t].x : 0u;
                uint32_t total;
                uint32_t ex = block_exclusive_scan(len, total, s_scan);
                if (t < NOFF) nb_cum[t] = carry + ex;
                carry += total;
            }
            if (tid == 0) nb_cum[NOFF] = carry;
            __syncthreads();
        }
        const uint32_t C = nb_cum[NOFF];

        // query coordinates
        float q[DIM];
        int32_t qi[DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            q[k] = a.qxsort[(int64_t)qs * pad_dim(DIM) + k];
            qi[k] = a.fixed_ok ? to_fixed(q[k], a.F) : 0;
        }

        // ---------------------------------------------------------------
        // Round 0: FP32 scan with threshold buffer.  Round 1 (only if some
        // warp overflowed): exact keys for the overflowed queries.
        // ---------------------------------------------------------------
        bool need_exact = false;
        int cnt = 0;
        float thr = __int_as_float(0x7f800000);
        uint64_t thrD = ~0ull;
        uint32_t thrI = ~0u;
        for (int round = 0; round < 2; ++round) {
            const bool exact_round = round == 1;
            if (exact_round) {
                if (tid == 0) s_exact = 0;
                __syncthreads();
                if (lane == 0 && has_q && need_exact) atomicOr(&s_exact, 1);
                __syncthreads();
                if (!s_exact) break;
                cnt = 0;
                thrD = ~0ull;
                thrI = ~0u;
            }
            const bool active_w = has_q && (exact_round ? need_exact : true);
            bool ovf = false;
            for (uint32_t c0 = 0; c0 < C; c0 += CH) {
                const int clen = (int)min((uint32_t)CH, C - c0);
                for (int t = tid; t < clen; t += SCAN_CTA) {
                    uint32_t g = c0 + t;
                    int lo = 0, hi = NOFF;  // last slot with nb_cum[slot] <= g
                    while (hi - lo > 1) {
                        int mid = (lo + hi) >> 1;
                        if (nb_cum[mid] <= g) lo = mid; else hi = mid;
                    }
                    uint32_t s = nb_range[lo].x + (g - nb_cum[lo]);
                    cs[t] = s;
#pragma unroll
                    for (int k = 0; k < DIM; ++k) cx[k * CH + t] = a.xsort[(int64_t)s * pad_dim(DIM) + k];
                }
                __syncthreads();
                if (active_w && !ovf) {
                    for (int base = 0; base < clen; base += 32) {
                        const int t = base + lane;
                        bool valid = t < clen;
                        uint32_t s = valid ? cs[t] : 0u;
                        valid = valid && s != qself && KNN_GUARD(s < a.n, 8);
                        if (!exact_round) {
                            float d2 = 0.0f;
                            if (valid) {
#pragma unroll
                                for (int k = 0; k < DIM; ++k) {
                                    float df = q[k] - cx[k * CH + t];
                                    d2 = fmaf(df, df, d2);
                                }
                                ++st_cand;
                            }
                            bool acc = valid && d2 <= thr;
                            uint32_t bal = __ballot_sync(FULL, acc);
                            int nnew = __popc(bal);
                            if (cnt + nnew > B) {
                                uint32_t T = warp_select(wkey, cnt, K, whist, lane);
                                thr = band_thr(T);
                                cnt = warp_compact(wkey, widx, cnt, __float_as_uint(thr), lane);
                                acc = valid && d2 <= thr;
                                bal = __ballot_sync(FULL, acc);
                                nnew = __popc(bal);
                                if (cnt + nnew > B) ovf = true;
                            }
                            if (!ovf) {
                                if (acc) {
                                    int p = cnt + __popc(bal & lanemask_lt());
                                    wkey[p] = __float_as_uint(d2);
                                    widx[p] = s;
                                }
                                cnt += nnew;
                            }
                        } else {
                            uint64_t D = ~0ull;
                            uint32_t id = ~0u;
                            if (valid) {
                                float c[DIM];
#pragma unroll
                                for (int k = 0; k < DIM; ++k) c[k] = cx[k * CH + t];
                                D = canon_d2_fp64<DIM>(q, c);
                                id = a.perm[s];
                            }
                            bool acc = valid && key_less(D, id, thrD, thrI);
                            uint32_t bal = __ballot_sync(FULL, acc);
                            int nnew = __popc(bal);
                            if (cnt + nnew > B) {
                                // keep the K smallest exact keys (unique: ids differ)
                                uint64_t kd[16];
                                uint32_t ki[16], kx[16], kr[16];
                                int mine = 0;
                                for (int i = lane; i < cnt; i += 32, ++mine) {
                                    kd[mine] = wxk[i];
                                    ki[mine] = wxi[i];
                                    kx[mine] = wxs[i];
                                    uint32_t r = 0;
                                    for (int j = 0; j < cnt; ++j) r += key_less(wxk[j], wxi[j], kd[mine], ki[mine]);
                                    kr[mine] = r;
                                }
                                __syncwarp();
                                for (int u = 0; u < mine; ++u)
                                    if (kr[u] < (uint32_t)K) {
                                        wxk[kr[u]] = kd[u];
                                        wxi[kr[u]] = ki[u];
                                        wxs[kr[u]] = kx[u];
                                    }
                                __syncwarp();
                                cnt = K;
                                thrD = wxk[K - 1];
                                thrI = wxi[K - 1];
                                acc = valid && key_less(D, id, thrD, thrI);
                                bal = __ballot_sync(FULL, acc);
                                nnew = __popc(bal);
                            }
                            if (acc) {
                                int p = cnt + __popc(bal & lanemask_lt());
                                wxk[p] = D;
                                wxi[p] = id;
                                wxs[p] = s;
                            }
                            cnt += nnew;
                        }
                        __syncwarp();
                        if (ovf) break;
                    }
                }
                __syncthreads();
            }

            if (!active_w) continue;
            if (!exact_round && ovf) {
                need_exact = true;
                if (lane == 0) ++st_ovf;
                continue;
            }

            // a9: band and exact keys (round 0), or the exact top K (round 1)
            int m = 0;
            if (!exact_round) {
                if (cnt >= K) {
                    uint32_t T = warp_select(wkey, cnt, K, whist, lane);
                    m = warp_compact(wkey, widx, cnt, __float_as_uint(band_thr(T)), lane);
                    if (m > B) m = B;  // cannot happen: m <= cnt <= B
                    for (int i = lane; i < m; i += 32) {
                        uint32_t s = widx[i];
                        wxk[i] = exact_d2<DIM>(q, qi, a, s);
                        wxi[i] = a.perm[s];
                        wxs[i] = s;
                    }
                    if (lane == 0) st_band += (unsigned long long)m;
                    __syncwarp();
                }
            } else {
                m = cnt;
            }
            // rank by (D, id); the K-th decides the certificate
            uint64_t rd[16];
            uint32_t rid[16], rr[16];
            int mine = 0;
            if (m >= K) {
                for (int i = lane; i < m; i += 32, ++mine) {
                    rd[mine] = wxk[i];
                    rid[mine] = wxi[i];
                    uint32_t r = 0;
                    for (int j = 0; j < m; ++j) r += key_less(wxk[j], wxi[j], rd[mine], rid[mine]);
                    rr[mine] = r;
                    if (r == (uint32_t)(K - 1)) s_dk[warp] = rd[mine];
                }
            }
            __syncwarp();
            bool certified = false;
            float R = __int_as_float(0x7f800000);
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                int cL = s_cell[k];
                if (cL >= 2) {
                    float f = face_of((cL - 1) << level, a.lo[k], a.w0);
                    R = fminf(R, __fsub_rd(q[k], f));
                }
                if (cL + 1 < cmaxL[k]) {
                    float f = face_of((cL + 2) << level, a.lo[k], a.w0);
                    R = fminf(R, __fsub_rd(f, q[k]));
                }
            }
            if (a.rcap > 0.0f) R = fminf(R, a.rcap);  // the paper's policy: K within eps
            if (m >= K) {
                if (isinf(R)) {
                    certified = true;
                } else {
                    float R2 = __fmul_rd(__fmul_rd(R, R), 1.0f - 0x1p-20f);
                    certified = s_dk[warp] < f32_to_f64_bits_floor(R2);
                }
            }
            if (certified) {
                const int64_t rowq = (int64_t)(a.sorted_rows ? qs : a.qperm[qs]) - a.row0;
                const bool rowin = rowq >= 0 && rowq < a.out_rows;  // checked in every build
                const bool rowok = KNN_GUARD(rowin, 9) && rowin;
                const int64_t row = rowq * K;
                for (int u = 0; u < mine; ++u)
                    if (rr[u] < (uint32_t)K && rowok) {
                        a.out_ids[row + rr[u]] = (int32_t)rid[u];
                        a.out_dist[row + rr[u]] = __longlong_as_double((long long)rd[u]);  // D; k_sqrt_rows converts
                    }
            }
            if (lane == 0) a.fail[qs] = certified ? 0u : 1u;
            if (exact_round || true) need_exact = exact_round ? false : need_exact;
        }
        __syncthreads();
    }
    // statistics
    for (int o = 16; o; o >>= 1) st_cand += __shfl_xor_sync(FULL, st_cand, o);
    if (lane == 0) {
        atomicAdd(&a.stats[0], st_cand);
        if (st_ovf) atomicAdd(&a.stats[1], st_ovf);
        if (st_band) atomicAdd(&a.stats[2], st_band);
    }
}

}  // namespace knn
