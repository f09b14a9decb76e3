// exact.cuh -- bit-exact canonical FP64 squared distance and correctly
// rounded square root, computed with integer and FP32 instructions.
//
// The join ranks neighbours by the canonical squared distance
//     D = fl64(...fl64(fl64(t_0) + fl64(t_1)) + ... + fl64(t_{d-1})),
//     t_k = fl64(fl64((double)a_k - (double)b_k)^2)
// (left-to-right sum, no fused multiply-add; the paper's Euclidean distance,
// Sec. 2.1, made exact) and reports sqrt(D) correctly rounded.  On B300 the
// FP64 pipe issues about 1.6 operations per clock per SM and an FP64 square
// root about 0.2, so this file reproduces every IEEE round-to-nearest-even
// step of that sequence bit for bit with 32/64-bit integer arithmetic (soft
// float) plus a few FP32 instructions, and never touches the FP64 pipe.
//
// Two evaluation paths for D:
//   * fixed-point: when every coordinate is an integer multiple of 2^-F with
//     magnitude below 2^30, each difference is an exact integer, and if the
//     integer sum of squares is below 2^53 no FP64 step of the canonical
//     sequence rounds, so D = N * 2^-2F exactly;
//   * general: decode the floats and emulate each rounding step.
// Both return the IEEE-754 bit pattern of D (always a positive normal double
// or +0 for float inputs: squares of float differences lie in [2^-298, 2^258]).
//
// The square root refines an FP32 estimate by one double-float Newton step and
// one integer Newton step, then decides the rounding exactly from the integer
// remainder M - R^2, which is small enough to be evaluated modulo 2^64.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define KNN_HD __host__ __device__ __forceinline__
#else
#include <math.h>
#include <string.h>
#define KNN_HD static inline
#endif

namespace knn {

KNN_HD int clz64(uint64_t x)
{
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

KNN_HD int ctz64(uint64_t x)
{
#ifdef __CUDA_ARCH__
    return __ffsll((long long)x) - 1;
#else
    return __builtin_ctzll(x);
#endif
}

KNN_HD uint64_t mulhi64(uint64_t a, uint64_t b)
{
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

KNN_HD uint32_t fbits(float f)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
#endif
}

KNN_HD float bitsf(uint32_t u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}

// ---------------------------------------------------------------------------
// Non-negative double as m * 2^e with m in [2^52, 2^53), or zero (m == 0).
// ---------------------------------------------------------------------------
struct Dbl {
    uint64_t m;
    int e;
};

// Round U * 2^e (U > 0) to 53 significant bits, ties to even.  When U is the
// exact value padded with a sticky bit in its least significant position (an
// odd U standing for "a little more than U - 1"), the result is still the
// correctly rounded one as long as at least two bits are dropped.
KNN_HD Dbl round53(uint64_t U, int e)
{
    int nb = 64 - clz64(U);
    if (nb <= 53) {
        Dbl r = {U << (53 - nb), e - (53 - nb)};
        return r;
    }
    int drop = nb - 53;
    uint64_t m = U >> drop;
    uint64_t rem = U & ((1ull << drop) - 1);
    uint64_t half = 1ull << (drop - 1);
    if (rem > half || (rem == half && (m & 1))) {
        ++m;
        if (m == (1ull << 53)) {
            m >>= 1;
            ++drop;
        }
    }
    Dbl r = {m, e + drop};
    return r;
}

KNN_HD uint64_t encode(Dbl x)
{
    if (!x.m) return 0;
    uint64_t be = (uint64_t)(x.e + 52 + 1023);
    return (be << 52) | (x.m & ((1ull << 52) - 1));
}

KNN_HD Dbl decode(uint64_t bits)
{
    Dbl r = {0, 0};
    if (!bits) return r;
    int be = (int)(bits >> 52);
    r.m = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    r.e = be - 1075;
    return r;
}

// |x| = M * 2^E with M < 2^24 (M = 0 for a zero).
KNN_HD void fdecode(float x, uint32_t &M, int &E)
{
    uint32_t b = fbits(x) & 0x7fffffffu;
    uint32_t ex = b >> 23, fr = b & 0x7fffffu;
    if (ex == 0) {
        M = fr;
        E = -149;
    } else {
        M = fr | 0x800000u;
        E = (int)ex - 150;
    }
}

// |fl64((double)a - (double)b)| for finite floats a, b.
KNN_HD Dbl absdiff(float a, float b)
{
    uint32_t Ma, Mb;
    int Ea, Eb;
    fdecode(a, Ma, Ea);
    fdecode(b, Mb, Eb);
    if (Mb == 0) {
        if (Ma == 0) { Dbl z = {0, 0}; return z; }
        return round53(Ma, Ea);
    }
    if (Ma == 0) return round53(Mb, Eb);
    bool add = ((fbits(a) ^ fbits(b)) >> 31) != 0;  // opposite signs: magnitudes add
    uint32_t Mh = Ma, Ml = Mb;
    int Eh = Ea, El = Eb;
    if (Ea < Eb) {
        Mh = Mb; Ml = Ma; Eh = Eb; El = Ea;
    }
    int sh = Eh - El;
    if (sh <= 38) {
        uint64_t H = (uint64_t)Mh << sh, L = Ml;
        uint64_t U = add ? H + L : (H >= L ? H - L : L - H);
        if (!U) { Dbl z = {0, 0}; return z; }
        return round53(U, El);
    }
    // The smaller operand lies far below the larger one's last bit: keep the
    // larger at bit 62, the smaller shifted down with a sticky bit.
    int s2 = sh - 38;
    uint64_t H = (uint64_t)Mh << 39;
    uint64_t L = s2 >= 32 ? 0 : ((uint64_t)Ml >> s2);
    bool sticky = s2 >= 32 ? (Ml != 0) : ((Ml & ((1u << s2) - 1)) != 0);
    uint64_t Lr = (L << 1) | (sticky ? 1u : 0u);
    uint64_t U = add ? H + Lr : H - Lr;
    return round53(U, El + s2 - 1);
}

// fl64(x^2)
KNN_HD Dbl square(Dbl x)
{
    if (!x.m) return x;
    int tz = ctz64(x.m);
    uint64_t U = x.m >> tz;
    int e = x.e + tz;
    if (U < (1ull << 32)) return round53(U * U, 2 * e);
    uint64_t hi = mulhi64(x.m, x.m), lo = x.m * x.m;
    int nbh = 64 - clz64(hi);  // 41 or 42
    int drop = nbh + 11;       // bit length - 53
    uint64_t m = (hi << (64 - drop)) | (lo >> drop);
    uint64_t rem = lo & ((1ull << drop) - 1);
    uint64_t half = 1ull << (drop - 1);
    if (rem > half || (rem == half && (m & 1))) {
        ++m;
        if (m == (1ull << 53)) {
            m >>= 1;
            ++drop;
        }
    }
    Dbl r = {m, 2 * x.e + drop};
    return r;
}

// fl64(x + y), x, y >= 0
KNN_HD Dbl add(Dbl x, Dbl y)
{
    if (!y.m) return x;
    if (!x.m) return y;
    if (x.e < y.e) {
        Dbl t = x; x = y; y = t;
    }
    int d = x.e - y.e;
    uint64_t X = x.m << 10;
    uint64_t ys = y.m << 10;
    uint64_t Y;
    bool sticky;
    if (d >= 63) {
        Y = 0;
        sticky = true;
    } else {
        Y = ys >> d;
        sticky = d > 0 && (ys & ((1ull << d) - 1)) != 0;
    }
    return round53(X + (Y | (sticky ? 1u : 0u)), x.e - 10);
}

// Canonical squared distance of two float vectors, general path.
template <int DIM>
KNN_HD uint64_t canon_d2_general(const float *a, const float *b)
{
    Dbl acc = square(absdiff(a[0], b[0]));
#pragma unroll
    for (int k = 1; k < DIM; ++k) acc = add(acc, square(absdiff(a[k], b[k])));
    return encode(acc);
}

KNN_HD uint64_t canon_d2_general_rt(const float *a, const float *b, int d)
{
    Dbl acc = square(absdiff(a[0], b[0]));
    for (int k = 1; k < d; ++k) acc = add(acc, square(absdiff(a[k], b[k])));
    return encode(acc);
}

#ifdef __CUDACC__
// Canonical squared distance on the FP64 pipe: the very IEEE operations of
// the definition (round to nearest, never fused).  Used on the device for
// inputs off a common dyadic grid, where the soft-float emulation above is
// slower than the FP64 unit's ~1.6 operations per clock per SM.
template <int DIM>
__device__ __forceinline__ uint64_t canon_d2_fp64(const float *a, const float *b)
{
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const double t = __dsub_rn((double)a[k], (double)b[k]);
        acc = __dadd_rn(acc, __dmul_rn(t, t));
    }
    return (uint64_t)__double_as_longlong(acc);
}
#endif

// Integer N * 2^e as a double bit pattern (N < 2^53: exact).
KNN_HD uint64_t encode_int(uint64_t N, int e)
{
    if (!N) return 0;
    int nb = 64 - clz64(N);
    Dbl r = {N << (53 - nb), e - (53 - nb)};
    return encode(r);
}

// Fixed-point coordinate: x = X * 2^-F exactly (the caller has checked that
// every coordinate admits this with |X| < 2^30).
KNN_HD int32_t to_fixed(float x, int F)
{
    uint32_t M;
    int E;
    fdecode(x, M, E);
    int s = E + F;
    int32_t X = (int32_t)(s >= 0 ? (M << s) : (M >> -s));
    return (fbits(x) >> 31) ? -X : X;
}

// Fixed-point path: true and D's bits when no canonical step rounds.
template <int DIM>
KNN_HD bool canon_d2_fixed(const int32_t *A, const int32_t *B, int F, uint64_t &bits)
{
    uint64_t N = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        int64_t df = (int64_t)A[k] - (int64_t)B[k];
        uint64_t ad = (uint64_t)(df < 0 ? -df : df);
        if (ad >= (1ull << 26)) return false;
        N += ad * ad;
    }
    if (N >= (1ull << 53)) return false;
    bits = encode_int(N, -2 * F);
    return true;
}

#ifdef __CUDACC__
// The same N from FP32 differences, for q and c on the common grid 2^-F:
// q - c is exact in FP32 whenever |Xq - Xc| < 2^24 (the exact difference is
// then representable), and (q - c) * 2^F (sc = 2^F) is that integer exactly.
// A rounded difference has |x| >= 2^24, which the test catches: false, and
// the caller takes the integer path above.
template <int DIM>
__device__ __forceinline__ bool canon_d2_fixed_f32(const float (&q)[DIM], const float (&c)[DIM], float sc, int F,
                                                   uint64_t &bits)
{
    uint64_t N = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const float x = __fmul_rn(__fsub_rn(q[k], c[k]), sc);
        if (!(fabsf(x) < 16777216.0f)) return false;
        const int64_t X = (int64_t)__float2int_rz(x);
        N += (uint64_t)(X * X);
    }
    bits = encode_int(N, -2 * F);  // N < 8 * 2^48 < 2^53: exact
    return true;
}
#endif

KNN_HD bool canon_d2_fixed_rt(const int32_t *A, const int32_t *B, int d, int F, uint64_t &bits)
{
    uint64_t N = 0;
    for (int k = 0; k < d; ++k) {
        int64_t df = (int64_t)A[k] - (int64_t)B[k];
        uint64_t ad = (uint64_t)(df < 0 ? -df : df);
        if (ad >= (1ull << 26)) return false;
        N += ad * ad;
    }
    if (N >= (1ull << 53)) return false;
    bits = encode_int(N, -2 * F);
    return true;
}

// ---------------------------------------------------------------------------
// Correctly rounded square root of a non-negative normal double (bit pattern).
// ---------------------------------------------------------------------------
KNN_HD float approx_rsqrt(float x)
{
#ifdef __CUDA_ARCH__
    return rsqrtf(x);
#else
    return 1.0f / sqrtf(x);
#endif
}

KNN_HD float sqrt_rn_f32(float x)
{
#ifdef __CUDA_ARCH__
    return __fsqrt_rn(x);
#else
    return sqrtf(x);
#endif
}

KNN_HD int f2i_rn(float x)
{
#ifdef __CUDA_ARCH__
    return __float2int_rn(x);
#else
    return (int)nearbyintf(x);
#endif
}

KNN_HD float i2f_rn(int64_t v)
{
#ifdef __CUDA_ARCH__
    return __ll2float_rn((long long)v);
#else
    return (float)v;
#endif
}

KNN_HD uint64_t sqrt_bits(uint64_t Dbits)
{
    if (!Dbits) return 0;
    int be = (int)(Dbits >> 52);
    uint64_t m = (Dbits & ((1ull << 52) - 1)) | (1ull << 52);
    int E = be - 1075;  // D = m * 2^E
    if (E & 1) {
        m <<= 1;
        E -= 1;
    }
    // M = m * 2^52 in [2^104, 2^106); the answer is R = round(sqrt(M)),
    // sqrt(D) = R * 2^((E - 52) / 2).  Work on x = m * 2^-22 in [2^30, 2^32),
    // sqrt(M) = sqrt(x) * 2^37.
    uint32_t mh = (uint32_t)(m >> 22);
    float xh = (float)mh;                          // 24-bit rounding of x, in [2^30, 2^32]
    uint32_t xb = fbits(xh);                       // xh as an integer, from its bits
    uint64_t xhi = (uint64_t)((xb & 0x7fffffu) | 0x800000u) << ((int)(xb >> 23) - 150);
    int64_t rl = (int64_t)m - (int64_t)(xhi << 22);
    float xl = i2f_rn(rl) * 0x1p-22f;              // x - xh, to 24 bits
    float r0 = approx_rsqrt(xh);
    float s0 = sqrt_rn_f32(xh);
    float e = fmaf(-s0, s0, xh) + xl;              // fmaf term is exact
    float c1 = e * (0.5f * r0);
    // S1 = (s0 + c1) * 2^37: s0 * 2^37 is an integer below 2^53.
    uint32_t sb = fbits(s0);
    uint64_t S1 = (uint64_t)((sb & 0x7fffffu) | 0x800000u) << ((int)(sb >> 23) - 150 + 37);
    S1 = (uint64_t)((int64_t)S1 + (int64_t)f2i_rn(c1 * 0x1p37f));
    uint64_t Mlo = m << 52;                        // M mod 2^64
    int64_t delta = (int64_t)(Mlo - S1 * S1);      // |M - S1^2| < 2^61
    float q = i2f_rn(delta) * (r0 * 0x1p-38f);     // delta / (2 S1)
    int64_t R = (int64_t)S1 + (int64_t)f2i_rn(q);  // within 0.51 of sqrt(M)
    int64_t d2 = (int64_t)(Mlo - (uint64_t)R * (uint64_t)R);
    if (d2 > R) ++R;                               // R = round(sqrt(M)) iff -R < M - R^2 <= R
    else if (d2 <= -R) --R;
    return encode(round53((uint64_t)R, (E - 52) / 2));
}

}  // namespace knn
