// dist32.cuh -- the FP32 filter distance of the scan (paper Alg. 1 kernel,
// distance calculations), shared by the scan kernel and the FP32-only
// ranking diagnostic, which must evaluate the identical expression.
#pragma once

namespace knn {

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

// Two candidates at once on the packed FP32 pipe (fma.rn.f32x2 and friends,
// sm_100 and later): a 64-bit register holds one value for candidate A (low
// half) and one for candidate B (high half).  Every packed instruction rounds
// each half exactly as the scalar instruction would, and the operations and
// their order are those of dist2_f32, so dA and dB are bit-identical to
// dist2_f32(q, cA) and dist2_f32(q, cB); only the instruction count halves.
__device__ __forceinline__ unsigned long long f32x2_pack(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f32x2_unpack(unsigned long long v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f32x2_sub(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f32x2_fma(unsigned long long a, unsigned long long b,
                                                        unsigned long long c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ unsigned long long f32x2_add(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// Packed sum rounded towards -inf (each half as __fadd_rd).
__device__ __forceinline__ unsigned long long f32x2_add_rd(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("add.rm.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// dist2_f32(q, cA) and dist2_f32(q, cB), with cp[k] = (cA[k], cB[k]) packed.
template <int DIM>
__device__ __forceinline__ void dist2_f32_x2(const float (&q)[DIM], const unsigned long long (&cp)[DIM], float &dA,
                                             float &dB)
{
    const unsigned long long z = 0ull;  // (+0, +0)
    if (DIM < 4) {
        unsigned long long d2 = z;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const unsigned long long df = f32x2_sub(f32x2_pack(q[k], q[k]), cp[k]);
            d2 = f32x2_fma(df, df, d2);
        }
        f32x2_unpack(d2, dA, dB);
        return;
    }
    unsigned long long e = z, o = z;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const unsigned long long df = f32x2_sub(f32x2_pack(q[k], q[k]), cp[k]);
        if (k & 1) o = f32x2_fma(df, df, o);
        else e = f32x2_fma(df, df, e);
    }
    f32x2_unpack(f32x2_add(e, o), dA, dB);
}

// dist2_f32(q0, c) and dist2_f32(q1, c) for two queries and one candidate:
// qp[k] = (q0[k], q1[k]) and cc[k] = (c[k], c[k]) packed.
template <int DIM>
__device__ __forceinline__ void dist2_f32_x2q(const unsigned long long (&qp)[DIM], const unsigned long long (&cc)[DIM],
                                              float &d0, float &d1)
{
    const unsigned long long z = 0ull;  // (+0, +0)
    if (DIM < 4) {
        unsigned long long d2 = z;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const unsigned long long df = f32x2_sub(qp[k], cc[k]);
            d2 = f32x2_fma(df, df, d2);
        }
        f32x2_unpack(d2, d0, d1);
        return;
    }
    unsigned long long e = z, o = z;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const unsigned long long df = f32x2_sub(qp[k], cc[k]);
        if (k & 1) o = f32x2_fma(df, df, o);
        else e = f32x2_fma(df, df, e);
    }
    f32x2_unpack(f32x2_add(e, o), d0, d1);
}

}  // namespace knn
