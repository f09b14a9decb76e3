// Host check of the exact-arithmetic header against the CPU's IEEE-754
// double arithmetic (x86-64 SSE2, round to nearest even, built with
// -ffp-contract=off so a*b+c is never fused).
//
// Checks: the canonical squared distance on random float pairs of many
// magnitude mixes (general path) and on dyadic-grid inputs (fixed-point
// path); the square root on random doubles, perfect squares and values next
// to rounding midpoints.  Prints counts and exits non-zero on any mismatch.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <random>
#include "../../paper_1810_04758_b300/csrc/exact.cuh"

static uint64_t dbits(double x) { uint64_t u; memcpy(&u, &x, 8); return u; }
static double bitsd(uint64_t u) { double x; memcpy(&x, &u, 8); return x; }

static double canon_ref(const float* a, const float* b, int d)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) { double t = (double)a[k] - (double)b[k]; double sq = t * t; s = s + sq; }
    return s;
}

int main(int argc, char** argv)
{
    long iters = argc > 1 ? atol(argv[1]) : 2000000;
    std::mt19937_64 rng(12345);
    long bad = 0, checked = 0;
    auto rfloat = [&](int mode) -> float {
        uint64_t r = rng();
        double u = (r >> 11) * 0x1p-53;
        switch (mode) {
        case 0: return (float)u;                                   // [0,1)
        case 1: return (float)(-std::log1p(-u) / 40.0);            // expo(40)
        case 2: return (float)std::ldexp(u, (int)(rng() % 120) - 100) * ((rng() & 1) ? 1 : -1);  // wide range
        case 3: { uint32_t b = (uint32_t)rng(); b &= 0x7f7fffffu; float f; memcpy(&f, &b, 4); return f; } // any finite >=0 incl. subnormal
        case 4: return (float)((r >> 40) * 0x1p-24);               // dyadic grid
        default: return (float)(u * 1e6 - 5e5);
        }
    };
    for (long it = 0; it < iters; ++it) {
        int d = 1 + (int)(rng() % 8);
        int mode = (int)(rng() % 6);
        float a[8], b[8];
        for (int k = 0; k < d; ++k) {
            a[k] = rfloat(mode);
            int mb = (rng() % 4 == 0) ? (int)(rng() % 6) : mode;
            b[k] = rfloat(mb);
            if (rng() % 8 == 0) b[k] = a[k];
            if (rng() % 16 == 0) b[k] = std::nextafter(a[k], 2.0f);
        }
        double ref = canon_ref(a, b, d);
        if (!std::isfinite(ref)) continue;
        uint64_t got = knn::canon_d2_general_rt(a, b, d);
        ++checked;
        if (got != dbits(ref)) {
            if (bad < 10) printf("D mismatch d=%d mode=%d ref=%.17g got=%.17g\n", d, mode, ref, bitsd(got));
            ++bad;
        }
        uint64_t s = knn::sqrt_bits(dbits(ref));
        if (s != dbits(std::sqrt(ref))) {
            if (bad < 10) printf("sqrt mismatch D=%.17g ref=%.17g got=%.17g\n", ref, std::sqrt(ref), bitsd(s));
            ++bad;
        }
    }
    // fixed-point path on the 2^-24 grid (F = 24)
    long fixed_used = 0;
    for (long it = 0; it < iters / 4; ++it) {
        int d = 1 + (int)(rng() % 8);
        float a[8], b[8];
        int32_t A[8], B[8];
        for (int k = 0; k < d; ++k) {
            a[k] = rfloat(4); b[k] = rfloat(4);
            A[k] = knn::to_fixed(a[k], 24); B[k] = knn::to_fixed(b[k], 24);
            if ((double)A[k] != std::ldexp((double)a[k], 24)) { printf("to_fixed wrong\n"); ++bad; }
        }
        uint64_t bits;
        if (knn::canon_d2_fixed_rt(A, B, d, 24, bits)) {
            ++fixed_used;
            if (bits != dbits(canon_ref(a, b, d))) { if (bad < 10) printf("fixed mismatch\n"); ++bad; }
        }
    }
    // square roots: random doubles over the whole normal range, perfect
    // squares, and neighbours of squares and of midpoints
    long sq_checked = 0;
    for (long it = 0; it < iters; ++it) {
        uint64_t r = rng();
        double x;
        int kind = it % 4;
        if (kind == 0) x = bitsd((r & 0x000fffffffffffffull) | ((uint64_t)(1 + rng() % 2046) << 52));
        else if (kind == 1) { double y = bitsd((r & 0x000fffffffffffffull) | ((uint64_t)(600 + rng() % 800) << 52)); x = y * y; }
        else if (kind == 2) { double y = bitsd((r & 0x000fffffffffffffull) | ((uint64_t)(600 + rng() % 800) << 52));
                              double yn = std::nextafter(y, 1e300); double mid = y + (yn - y) / 2; x = mid * mid;
                              x = bitsd(dbits(x) + (int64_t)(rng() % 5) - 2); }
        else { uint64_t N = (r >> 11); x = std::ldexp((double)N, -48); }
        if (!(x > 0) || !std::isfinite(x)) continue;
        ++sq_checked;
        uint64_t s = knn::sqrt_bits(dbits(x));
        if (s != dbits(std::sqrt(x))) { if (bad < 20) printf("sqrt mismatch x=%.17g\n", x); ++bad; }
    }
    printf("checked D=%ld fixed=%ld sqrt=%ld bad=%ld\n", checked, fixed_used, sq_checked, bad);
    return bad ? 1 : 0;
}
