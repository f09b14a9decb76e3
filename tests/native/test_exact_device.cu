// Device check of exact.cuh against CUDA's FP64 arithmetic on the GPU:
// canonical squared distance (vs __dsub_rn/__dmul_rn/__dadd_rn in sequence)
// and the square root (vs __dsqrt_rn), on counter-generated inputs of many
// magnitude mixes.  One thread per case; every index is < N and every buffer
// holds N entries.  Prints the mismatch counts; exit status 1 on a mismatch.
#include <cstdio>
#include <cstdint>
#include "../../paper_1810_04758_b300/csrc/exact.cuh"

__device__ uint64_t mixu(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ float gen(uint64_t r, int mode)
{
    double u = (double)(r >> 11) * 0x1p-53;
    switch (mode) {
    case 0: return (float)u;
    case 1: return (float)(-log1p(-u) / 40.0);
    case 2: return (float)ldexp(u, (int)(r % 120) - 100) * ((r >> 7) & 1 ? 1.f : -1.f);
    case 3: return __uint_as_float((uint32_t)r & 0x7f7fffffu);
    default: return (float)((r >> 40) * 0x1p-24);
    }
}

__global__ void k_check(int64_t N, unsigned long long *bad)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    uint64_t r = mixu((uint64_t)i * 7919u + 17u);
    int d = 1 + (int)(r % 8);
    int mode = (int)((r >> 8) % 5);
    float a[8], b[8];
    for (int k = 0; k < d; ++k) {
        uint64_t r1 = mixu(r + 2 * k + 1), r2 = mixu(r + 2 * k + 2);
        a[k] = gen(r1, mode);
        b[k] = gen(r2, (r2 & 3) == 0 ? (int)(r2 % 5) : mode);
        if ((r2 & 15) == 1) b[k] = a[k];
    }
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = __dsub_rn((double)a[k], (double)b[k]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    if (!isfinite(s)) return;
    uint64_t ref = (uint64_t)__double_as_longlong(s);
    if (knn::canon_d2_general_rt(a, b, d) != ref) atomicAdd(&bad[0], 1ull);
    if (knn::sqrt_bits(ref) != (uint64_t)__double_as_longlong(__dsqrt_rn(s))) atomicAdd(&bad[1], 1ull);
    // sqrt over the whole normal range
    uint64_t x = (mixu(r ^ 0xabcdef) & 0x000fffffffffffffull) | ((uint64_t)(1 + (r >> 20) % 2046) << 52);
    double xd = __longlong_as_double((long long)x);
    if (knn::sqrt_bits(x) != (uint64_t)__double_as_longlong(__dsqrt_rn(xd))) atomicAdd(&bad[2], 1ull);
}

int main(int argc, char **argv)
{
    int64_t N = argc > 1 ? atoll(argv[1]) : (1 << 24);
    unsigned long long *bad;
    cudaMalloc(&bad, 3 * sizeof(unsigned long long));
    cudaMemset(bad, 0, 3 * sizeof(unsigned long long));
    k_check<<<(unsigned)((N + 255) / 256), 256>>>(N, bad);
    unsigned long long h[3] = {0, 0, 0};
    cudaError_t e = cudaMemcpy(h, bad, sizeof(h), cudaMemcpyDeviceToHost);
    printf("cases=%lld d2_bad=%llu sqrt_bad=%llu sqrt_range_bad=%llu err=%s\n", (long long)N, h[0], h[1],
           h[2], cudaGetErrorString(e));
    return (e != cudaSuccess || h[0] || h[1] || h[2]) ? 1 : 0;
}
