// Arithmetic throughput of one GPU: the denominators of the FP32 and FP64
// roofline fractions of the scan kernel (the FP32 distance filter and the
// exact FP64 re-score budget).
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o alu_peaks alu_peaks.cu && ./alu_peaks
//
// Each thread runs 8 independent dependency chains of one operation for ITERS
// iterations; the grid is SMs x 8 CTAs x 256 threads.  Every thread writes one
// word of its chains' sum, so the work cannot be removed.  Three timed
// repetitions (CUDA events), the last reported.
#include <cstdio>
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { \
    std::fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_)); return 1; } } while (0)

constexpr int ITERS = 4096;
constexpr int CHAINS = 8;

__global__ void k_ffma(float *out, float a, float b) {
  float x[CHAINS];
  for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x + c;
  for (int i = 0; i < ITERS; ++i)
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = __fmaf_rn(x[c], a, b);
  float s = 0;
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dfma(double *out, double a, double b) {
  double x[CHAINS];
  for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x + c;
  for (int i = 0; i < ITERS; ++i)
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = __fma_rn(x[c], a, b);
  double s = 0;
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dadd(double *out, double a, double b) {
  double x[CHAINS];
  for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x + c;
  for (int i = 0; i < ITERS; ++i)
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = __dadd_rn(x[c], a);
  double s = b;
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dmul(double *out, double a, double b) {
  double x[CHAINS];
  for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x + c + 1;
  for (int i = 0; i < ITERS; ++i)
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = __dmul_rn(x[c], a);
  double s = b;
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dsqrt(double *out, double a, double b) {
  double x[CHAINS];
  for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x + c + 2;
  for (int i = 0; i < ITERS / 16; ++i)
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = __dsqrt_rn(x[c]) + a;
  double s = b;
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_fsqrt(float *out, float a, float b) {
  float x[CHAINS];
  for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x + c + 2;
  for (int i = 0; i < ITERS; ++i)
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = __fsqrt_rn(x[c]) + a;
  float s = b;
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_cvt(float *out, float a, float b) {
  float x[CHAINS];
  for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x + c;
  for (int i = 0; i < ITERS; ++i)
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = (float)__fma_rn((double)x[c], (double)a, (double)b);
  float s = 0;
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_umulhi(unsigned long long *out, unsigned long long a, unsigned long long b) {
  unsigned long long x[CHAINS];
  for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x * 0x9e3779b97f4a7c15ull + c;
  for (int i = 0; i < ITERS; ++i)
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = __umul64hi(x[c], a) ^ b;
  unsigned long long s = 0;
  for (int c = 0; c < CHAINS; ++c) s ^= x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class F>
static int time_it(const char *name, double ops_per_thread, double flops_per_op, int blocks,
                   int threads, double clk_ghz, int sms, F launch) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float ms = 0;
  for (int rep = 0; rep < 3; ++rep) {
    CK(cudaEventRecord(e0));
    launch();
    CK(cudaGetLastError());
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
  }
  const double ops = ops_per_thread * blocks * threads;
  const double gops = ops / (ms * 1e-3) / 1e9;
  std::printf("| %s | %.0f | %s | %.2f |\n", name, gops,
              flops_per_op > 0 ? std::to_string(gops * flops_per_op / 1e3).substr(0, 6).c_str() : "-",
              gops / (clk_ghz * sms));
  CK(cudaEventDestroy(e0));
  CK(cudaEventDestroy(e1));
  return 0;
}


int main() {
  int dev = 0, sms = 0, clk_khz = 0;
  CK(cudaSetDevice(dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, dev));
  const int threads = 256, blocks = sms * 8;
  const double ghz = clk_khz / 1e6;
  void *buf = nullptr;
  CK(cudaMalloc(&buf, (size_t)blocks * threads * 8));
  std::printf("# %s: %d SMs, %.0f MHz (device attribute)\n\n", prop.name, sms, ghz * 1e3);
  std::printf("| op | Gop/s | TFLOP/s | ops/clk/SM |\n|---|---|---|---|\n");
  const double n = (double)ITERS * CHAINS;
  if (time_it("FP32 FFMA", n, 2, blocks, threads, ghz, sms,
              [&] { k_ffma<<<blocks, threads>>>((float *)buf, 0.999f, 1e-3f); })) return 1;
  if (time_it("FP64 DFMA", n, 2, blocks, threads, ghz, sms,
              [&] { k_dfma<<<blocks, threads>>>((double *)buf, 0.999, 1e-3); })) return 1;
  if (time_it("FP64 DADD (__dadd_rn)", n, 1, blocks, threads, ghz, sms,
              [&] { k_dadd<<<blocks, threads>>>((double *)buf, 1e-3, 0.0); })) return 1;
  if (time_it("FP64 DMUL (__dmul_rn)", n, 1, blocks, threads, ghz, sms,
              [&] { k_dmul<<<blocks, threads>>>((double *)buf, 0.9999999, 0.0); })) return 1;
  if (time_it("FP64 sqrt (__dsqrt_rn)", n / 16, 0, blocks, threads, ghz, sms,
              [&] { k_dsqrt<<<blocks, threads>>>((double *)buf, 1.0, 0.0); })) return 1;
  if (time_it("FP32 sqrt (__fsqrt_rn)", n, 0, blocks, threads, ghz, sms,
              [&] { k_fsqrt<<<blocks, threads>>>((float *)buf, 1.0f, 0.0f); })) return 1;
  if (time_it("float->double->float round trip (2 cvt + 1 DFMA)", n, 0, blocks, threads, ghz, sms,
              [&] { k_cvt<<<blocks, threads>>>((float *)buf, 0.999f, 1e-3f); })) return 1;
  if (time_it("64-bit __umul64hi", n, 0, blocks, threads, ghz, sms,
              [&] { k_umulhi<<<blocks, threads>>>((unsigned long long *)buf,
                                                   0x9e3779b97f4a7c15ull, 12345ull); })) return 1;
  CK(cudaFree(buf));
  return 0;
}
