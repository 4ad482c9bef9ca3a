// ALU throughput microbenchmark for the per-patch SRHD update.
//
// The fluid update is bound by plain ALU arithmetic (Newton solves with
// square roots and divisions), not by HBM and not by tensor cores, so its
// roofline denominators are the FP32 FMA, FP64 FMA and special-function
// rates of the GPU. This program measures them with long chains of
// independent operations per thread, a grid that is a multiple of the SM
// count, and CUDA events. It prints one JSON object.
//
// Build and run (one GPU):
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o alu_peaks alu_peaks.cu
//   ./alu_peaks
#include <cstdio>
#include <cuda_runtime.h>

#define CK(x)                                                                 \
  do {                                                                        \
    cudaError_t e_ = (x);                                                     \
    if (e_ != cudaSuccess) {                                                  \
      fprintf(stderr, "CUDA error %s at %s:%d\n", cudaGetErrorString(e_),     \
              __FILE__, __LINE__);                                            \
      return 1;                                                               \
    }                                                                         \
  } while (0)

constexpr int kChains = 8;

template <typename T>
__global__ void fma_chain(T* out, T b, T c, int iters) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = a[k] * b + c;
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == T(-12345.678)) out[blockIdx.x] = s;  // never true; keeps the chains live
}

// x <- c / (x + b): one division per step, kChains independent chains.
template <typename T>
__global__ void div_chain(T* out, T b, T c, int iters) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = T(1) + T(threadIdx.x + k) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = c / (a[k] + b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == T(-12345.678)) out[blockIdx.x] = s;
}

// x <- sqrt(x + b): one square root per step.
template <typename T>
__global__ void sqrt_chain(T* out, T b, int iters) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = T(1) + T(threadIdx.x + k) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = sqrt(a[k] + b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == T(-12345.678)) out[blockIdx.x] = s;
}

// Packed FP32 (sm_100 family): one instruction performs two FMAs, a <- a b + c
// on float2, kChains independent chains per thread.
__global__ void ffma2_chain(float* out, float b, float c, int iters) {
  float2 a[kChains];
  const float2 bb = make_float2(b, b), cc = make_float2(c, c);
#pragma unroll
  for (int k = 0; k < kChains; ++k)
    a[k] = make_float2(float(threadIdx.x + k) * 1e-3f, float(threadIdx.x + 2 * k) * 1e-3f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], bb, cc);
  }
  float s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
  if (s == -12345.678f) out[blockIdx.x] = s;
}

// FP32 approximate division (__fdividef: reciprocal on the special-function
// unit and one multiply): x <- c / (x + b).
__global__ void fdiv_chain(float* out, float b, float c, int iters) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.f + float(threadIdx.x + k) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = __fdividef(c, a[k] + b);
  }
  float s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -12345.678f) out[blockIdx.x] = s;
}

// Special-function unit: x <- rsqrtf(x + b) (approximate, one MUFU op + FADD).
__global__ void rsqrt_chain(float* out, float b, int iters) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.f + float(threadIdx.x + k) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = rsqrtf(a[k] + b);
  }
  float s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -12345.678f) out[blockIdx.x] = s;
}

template <typename K>
static float time_ms(K launch, cudaEvent_t e0, cudaEvent_t e1) {
  launch();  // warm-up
  cudaDeviceSynchronize();
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  return best;
}

int main() {
  int dev = 0, nsm = 0, clk_khz = 0;
  CK(cudaSetDevice(dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  const int threads = 256;
  const int blocks = nsm * 8;
  const double nthreads = double(threads) * blocks;
  void* out = nullptr;
  CK(cudaMalloc(&out, sizeof(double) * blocks));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));

  const int it32 = 4096, it64 = 256, itdiv64 = 32, itdiv32 = 512, itmufu = 2048;
  float* o32 = static_cast<float*>(out);
  double* o64 = static_cast<double*>(out);

  float t_f32 = time_ms([&] { fma_chain<float><<<blocks, threads>>>(o32, 0.999f, 1e-4f, it32); }, e0, e1);
  float t_f64 = time_ms([&] { fma_chain<double><<<blocks, threads>>>(o64, 0.999, 1e-4, it64); }, e0, e1);
  float t_d64 = time_ms([&] { div_chain<double><<<blocks, threads>>>(o64, 0.5, 1.5, itdiv64); }, e0, e1);
  float t_s64 = time_ms([&] { sqrt_chain<double><<<blocks, threads>>>(o64, 0.5, itdiv64); }, e0, e1);
  float t_d32 = time_ms([&] { div_chain<float><<<blocks, threads>>>(o32, 0.5f, 1.5f, itdiv32); }, e0, e1);
  float t_s32 = time_ms([&] { sqrt_chain<float><<<blocks, threads>>>(o32, 0.5f, itdiv32); }, e0, e1);
  float t_rsq = time_ms([&] { rsqrt_chain<<<blocks, threads>>>(o32, 0.5f, itmufu); }, e0, e1);
  float t_f2 = time_ms([&] { ffma2_chain<<<blocks, threads>>>(o32, 0.999f, 1e-4f, it32); }, e0, e1);
  float t_fd = time_ms([&] { fdiv_chain<<<blocks, threads>>>(o32, 0.5f, 1.5f, itmufu); }, e0, e1);
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());

  auto rate = [&](int iters, float ms) { return nthreads * kChains * iters / (ms * 1e-3); };
  printf("{\"sm_count\": %d, \"clock_mhz_attr\": %.0f,\n", nsm, clk_khz / 1e3);
  printf(" \"fp32_fma_tflops\": %.3f,\n", 2.0 * rate(it32, t_f32) / 1e12);
  printf(" \"fp64_fma_tflops\": %.4f,\n", 2.0 * rate(it64, t_f64) / 1e12);
  printf(" \"fp64_div_gops\": %.3f,\n", rate(itdiv64, t_d64) / 1e9);
  printf(" \"fp64_sqrt_gops\": %.3f,\n", rate(itdiv64, t_s64) / 1e9);
  printf(" \"fp32_ieee_div_gops\": %.3f,\n", rate(itdiv32, t_d32) / 1e9);
  printf(" \"fp32_ieee_sqrt_gops\": %.3f,\n", rate(itdiv32, t_s32) / 1e9);
  printf(" \"fp32_rsqrt_mufu_gops\": %.3f,\n", rate(itmufu, t_rsq) / 1e9);
  printf(" \"fp32x2_ffma2_tflops\": %.3f,\n", 4.0 * rate(it32, t_f2) / 1e12);
  printf(" \"fp32_fdividef_gops\": %.3f}\n", rate(itmufu, t_fd) / 1e9);
  cudaFree(out);
  return 0;
}
