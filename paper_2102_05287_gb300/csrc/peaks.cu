// Vector-pipe peak microbenchmarks for the stencil roofline.
//
// The RHS evaluation has no dense contraction, so its roofline is set by
// the FP64 and FP32 vector pipes (and HBM for the byte term).  This
// stand-alone program measures, on the device it runs on:
//   * FP64 FMA throughput  (independent dependent-chains, 2 flop per FMA)
//   * FP32 FMA throughput
//   * FP64 division and square-root throughput (operations/s; these are
//     multi-instruction sequences, reported as ops, not flops)
//   * FP32 division (IEEE a / b and the approximate __fdividef) and sqrtf
//     throughput, the forms the mixed-precision sweeps use
//   * a STREAM-style FP64 copy bandwidth
// and prints one JSON object.  Timing uses CUDA events after warm-up.
//
// Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3 peaks.cu -o peaks
#include <cstdio>
#include <cstdlib>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { \
  fprintf(stderr, "CUDA error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
  exit(1); } } while (0)

template <typename T, int NCHAIN>
__global__ void fma_chain(T *out, int iters, T a, T b) {
  T acc[NCHAIN];
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) acc[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) acc[c] = acc[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) s += acc[c];
  if (s == (T)-12345.678) out[blockIdx.x] = s;  // never true; keeps the work live
}

template <int NCHAIN>
__global__ void div_chain(double *out, int iters, double b) {
  double acc[NCHAIN];
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) acc[c] = 1.0 + (threadIdx.x + c) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) acc[c] = b / acc[c];
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) s += acc[c];
  if (s == -12345.678) out[blockIdx.x] = s;
}

template <int NCHAIN>
__global__ void sqrt_chain(double *out, int iters) {
  double acc[NCHAIN];
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) acc[c] = 2.0 + (threadIdx.x + c) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) acc[c] = sqrt(acc[c]) + 1.0;
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) s += acc[c];
  if (s == -12345.678) out[blockIdx.x] = s;
}

// FP32 division chains: IEEE-rounded a / b (FAST = false) or __fdividef.
template <int NCHAIN, bool FAST>
__global__ void div32_chain(float *out, int iters, float b) {
  float acc[NCHAIN];
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) acc[c] = 1.0f + (threadIdx.x + c) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) acc[c] = FAST ? __fdividef(b, acc[c]) : b / acc[c];
  }
  float s = 0;
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) s += acc[c];
  if (s == -12345.678f) out[blockIdx.x] = s;
}

template <int NCHAIN>
__global__ void sqrt32_chain(float *out, int iters) {
  float acc[NCHAIN];
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) acc[c] = 2.0f + (threadIdx.x + c) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) acc[c] = sqrtf(acc[c]) + 1.0f;
  }
  float s = 0;
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) s += acc[c];
  if (s == -12345.678f) out[blockIdx.x] = s;
}

__global__ void copy_kernel(const double2 *__restrict__ src, double2 *__restrict__ dst, size_t n) {
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

template <typename F>
static float time_ms(F launch, int reps) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int w = 0; w < 3; ++w) launch();
  CK(cudaDeviceSynchronize());
  CK(cudaEventRecord(e0));
  for (int r = 0; r < reps; ++r) launch();
  CK(cudaEventRecord(e1));
  CK(cudaEventSynchronize(e1));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  CK(cudaEventDestroy(e0));
  CK(cudaEventDestroy(e1));
  return ms / reps;
}

int main() {
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, 0));
  int sms = prop.multiProcessorCount;
  double *out;
  CK(cudaMalloc(&out, 1 << 20));
  const int threads = 256;
  const int blocks = sms * 8;
  const double nthreads = (double)blocks * threads;

  const int it64 = 4096;
  float ms64 = time_ms([&] { fma_chain<double, 8><<<blocks, threads>>>(out, it64, 0.999999, 1e-7); }, 5);
  double fp64_tflops = nthreads * it64 * 8 * 2.0 / (ms64 * 1e-3) / 1e12;

  const int it32 = 65536;
  float ms32 = time_ms([&] { fma_chain<float, 8><<<blocks, threads>>>((float *)out, it32, 0.999999f, 1e-7f); }, 5);
  double fp32_tflops = nthreads * it32 * 8 * 2.0 / (ms32 * 1e-3) / 1e12;

  const int itd = 512;
  float msd = time_ms([&] { div_chain<4><<<blocks, threads>>>(out, itd, 1.5); }, 3);
  double div_gops = nthreads * itd * 4 / (msd * 1e-3) / 1e9;

  const int its = 512;
  float mss = time_ms([&] { sqrt_chain<4><<<blocks, threads>>>(out, its); }, 3);
  double sqrt_gops = nthreads * its * 4 / (mss * 1e-3) / 1e9;

  const int it32d = 4096;
  float msd32 = time_ms([&] { div32_chain<8, false><<<blocks, threads>>>((float *)out, it32d, 1.5f); }, 3);
  double div32_gops = nthreads * it32d * 8 / (msd32 * 1e-3) / 1e9;
  float msf32 = time_ms([&] { div32_chain<8, true><<<blocks, threads>>>((float *)out, it32d, 1.5f); }, 3);
  double fdiv32_gops = nthreads * it32d * 8 / (msf32 * 1e-3) / 1e9;
  float mss32 = time_ms([&] { sqrt32_chain<8><<<blocks, threads>>>((float *)out, it32d); }, 3);
  double sqrt32_gops = nthreads * it32d * 8 / (mss32 * 1e-3) / 1e9;

  size_t nbytes = (size_t)2 << 30;  // 2 GiB per buffer, far above L2
  size_t n2 = nbytes / sizeof(double2);
  double2 *a, *b;
  CK(cudaMalloc(&a, nbytes));
  CK(cudaMalloc(&b, nbytes));
  CK(cudaMemset(a, 0, nbytes));
  float msc = time_ms([&] { copy_kernel<<<sms * 16, 512>>>(a, b, n2); }, 10);
  double copy_gbs = 2.0 * nbytes / (msc * 1e-3) / 1e9;

  int clock_khz = 0;
  CK(cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, 0));
  printf("{\"device\": \"%s\", \"sms\": %d, \"fp64_fma_tflops\": %.4f, \"fp32_fma_tflops\": %.3f, "
         "\"fp64_div_gops\": %.2f, \"fp64_sqrt_gops\": %.2f, \"fp32_div_gops\": %.1f, "
         "\"fp32_fdividef_gops\": %.1f, \"fp32_sqrt_gops\": %.1f, \"fp64_copy_gbs\": %.1f, "
         "\"clock_khz\": %d}\n",
         prop.name, sms, fp64_tflops, fp32_tflops, div_gops, sqrt_gops, div32_gops, fdiv32_gops, sqrt32_gops,
         copy_gbs, clock_khz);
  CK(cudaFree(a));
  CK(cudaFree(b));
  CK(cudaFree(out));
  return 0;
}
