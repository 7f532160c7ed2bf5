// dies_peaks.cu -- microbenchmarks for the roofline denominators of the IRE
// transport.  The path is neither a dense contraction nor a stream: its
// bounds are SM instruction issue (FP32, integer and MUFU work per crossing
// and per event) and the L2 FP64 atomic add with return that every
// absorption performs (Sect. 2.1: the absorbed energy updates the cell at
// once, and the old value fixes the re-emission interval).  Each kernel
// below saturates one of these on the whole GPU; rates are timed with CUDA
// events around a single launch after a warm-up launch.
#include "dies_common.cuh"

#include "dies.h"

namespace dies {
namespace {

constexpr int kPeakBlock = 256;
constexpr int kChains = 8;  // independent dependency chains per thread

// FP32 FMA issue: kChains independent chains of fmaf per thread.
__global__ void __launch_bounds__(kPeakBlock) k_peak_ffma(int iters, float a, float b, float *out) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 123.456f) out[0] = s;  // keeps the chains live
}

// Integer multiply-add issue (the Philox rounds are 32x32->64 multiplies).
__global__ void __launch_bounds__(kPeakBlock) k_peak_imad(int iters, uint32_t a, uint32_t b, uint32_t *out) {
  uint32_t x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 2654435761u + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;
  }
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s ^= x[c];
  if (s == 0x12345678u) out[0] = s;
}

// MUFU (special-function unit): base-2 logarithm of a running value.
__global__ void __launch_bounds__(kPeakBlock) k_peak_mufu(int iters, float a, float *out) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.5f + (float)(threadIdx.x + c) * 1e-4f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = __log2f(x[c]) + a;
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 123.456f) out[0] = s;
}

// FP64 FMA issue.
__global__ void __launch_bounds__(kPeakBlock) k_peak_dfma(int iters, double a, double b, double *out) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 123.456) out[0] = s;
}

// FP64 atomic add with return in L2: each thread adds to address
// (thread * stride + i * step) mod n_addr, n_addr = 1 gives one hot address.
// The returned values are summed so the returns cannot be dropped.
__global__ void __launch_bounds__(kPeakBlock) k_peak_atomic(int iters, double *acc, unsigned n_addr, double *out) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  unsigned a = (t * 2654435761u) % n_addr;
  for (int i = 0; i < iters; ++i) {
    s += atomicAdd(acc + a, 1.0);
    a += 97u;
    if (a >= n_addr) a -= n_addr * (a / n_addr);
  }
  if (s == -1.0) out[0] = s;
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

template <class F>
cudaError_t time_launch(F launch, float *ms) {
  cudaEvent_t e0, e1;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  launch();  // warm-up
  cudaEventRecord(e0, 0);
  launch();
  cudaEventRecord(e1, 0);
  e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace
}  // namespace dies

extern "C" int dies_measure_peaks(dies_peaks *out) {
  using namespace dies;
  if (!out) return DIES_EINVAL;
  *out = dies_peaks{};
  const int sms = sm_count();
  if (sms <= 0) return DIES_ECUDA;
  const int grid = sms * 8;  // 8 CTAs of 256 threads per SM: full occupancy for these small kernels
  const double threads = (double)grid * kPeakBlock;
  const size_t n_acc = (size_t)1 << 20;
  void *buf = nullptr;
  if (cudaMalloc(&buf, n_acc * sizeof(double) + 256) != cudaSuccess) return DIES_ENOMEM;
  double *acc = static_cast<double *>(buf);
  float *fsink = reinterpret_cast<float *>(static_cast<char *>(buf) + n_acc * sizeof(double));
  cudaError_t e = cudaMemset(buf, 0, n_acc * sizeof(double) + 256);
  float ms = 0.0f;
  const int it_alu = 1024, it_mufu = 1024, it_d = 512, it_atom = 64;
  auto rate = [&](double ops) { return ms > 0.0f ? ops / (ms * 1e-3) : 0.0; };
  if (e == cudaSuccess)
    e = time_launch([&] { k_peak_ffma<<<grid, kPeakBlock>>>(it_alu, 0.999f, 1e-3f, fsink); }, &ms);
  if (e == cudaSuccess) out->fp32_fma_per_s = rate(threads * it_alu * kChains);
  if (e == cudaSuccess)
    e = time_launch([&] { k_peak_imad<<<grid, kPeakBlock>>>(it_alu, 0x9e3779b9u, 7u, (uint32_t *)fsink); }, &ms);
  if (e == cudaSuccess) out->int_mad_per_s = rate(threads * it_alu * kChains);
  if (e == cudaSuccess)
    e = time_launch([&] { k_peak_mufu<<<grid, kPeakBlock>>>(it_mufu, 1.25f, fsink); }, &ms);
  if (e == cudaSuccess) out->mufu_per_s = rate(threads * it_mufu * kChains);
  if (e == cudaSuccess)
    e = time_launch([&] { k_peak_dfma<<<grid, kPeakBlock>>>(it_d, 0.999, 1e-3, (double *)fsink); }, &ms);
  if (e == cudaSuccess) out->fp64_fma_per_s = rate(threads * it_d * kChains);
  if (e == cudaSuccess)
    e = time_launch([&] { k_peak_atomic<<<grid, kPeakBlock>>>(it_atom, acc, (unsigned)n_acc, acc); }, &ms);
  if (e == cudaSuccess) out->atomic_f64_ret_distinct_per_s = rate(threads * it_atom);
  if (e == cudaSuccess)
    e = time_launch([&] { k_peak_atomic<<<grid, kPeakBlock>>>(it_atom / 4, acc, 64u, acc); }, &ms);
  if (e == cudaSuccess) out->atomic_f64_ret_64addr_per_s = rate(threads * (it_atom / 4));
  if (e == cudaSuccess)
    e = time_launch([&] { k_peak_atomic<<<grid, kPeakBlock>>>(1, acc, 1u, acc); }, &ms);
  if (e == cudaSuccess) out->atomic_f64_ret_same_per_s = rate(threads);
  out->sm_count = sms;
  launch_counter_add(14);
  cudaFree(buf);
  return e == cudaSuccess ? DIES_OK : DIES_ECUDA;
}
