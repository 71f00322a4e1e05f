// FP64 throughput of this GPU, measured: the denominator of the roofline fractions that the
// benchmark reports for the hQR kernels (every kernel of the path is bound by FP64 arithmetic,
// not by memory traffic).  Two instruction paths are timed:
//
//  * DFMA: each thread runs 8 independent fused multiply-add chains (enough independent work
//    to hide the FMA latency), grid of 4 CTAs of 256 threads per SM;
//  * DMMA: the FP64 tensor-core instruction mma.sync.m8n8k4 (one 8x8x4 product, 512 flops
//    per warp instruction), 8 independent accumulator pairs per warp, same grid.
//
// The elapsed time is taken with CUDA events around each launch on a private stream, best of
// `reps` launches.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/hodlr_qr.h"
#include "common.cuh"

namespace hq {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;
constexpr int kPeakUnroll = 16;

__global__ void __launch_bounds__(kPeakThreads) dfma_peak_kernel(double* sink, int iters, double a, double b) {
  double x[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) x[c] = 1e-3 * (threadIdx.x + 1) + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kPeakChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) s += x[c];
  if (s == -1.0) sink[0] = s;                     // never taken; keeps the chains live
}

__global__ void __launch_bounds__(kPeakThreads) dmma_peak_kernel(double* sink, int iters, double a, double b) {
  double c0[kPeakChains], c1[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) {
    c0[c] = 1e-3 * threadIdx.x + c;
    c1[c] = 2e-3 * threadIdx.x - c;
  }
  const double av = a * (1.0 + 1e-6 * (threadIdx.x & 31)), bv = b;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kPeakChains; ++c)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                     : "+d"(c0[c]), "+d"(c1[c])
                     : "d"(av), "d"(bv));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) s += c0[c] + c1[c];
  if (s == -1.0) sink[0] = s;
}

}  // namespace hq

extern "C" int hodlr_fp64_peak(int device, int iters, int reps, double* dfma_tflops, double* dmma_tflops) {
  using namespace hq;
  if (iters < 1 || reps < 1 || !dfma_tflops || !dmma_tflops) return HODLR_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return HODLR_EINVAL;
  }
  HQ_CUDA_OK(cudaSetDevice(device));
  int sms = 0;
  HQ_CUDA_OK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  const int blocks = 4 * sms;          // 4 x 256 threads per SM: 32 warps of independent chains
  double* sink = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = HODLR_OK;
  if (cudaMalloc(&sink, sizeof(double)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    rc = HODLR_ENOMEM;
  }
  double best[2] = {0.0, 0.0};
  for (int kind = 0; kind < 2 && rc == HODLR_OK; ++kind) {
    // flops of one launch: DFMA 2 per lane per FMA; DMMA 2 * 8 * 8 * 4 per warp instruction
    const double per_iter = kind == 0 ? 2.0 * kPeakChains * kPeakUnroll * kPeakThreads
                                      : 512.0 * kPeakChains * kPeakUnroll * (kPeakThreads / 32);
    const double flops = per_iter * iters * blocks;
    for (int r = 0; r <= reps && rc == HODLR_OK; ++r) {   // launch 0 warms up
      cudaEventRecord(e0, s);
      if (kind == 0) dfma_peak_kernel<<<blocks, kPeakThreads, 0, s>>>(sink, iters, 0.9999999, 1e-7);
      else dmma_peak_kernel<<<blocks, kPeakThreads, 0, s>>>(sink, iters, 0.9999999, 1e-7);
      cudaEventRecord(e1, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), __FILE__, __LINE__);
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r == 0 || ms <= 0.0f) continue;
      best[kind] = std::max(best[kind], flops / (ms * 1e-3) / 1e12);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (sink) cudaFree(sink);
  if (rc) return rc;
  *dfma_tflops = best[0];
  *dmma_tflops = best[1];
  return HODLR_OK;
}
