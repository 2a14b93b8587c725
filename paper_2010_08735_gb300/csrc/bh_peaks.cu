// Issue-rate microbenchmark of the GPU's SMs, for the roofline denominators of
// the render kernel: scalar FP32 FMA, packed FP32 (f32x2) FMA and the special
// function unit (reciprocal square root), each measured as results per SM per
// clock with independent dependency chains that fill every SM.  The paper has
// no counterpart; this measures the hardware the beam tracer runs on.
#include <algorithm>

#include "bh_internal.cuh"

namespace bh {

constexpr int kPeakChains = 8;     // independent chains per thread
constexpr int kPeakThreads = 256;  // threads per block
constexpr int kPeakBlocksPerSm = 4;

__device__ __forceinline__ void note_cycles(unsigned long long *cyc, long long t0) {
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(cyc, (unsigned long long)(clock64() - t0));
}

__global__ void __launch_bounds__(kPeakThreads) peak_fma_kernel(int iters, float a, float b, float *sink,
                                                                unsigned long long *cyc) {
  float x[kPeakChains];
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) x[k] = threadIdx.x * 1e-3f + k;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) x[k] = fmaf(x[k], a, b);
  }
  note_cycles(cyc, t0);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) s += x[k];
  if (s == 1234.5f) sink[threadIdx.x] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(kPeakThreads) peak_ffma2_kernel(int iters, float a, float b, float *sink,
                                                                  unsigned long long *cyc) {
  float2 x[kPeakChains];
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) x[k] = make_float2(threadIdx.x * 1e-3f + k, k - threadIdx.x * 1e-3f);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
  }
  note_cycles(cyc, t0);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) s += x[k].x + x[k].y;
  if (s == 1234.5f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) peak_mufu_kernel(int iters, float *sink, unsigned long long *cyc) {
  float x[kPeakChains];
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) x[k] = 1.5f + threadIdx.x * 1e-3f + k;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(x[k]));
  }
  note_cycles(cyc, t0);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) s += x[k];
  if (s == 1234.5f) sink[threadIdx.x] = s;
}

// Zero-copy stores into mapped pinned host memory: every thread writes
// 16-byte chunks, a warp 512 contiguous bytes per instruction (whole 128-byte
// lines), grid-stride.
__global__ void link_store_kernel(float4 *dst, long long n4) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = make_float4((float)(i & 1023), 1.f, 2.f, 3.f);
}

}  // namespace bh

using namespace bh;

// Bandwidth of the link from the device to host memory, for the end-to-end
// (frames to the host) roofline: bytes (rounded down to 16) moved from device
// memory to pinned host memory by the copy engine, and written into pinned
// host memory by kernel stores; best of five timed runs each after one
// untimed.
extern "C" bh_status bh_measure_host_link(int device, size_t bytes, double *out) {
  if (!out || bytes < 16) { set_error("bh_measure_host_link: NULL out or fewer than 16 bytes"); return BH_ERR_INVALID_ARG; }
  bytes &= ~(size_t)15;
  BH_CUDA(cudaSetDevice(device));
  int sms = 0;
  BH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  void *dev = nullptr, *host = nullptr, *mapped = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&dev, bytes);
  if (e == cudaSuccess) e = cudaHostAlloc(&host, bytes, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&mapped, host, 0);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMemsetAsync(dev, 0, bytes, s);
  double gbs[2] = {0.0, 0.0};
  for (int which = 0; which < 2 && e == cudaSuccess; ++which) {
    for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
      cudaEventRecord(e0, s);
      if (which == 0) e = cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, s);
      else link_store_kernel<<<sms * 4, 256, 0, s>>>(static_cast<float4 *>(mapped), (long long)(bytes / 16));
      if (e == cudaSuccess) e = cudaGetLastError();
      cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && rep > 0 && ms > 0.f) gbs[which] = std::max(gbs[which], bytes / (ms * 1e-3) / 1e9);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (host) cudaFreeHost(host);
  if (dev) cudaFree(dev);
  if (e != cudaSuccess) return cuda_fail(e, "bh_measure_host_link");
  out[0] = gbs[0];
  out[1] = gbs[1];
  return BH_OK;
}

extern "C" bh_status bh_measure_issue_rates(int device, double *out) {
  if (!out) { set_error("bh_measure_issue_rates: NULL argument"); return BH_ERR_INVALID_ARG; }
  BH_CUDA(cudaSetDevice(device));
  int sms = 0;
  BH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  float *sink = nullptr;
  unsigned long long *cyc = nullptr;
  cudaError_t e = cudaMalloc((void **)&sink, sizeof(float) * kPeakThreads);
  if (e == cudaSuccess) e = cudaMalloc((void **)&cyc, sizeof(unsigned long long));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int grid = sms * kPeakBlocksPerSm;
  const int iters = 4096;
  // per thread: iters * 4 * chains operations (FFMA2: two FMAs each)
  const double ops_per_thread = (double)iters * 4 * kPeakChains;
  double rate[3] = {0, 0, 0}, mhz = 0.0;
  for (int which = 0; which < 3 && e == cudaSuccess; ++which) {
    double best = 0.0;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      e = cudaMemset(cyc, 0, sizeof(unsigned long long));
      if (e != cudaSuccess) break;
      cudaEventRecord(e0);
      if (which == 0) peak_fma_kernel<<<grid, kPeakThreads>>>(iters, 0.9999999f, 1e-7f, sink, cyc);
      else if (which == 1) peak_ffma2_kernel<<<grid, kPeakThreads>>>(iters, 0.9999999f, 1e-7f, sink, cyc);
      else peak_mufu_kernel<<<grid, kPeakThreads>>>(iters, sink, cyc);
      cudaEventRecord(e1);
      e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaGetLastError();
      unsigned long long c = 0;
      if (e == cudaSuccess) e = cudaMemcpy(&c, cyc, sizeof c, cudaMemcpyDeviceToHost);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess || c == 0) break;
      // every block of the grid is resident at once: an SM runs kPeakBlocksPerSm
      // blocks' operations in the longest block's cycles
      const double per_sm = ops_per_thread * kPeakThreads * kPeakBlocksPerSm * (which == 1 ? 2.0 : 1.0);
      const double r = per_sm / (double)c;
      if (r > best) {
        best = r;
        if (ms > 0.f) mhz = std::max(mhz, (double)c / (ms * 1e3));
      }
    }
    rate[which] = best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  cudaFree(cyc);
  if (e != cudaSuccess) return cuda_fail(e, "bh_measure_issue_rates");
  out[0] = rate[0];
  out[1] = rate[1];
  out[2] = rate[2];
  out[3] = (double)sms;
  out[4] = mhz;
  return BH_OK;
}
