// Lens glare (Sec. 3.4.3): a bloom applied to the linear-RGB frame before
// tone mapping, made of small filter kernels on a mip pyramid of the frame
// that together approximate the photopic point spread function of Spencer,
// Shirley, Zimmerman and Greenberg (SIGGRAPH 1995), as the paper does.
//
// Pyramid: D_0 = the frame; D_k = 2x2 box average of D_{k-1} (sizes rounded
// up, indices clamped); B_k = D_k blurred by a separable 7-tap Gaussian of
// one texel's standard deviation (clamped edges).  Output:
//   out = w_0 in + sum_{k=1..K} w_k bilinear(B_k)  (texel centres, clamped)
// with w_k the share of the PSF's energy in the annulus of radii
// [2^(k-1/2), 2^(k+1/2)) pixels (w_0: radii below 2^(1/2)), normalised over
// radii below 2^(K+1/2); pixel angle = fov_y / height.  The weights are
// computed on the host from the PSF's closed-form annulus integrals.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "bh_internal.cuh"

namespace bh {

constexpr int kBloomMaxLevels = 10;

// Spencer et al.'s photopic PSF, theta in degrees: 0.384 f0 + 0.478 f1 + 0.138 f2,
// f0 = 2.61e6 exp(-(theta/0.02)^2), f1 = 20.91/(theta+0.02)^3, f2 = 72.37/(theta+0.02)^2.
// Energy of the PSF between angles a and b: the integral of P(theta) 2 pi theta dtheta.
static double psf_energy(double a, double b) {
  const double s = 0.02, c = 0.02;
  auto e0 = [&](double t) { return -2.61e6 * kPi * s * s * exp(-(t / s) * (t / s)); };
  auto e1 = [&](double t) { double u = t + c; return 2.0 * kPi * 20.91 * (-1.0 / u + c / (2.0 * u * u)); };
  auto e2 = [&](double t) { double u = t + c; return 2.0 * kPi * 72.37 * (log(u) + c / u); };
  return 0.384 * (e0(b) - e0(a)) + 0.478 * (e1(b) - e1(a)) + 0.138 * (e2(b) - e2(a));
}

__global__ void bloom_down_kernel(const float4 *src, int sw, int sh, float4 *dst, int dw, int dh) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= dw || y >= dh) return;
  const int x0 = min(2 * x, sw - 1), x1 = min(2 * x + 1, sw - 1);
  const int y0 = min(2 * y, sh - 1), y1 = min(2 * y + 1, sh - 1);
  const float4 a = src[(size_t)y0 * sw + x0], b = src[(size_t)y0 * sw + x1];
  const float4 c = src[(size_t)y1 * sw + x0], d = src[(size_t)y1 * sw + x1];
  dst[(size_t)y * dw + x] = make_float4(0.25f * ((a.x + b.x) + (c.x + d.x)), 0.25f * ((a.y + b.y) + (c.y + d.y)),
                                        0.25f * ((a.z + b.z) + (c.z + d.z)), 1.f);
}

// 7-tap Gaussian of unit standard deviation, normalised (taps at -3..3)
__constant__ float cBloomTaps[4];

// dir 0: along x, 1: along y
__global__ void bloom_blur_kernel(const float4 *src, float4 *dst, int w, int h, int dir) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= w || y >= h) return;
  float r = 0.f, g = 0.f, b = 0.f;
#pragma unroll
  for (int t = -3; t <= 3; ++t) {
    const int xx = dir == 0 ? min(max(x + t, 0), w - 1) : x;
    const int yy = dir == 1 ? min(max(y + t, 0), h - 1) : y;
    const float4 v = src[(size_t)yy * w + xx];
    const float k = cBloomTaps[t < 0 ? -t : t];
    r = fmaf(k, v.x, r);
    g = fmaf(k, v.y, g);
    b = fmaf(k, v.z, b);
  }
  dst[(size_t)y * w + x] = make_float4(r, g, b, 1.f);
}

struct BloomLevels {
  const float4 *lev[kBloomMaxLevels + 1];
  int w[kBloomMaxLevels + 1], h[kBloomMaxLevels + 1];
  float wt[kBloomMaxLevels + 1];
  int n;
};

__global__ void bloom_composite_kernel(const float4 *in, float4 *out, int W, int H, const BloomLevels L) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  const float4 c = in[(size_t)y * W + x];
  float r = L.wt[0] * c.x, g = L.wt[0] * c.y, b = L.wt[0] * c.z;
  for (int k = 1; k <= L.n; ++k) {
    const float s = 1.f / (float)(1 << k);
    const float u = fmaf((float)x + 0.5f, s, -0.5f), v = fmaf((float)y + 0.5f, s, -0.5f);
    const float fu = floorf(u), fv = floorf(v);
    const float tu = u - fu, tv = v - fv;
    const int w = L.w[k], h = L.h[k];
    const int i0 = min(max((int)fu, 0), w - 1), i1 = min(max((int)fu + 1, 0), w - 1);
    const int j0 = min(max((int)fv, 0), h - 1), j1 = min(max((int)fv + 1, 0), h - 1);
    const float4 *p = L.lev[k];
    const float4 a = p[(size_t)j0 * w + i0], bb = p[(size_t)j0 * w + i1];
    const float4 cc = p[(size_t)j1 * w + i0], d = p[(size_t)j1 * w + i1];
    const float wk = L.wt[k];
    const float lr = fmaf(tv, fmaf(tu, d.x - cc.x, cc.x) - fmaf(tu, bb.x - a.x, a.x), fmaf(tu, bb.x - a.x, a.x));
    const float lg = fmaf(tv, fmaf(tu, d.y - cc.y, cc.y) - fmaf(tu, bb.y - a.y, a.y), fmaf(tu, bb.y - a.y, a.y));
    const float lb = fmaf(tv, fmaf(tu, d.z - cc.z, cc.z) - fmaf(tu, bb.z - a.z, a.z), fmaf(tu, bb.z - a.z, a.z));
    r = fmaf(wk, lr, r);
    g = fmaf(wk, lg, g);
    b = fmaf(wk, lb, b);
  }
  out[(size_t)y * W + x] = make_float4(r, g, b, 1.f);
}

}  // namespace bh

using namespace bh;

extern "C" bh_status bh_bloom_weights(double fov_y, int height, int levels, double *weights) {
  if (!weights || !(fov_y > 0.0 && fov_y < kPi) || height < 1 || levels < 0 || levels > kBloomMaxLevels) {
    set_error("bh_bloom_weights: need 0 < fov_y < pi, height >= 1, 0 <= levels <= %d", kBloomMaxLevels);
    return BH_ERR_INVALID_ARG;
  }
  const double a = fov_y * 180.0 / kPi / height;  // degrees per pixel
  const double total = psf_energy(0.0, a * ldexp(1.0, levels) * sqrt(2.0));
  weights[0] = psf_energy(0.0, a * sqrt(2.0)) / total;
  for (int k = 1; k <= levels; ++k)
    weights[k] = psf_energy(a * ldexp(1.0, k) / sqrt(2.0), a * ldexp(1.0, k) * sqrt(2.0)) / total;
  return BH_OK;
}

extern "C" bh_status bh_bloom(bh_ctx *ctx, const float *in_device, float *out_device, int width, int height,
                              int levels, const double *weights, void *stream) {
  TraceRange trace_("bh_bloom");
  if (!ctx || !in_device || !out_device || !weights) { set_error("bh_bloom: NULL argument"); return BH_ERR_INVALID_ARG; }
  if (width < 1 || height < 1 || width > 16384 || height > 16384 || levels < 0 || levels > kBloomMaxLevels) {
    set_error("bh_bloom: size %dx%d out of 1..16384 or levels %d out of 0..%d", width, height, levels,
              kBloomMaxLevels);
    return BH_ERR_INVALID_ARG;
  }
  if (((uintptr_t)in_device & 15) || ((uintptr_t)out_device & 15)) {
    set_error("bh_bloom: buffers must be 16-byte aligned");
    return BH_ERR_INVALID_ARG;
  }
  BH_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  // pyramid sizes and scratch: D_k and B_k per level, plus one blur temporary
  int w[kBloomMaxLevels + 1], h[kBloomMaxLevels + 1];
  w[0] = width;
  h[0] = height;
  size_t texels = 0, tmp = 0;
  for (int k = 1; k <= levels; ++k) {
    w[k] = (w[k - 1] + 1) / 2;
    h[k] = (h[k - 1] + 1) / 2;
    texels += 2 * (size_t)w[k] * h[k];
    tmp = std::max(tmp, (size_t)w[k] * h[k]);
  }
  const size_t need = (texels + tmp) * sizeof(float4);
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (need > ctx->bloom_cap) {
    if (ctx->bloom_dev) {
      BH_CUDA(cudaStreamSynchronize(s));
      cudaFree(ctx->bloom_dev);
      ctx->bloom_dev = nullptr;
      ctx->bloom_cap = 0;
    }
    BH_CUDA(cudaMalloc((void **)&ctx->bloom_dev, need));
    ctx->bloom_cap = need;
  }
  static bool taps_ready[64] = {false};
  if (ctx->device < 64 && !taps_ready[ctx->device]) {
    double t[4], sum = 0.0;
    for (int i = 0; i < 4; ++i) {
      t[i] = exp(-0.5 * i * i);
      sum += (i == 0 ? 1.0 : 2.0) * t[i];
    }
    float tf[4];
    for (int i = 0; i < 4; ++i) tf[i] = (float)(t[i] / sum);
    BH_CUDA(cudaMemcpyToSymbol(cBloomTaps, tf, sizeof tf));
    taps_ready[ctx->device] = true;
  }
  BloomLevels L;
  memset(&L, 0, sizeof L);
  L.n = levels;
  for (int k = 0; k <= levels; ++k) {
    L.w[k] = w[k];
    L.h[k] = h[k];
    L.wt[k] = (float)weights[k];
  }
  float4 *base = reinterpret_cast<float4 *>(ctx->bloom_dev);
  float4 *scratch = base + texels;
  const float4 *prev = reinterpret_cast<const float4 *>(in_device);
  float4 *cur = base;
  const dim3 blk(32, 8);
  for (int k = 1; k <= levels; ++k) {
    float4 *Dk = cur, *Bk = cur + (size_t)w[k] * h[k];
    const dim3 g((w[k] + 31) / 32, (h[k] + 7) / 8);
    bloom_down_kernel<<<g, blk, 0, s>>>(prev, w[k - 1], h[k - 1], Dk, w[k], h[k]);
    bloom_blur_kernel<<<g, blk, 0, s>>>(Dk, scratch, w[k], h[k], 0);
    bloom_blur_kernel<<<g, blk, 0, s>>>(scratch, Bk, w[k], h[k], 1);
    L.lev[k] = Bk;
    prev = Dk;
    cur = Bk + (size_t)w[k] * h[k];
  }
  bloom_composite_kernel<<<dim3((width + 31) / 32, (height + 7) / 8), blk, 0, s>>>(
      reinterpret_cast<const float4 *>(in_device), reinterpret_cast<float4 *>(out_device), width, height, L);
  count_launch(ctx, 3 * levels + 1);
  BH_CUDA(cudaGetLastError());
  return BH_OK;
}
