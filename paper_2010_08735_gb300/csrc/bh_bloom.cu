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
// computed on the host from the PSF's closed-form annulus integrals.  The
// whole bloom is one cooperative launch: the levels are separated by a
// bounded grid barrier (a timeout sets a status bit, never hangs).
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

// 7-tap Gaussian of unit standard deviation, normalised (taps at -3..3)
__constant__ float cBloomTaps[4];

constexpr int kBloomTile = 64;                      // output texels per tile side
constexpr int kBloomHalo = 3;                       // blur radius
constexpr int kBloomSpan = kBloomTile + 2 * kBloomHalo;
constexpr int kBloomThreads = 1024;
// composite tiles: per level at most ceil((kCompH - 1) 2^-k) + 2 staged texel rows of kCompW entries
constexpr int kCompW = 256, kCompH = 32;
constexpr int comp_rows() {
  int n = 0;
  for (int k = 1; k <= kBloomMaxLevels; ++k) n += ((kCompH - 1) + (1 << k) - 1) / (1 << k) + 2;
  return n;
}
// shared-memory row strides, padded so that lanes on consecutive rows of sD
// or sH address distinct 16-byte bank groups
constexpr int kSDStride = kBloomSpan + 1, kSHStride = kBloomTile + 1;
constexpr int kBlurRun = 8;  // consecutive outputs per thread in each blur pass (a sliding window of taps)
constexpr size_t kBlurSmem = sizeof(float4) * (kBloomSpan * kSDStride + kBloomSpan * kSHStride);
constexpr size_t kCompSmem = sizeof(float4) * kCompW * comp_rows();
constexpr size_t kBloomSmem = kBlurSmem > kCompSmem ? kBlurSmem : kCompSmem;
// with the composite's per-row tables (2 x kCompH x kBloomMaxLevels words) and
// the barrier flag in static shared memory
static_assert(kBloomSmem + 2 * 4 * kCompH * kBloomMaxLevels + 16 <= 227 * 1024, "bloom shared memory");

struct BloomParams {
  const float4 *in;
  float4 *out;
  float4 *D[kBloomMaxLevels + 1];  // box levels (D[0] = in)
  float4 *B[kBloomMaxLevels + 1];  // blurred levels
  int w[kBloomMaxLevels + 1], h[kBloomMaxLevels + 1];
  float wt[kBloomMaxLevels + 1];
  int n;
  unsigned *bar;        // [0] grid-barrier arrivals, [1] blocks done (both zero at launch)
  unsigned *status;
  unsigned long long wait_ns;
  int inject;           // fault injection: block 0 never arrives at the first barrier
};

// Grid-wide barrier for a cooperative launch (every block resident): each
// block arrives once per phase and waits, for a bounded time, until all have
// arrived.  On expiry it sets a status bit and returns false (the caller
// stops), so a barrier can never hang the GPU.
__device__ bool grid_barrier(const BloomParams &P, unsigned phase) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    __threadfence();
    if (!(P.inject && phase == 1 && blockIdx.x == 0)) atomicAdd(P.bar, 1u);
    const unsigned target = gridDim.x * phase;
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    ok = 1;
    unsigned seen;
    for (;;) {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(seen) : "l"(P.bar) : "memory");
      if (seen >= target) break;
      __nanosleep(100);
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > P.wait_ns) {
        atomicOr(P.status, kStatusBarrierTimeout);
        ok = 0;
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Pull the frame rows of composite tile `tile` into L2 (one bulk prefetch per
// pixel row, issued by the lanes of warp 0): the composite of that tile then
// finds them there.  Rows start 16-byte aligned and span whole pixels.
__device__ __forceinline__ void prefetch_comp_tile(const BloomParams &P, int tile, int kw, int kh) {
  const int W = P.w[0], H = P.h[0];
  const int tcx = (W + kw - 1) / kw, ntiles = tcx * ((H + kh - 1) / kh);
  if (threadIdx.x >= 32 || tile >= ntiles) return;
  const int X0 = (tile % tcx) * kw, y = (tile / tcx) * kh + (int)threadIdx.x;
  if ((int)threadIdx.x >= kh || y >= H) return;
  const float4 *src = P.in + ((size_t)y * W + X0);
  const unsigned bytes = (unsigned)(sizeof(float4) * min(kw, W - X0));
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Pull the frame rows that region `reg` reads (its level-1 texels with their
// 3-texel halo: 140 x 140 pixels, clamped to the frame) into L2, one bulk
// prefetch per pixel row.
__device__ __forceinline__ void prefetch_region(const BloomParams &P, int reg) {
  const int W = P.w[0], H = P.h[0];
  const int rx = (P.w[1] + kBloomTile - 1) / kBloomTile, regions = rx * ((P.h[1] + kBloomTile - 1) / kBloomTile);
  constexpr int kRows = 2 * kBloomSpan;
  if (reg >= regions || (int)threadIdx.x >= kRows) return;
  const int gx = reg % rx, gy = reg / rx;
  const int y = 2 * (gy * kBloomTile - kBloomHalo) + (int)threadIdx.x;
  const int xa = max(2 * (gx * kBloomTile - kBloomHalo), 0), xb = min(2 * (gx * kBloomTile + kBloomTile + kBloomHalo), W);
  if (y < 0 || y >= H || xa >= xb) return;
  const float4 *src = P.in + ((size_t)y * W + xa);
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"((unsigned)(sizeof(float4) * (xb - xa)))
               : "memory");
}

// Box level k at texel (x, y), indices clamped to level k, from level k-1.
__device__ __forceinline__ float4 box_texel(const BloomParams &P, int k, int x, int y) {
  x = min(max(x, 0), P.w[k] - 1);
  y = min(max(y, 0), P.h[k] - 1);
  const int sw = P.w[k - 1], sh = P.h[k - 1];
  const float4 *src = P.D[k - 1];
  const int x0 = min(2 * x, sw - 1), x1 = min(2 * x + 1, sw - 1);
  const int y0 = min(2 * y, sh - 1), y1 = min(2 * y + 1, sh - 1);
  const float4 a = src[(size_t)y0 * sw + x0], b = src[(size_t)y0 * sw + x1];
  const float4 c = src[(size_t)y1 * sw + x0], d = src[(size_t)y1 * sw + x1];
  return make_float4(0.25f * ((a.x + b.x) + (c.x + d.x)), 0.25f * ((a.y + b.y) + (c.y + d.y)),
                     0.25f * ((a.z + b.z) + (c.z + d.z)), 1.f);
}

// Levels built in one pass from regions of the frame: a region is 64 x 64
// texels of level 1 (128 x 128 pixels), 32 x 32 of level 2, ..., one texel of
// level 7; a level-k texel's four children lie in its own region (clamped
// children at an odd edge are the texel's own first child), so a block
// reduces a region level by level in shared memory with no grid barrier.
constexpr int kBloomRegionLevels = 7;

// Blur (7 taps along x, then along y, clamped) of one 64x64 tile of level k
// whose box texels, with a 3-texel halo at clamped coordinates, are in sD.
__device__ void blur_staged(const BloomParams &P, int k, int x0, int y0, const float4 *sD, float4 *sH);

// The same, the box texels read from level k in global memory.
__device__ void blur_tile(const BloomParams &P, int k, int x0, int y0, float4 *sD, float4 *sH) {
  const int w = P.w[k], h = P.h[k];
  const float4 *Dk = P.D[k];
  for (int i = threadIdx.x; i < kBloomSpan * kBloomSpan; i += blockDim.x) {
    const int r = i / kBloomSpan, c = i - r * kBloomSpan;
    const int x = min(max(x0 + c - kBloomHalo, 0), w - 1), y = min(max(y0 + r - kBloomHalo, 0), h - 1);
    sD[r * kSDStride + c] = Dk[(size_t)y * w + x];
  }
  blur_staged(P, k, x0, y0, sD, sH);
}

__device__ void blur_staged(const BloomParams &P, int k, int x0, int y0, const float4 *sD, float4 *sH) {
  const int w = P.w[k], h = P.h[k];
  // Slot (r, c) of sD holds the texel at the clamped coordinates (x0 + c - 3,
  // y0 + r - 3), so a tap past the level's edge finds the clamped texel in its
  // own slot.  Each pass gives a thread kBlurRun consecutive outputs: it
  // streams their kBlurRun + 6 texels once, in order, each into the sums of
  // the outputs it is a tap of, so every output still sums its seven taps
  // from -3 to 3.
  __syncthreads();
  constexpr int kWin = kBlurRun + 2 * kBloomHalo;
  constexpr int kXItems = kBloomSpan * (kBloomTile / kBlurRun);
  for (int it = threadIdx.x; it < kXItems; it += blockDim.x) {
    const int r = it % kBloomSpan, c0 = (it / kBloomSpan) * kBlurRun;  // lanes on consecutive rows
    float3 acc[kBlurRun];
#pragma unroll
    for (int o = 0; o < kBlurRun; ++o) acc[o] = make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < kWin; ++j) {
      const float4 v = sD[r * kSDStride + c0 + j];
#pragma unroll
      for (int o = 0; o < kBlurRun; ++o) {
        const int t = j - o - kBloomHalo;  // this texel is tap t of output o
        if (t >= -kBloomHalo && t <= kBloomHalo) {
          const float kt = cBloomTaps[t < 0 ? -t : t];
          acc[o].x = fmaf(kt, v.x, acc[o].x);
          acc[o].y = fmaf(kt, v.y, acc[o].y);
          acc[o].z = fmaf(kt, v.z, acc[o].z);
        }
      }
    }
#pragma unroll
    for (int o = 0; o < kBlurRun; ++o) sH[r * kSHStride + c0 + o] = make_float4(acc[o].x, acc[o].y, acc[o].z, 1.f);
  }
  __syncthreads();
  constexpr int kYItems = kBloomTile * (kBloomTile / kBlurRun);
  for (int it = threadIdx.x; it < kYItems; it += blockDim.x) {
    const int c = it % kBloomTile, r0 = (it / kBloomTile) * kBlurRun;  // lanes on consecutive columns
    float3 acc[kBlurRun];
#pragma unroll
    for (int o = 0; o < kBlurRun; ++o) acc[o] = make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < kWin; ++j) {
      const float4 v = sH[(r0 + j) * kSHStride + c];
#pragma unroll
      for (int o = 0; o < kBlurRun; ++o) {
        const int t = j - o - kBloomHalo;
        if (t >= -kBloomHalo && t <= kBloomHalo) {
          const float kt = cBloomTaps[t < 0 ? -t : t];
          acc[o].x = fmaf(kt, v.x, acc[o].x);
          acc[o].y = fmaf(kt, v.y, acc[o].y);
          acc[o].z = fmaf(kt, v.z, acc[o].z);
        }
      }
    }
    const int x = x0 + c;
#pragma unroll
    for (int o = 0; o < kBlurRun; ++o) {
      const int y = y0 + r0 + o;
      if (x < w && y < h) P.B[k][(size_t)y * w + x] = make_float4(acc[o].x, acc[o].y, acc[o].z, 1.f);
    }
  }
  __syncthreads();
}

// One launch for the whole bloom, in three phases separated by grid
// barriers: the box levels (regions of the frame reduced in shared memory;
// levels past the seventh one grid-wide pass each), the blur of every tile of
// every level, then the composite of every pixel.
__device__ void bloom_body(const BloomParams &P);

// The kernel proper, then its exit: the last block to leave (every block
// leaves, barrier timeouts included) re-arms both counters for the next
// launch, so no launch needs a reset of its own.
__global__ void __launch_bounds__(kBloomThreads) bloom_kernel(const BloomParams P) {
  bloom_body(P);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(P.bar + 1, 1u) == gridDim.x - 1u) {
      atomicExch(P.bar, 0u);
      atomicExch(P.bar + 1, 0u);
    }
  }
}

__device__ void bloom_body(const BloomParams &P) {
  extern __shared__ float4 sb[];
  float4 *sD = sb;                              // kBloomSpan x kBloomSpan box texels (row stride kSDStride)
  float4 *sH = sb + kBloomSpan * kSDStride;     // kBloomSpan rows x kBloomTile blurred along x (stride kSHStride)
  unsigned phase = 0;
  if (P.n > 0) prefetch_region(P, blockIdx.x);        // read at once
  prefetch_comp_tile(P, blockIdx.x, kCompW, kCompH);  // read after the pyramid is built
  if (P.n > 0) {
    // ---- box levels 1..7 by regions.  Level 1 of a region (64 x 64 texels)
    // is built with a 3-texel halo at clamped coordinates straight from the
    // frame and blurred in place (its halo texels are those of the
    // neighbouring regions, recomputed); levels 2.. are reduced from its
    // interior in shared memory, alternately in sH and sD.
    const int nr = min(P.n, kBloomRegionLevels);
    const int rx = (P.w[1] + kBloomTile - 1) / kBloomTile, regions = rx * ((P.h[1] + kBloomTile - 1) / kBloomTile);
    for (int reg = blockIdx.x; reg < regions; reg += gridDim.x) {
      const int gx = reg % rx, gy = reg / rx;
      {
        const int w = P.w[1], h = P.h[1];
        if (reg + (int)gridDim.x < regions) prefetch_region(P, reg + gridDim.x);
        constexpr int kIt = (kBloomSpan * kBloomSpan + kBloomThreads - 1) / kBloomThreads;
#pragma unroll
        for (int j = 0; j < kIt; ++j) {
          const int i = threadIdx.x + j * kBloomThreads;
          if (i < kBloomSpan * kBloomSpan) {
            const int r = i / kBloomSpan, c = i - r * kBloomSpan;
            const int x = min(max(gx * kBloomTile + c - kBloomHalo, 0), w - 1);
            const int y = min(max(gy * kBloomTile + r - kBloomHalo, 0), h - 1);
            sD[r * kSDStride + c] = box_texel(P, 1, x, y);
          }
        }
        blur_staged(P, 1, gx * kBloomTile, gy * kBloomTile, sD, sH);  // ends with __syncthreads
      }
      // level k - 1 of the region: at src with row stride sstr (level 1: sD's interior)
      const float4 *src = sD + kBloomHalo * kSDStride + kBloomHalo;
      int sstr = kSDStride;
      for (int k = 2; k <= nr; ++k) {
        const int side = kBloomTile >> (k - 1);  // texels of level k per region side
        const int w = P.w[k], h = P.h[k];
        float4 *dst = (k & 1) ? sD : sH;
        for (int i = threadIdx.x; i < side * side; i += blockDim.x) {
          const int lx = i % side, ly = i / side;
          const int x = gx * side + lx, y = gy * side + ly;
          if (x >= w || y >= h) continue;
          // children in the previous level's region (side 2 * side)
          const int pw = P.w[k - 1], ph = P.h[k - 1];
          const int cx0 = min(2 * x, pw - 1) - 2 * gx * side, cx1 = min(2 * x + 1, pw - 1) - 2 * gx * side;
          const int cy0 = min(2 * y, ph - 1) - 2 * gy * side, cy1 = min(2 * y + 1, ph - 1) - 2 * gy * side;
          const float4 a = src[cy0 * sstr + cx0], b = src[cy0 * sstr + cx1];
          const float4 c = src[cy1 * sstr + cx0], d = src[cy1 * sstr + cx1];
          const float4 v = make_float4(0.25f * ((a.x + b.x) + (c.x + d.x)), 0.25f * ((a.y + b.y) + (c.y + d.y)),
                                       0.25f * ((a.z + b.z) + (c.z + d.z)), 1.f);
          dst[i] = v;
          P.D[k][(size_t)y * w + x] = v;
        }
        __syncthreads();
        src = dst;
        sstr = side;
      }
      __syncthreads();  // the region's shared buffers are free for the next one
    }
    // ---- levels past the region's depth: one grid-wide pass each
    for (int k = kBloomRegionLevels + 1; k <= P.n; ++k) {
      if (!grid_barrier(P, ++phase)) return;
      const long long nt = (long long)P.w[k] * P.h[k];
      for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / P.w[k]), x = (int)(i - (long long)y * P.w[k]);
        P.D[k][i] = box_texel(P, k, x, y);
      }
    }
    if (!grid_barrier(P, ++phase)) return;
    // ---- blur every 64x64 tile of levels 2.. (level 1 was blurred by regions)
    int tiles_before[kBloomMaxLevels + 2];
    tiles_before[1] = tiles_before[2] = 0;
    for (int k = 2; k <= P.n; ++k)
      tiles_before[k + 1] = tiles_before[k] + ((P.w[k] + kBloomTile - 1) / kBloomTile) * ((P.h[k] + kBloomTile - 1) / kBloomTile);
    for (int tile = blockIdx.x; tile < tiles_before[P.n + 1]; tile += gridDim.x) {
      int k = 2;
      while (tile >= tiles_before[k + 1]) ++k;
      const int t = tile - tiles_before[k], tx = (P.w[k] + kBloomTile - 1) / kBloomTile;
      blur_tile(P, k, (t % tx) * kBloomTile, (t / tx) * kBloomTile, sD, sH);
    }
    if (!grid_barrier(P, ++phase)) return;
  }
  // composite at full resolution, by tiles of kCompW x kCompH pixels.  The
  // bilinear lookup of level k at pixel (x, y) is a lerp along v of two
  // lerps along u; the lerps along u depend only on the pixel's column and
  // the texel row, so for each level the tile's texel rows are first
  // interpolated along u at every pixel column of the tile and staged in
  // shared memory (hrow), and each pixel then takes one lerp along v per
  // level from two staged values.  The arithmetic per pixel is exactly that
  // of interpolating alone.
  const int W = P.w[0], H = P.h[0];
  const int tcx = (W + kCompW - 1) / kCompW, ntiles = tcx * ((H + kCompH - 1) / kCompH);
  float4 *hrow = sb;
  // per tile row and level: tv, and the staged index of the row's upper texel row
  __shared__ float s_tv[kCompH][kBloomMaxLevels];  // [row][k - 1]
  __shared__ int s_ri[kCompH][kBloomMaxLevels];
  static_assert(kBloomThreads % kCompW == 0 && kBloomThreads / 32 == kCompH, "composite thread mapping");
  const int cc = threadIdx.x % kCompW, rstep = kBloomThreads / kCompW;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int X0 = (tile % tcx) * kCompW, Y0 = (tile / tcx) * kCompH;
    __syncthreads();  // the previous tile's staged rows have been read
    prefetch_comp_tile(P, tile + gridDim.x, kCompW, kCompH);
    int off = 0;
    for (int k = 1; k <= P.n; ++k) {
      const float s = __int_as_float((127 - k) << 23);  // 2^-k
      const int w = P.w[k], h = P.h[k];
      // texel rows jb .. jb + nr - 1 (contents clamped) serve the tile's pixel rows
      const int jb = (int)floorf(fmaf((float)Y0 + 0.5f, s, -0.5f));
      const int nr = (int)floorf(fmaf((float)(Y0 + kCompH - 1) + 0.5f, s, -0.5f)) - jb + 2;
      if ((int)threadIdx.x < kCompH) {
        const float v = fmaf((float)(Y0 + (int)threadIdx.x) + 0.5f, s, -0.5f);
        const float fv = floorf(v);
        s_tv[threadIdx.x][k - 1] = v - fv;
        s_ri[threadIdx.x][k - 1] = off + (int)fv - jb;
      }
      // this thread's column of the tile: its u, once per level
      const float u = fmaf((float)(X0 + cc) + 0.5f, s, -0.5f);
      const float fu = floorf(u), tu = u - fu;
      const int i0 = min(max((int)fu, 0), w - 1), i1 = min(max((int)fu + 1, 0), w - 1);
      const float4 *Bk = P.B[k];
      for (int r = threadIdx.x / kCompW; r < nr; r += rstep) {
        const float4 *row = Bk + (size_t)min(max(jb + r, 0), h - 1) * w;
        const float4 a = row[i0], b = row[i1];
        hrow[(off + r) * kCompW + cc] =
            make_float4(fmaf(tu, b.x - a.x, a.x), fmaf(tu, b.y - a.y, a.y), fmaf(tu, b.z - a.z, a.z), 0.f);
      }
      off += nr;
    }
    __syncthreads();
    // warp yy takes tile row yy, its lanes every 32nd column
    const int yy = threadIdx.x >> 5, y = Y0 + yy;
    if (y < H) {
      for (int c = threadIdx.x & 31; c < kCompW; c += 32) {
        const int x = X0 + c;
        if (x >= W) break;
        const long long p = (long long)y * W + x;
        const float4 cp = P.in[p];
        float r = P.wt[0] * cp.x, g = P.wt[0] * cp.y, b = P.wt[0] * cp.z;
        for (int k = 1; k <= P.n; ++k) {
          const float tv = s_tv[yy][k - 1];
          const int ri = s_ri[yy][k - 1];
          const float4 h0 = hrow[ri * kCompW + c], h1 = hrow[(ri + 1) * kCompW + c];
          const float wk = P.wt[k];
          r = fmaf(wk, fmaf(tv, h1.x - h0.x, h0.x), r);
          g = fmaf(wk, fmaf(tv, h1.y - h0.y, h0.y), g);
          b = fmaf(wk, fmaf(tv, h1.z - h0.z, h0.z), b);
        }
        P.out[p] = make_float4(r, g, b, 1.f);
      }
    }
  }
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
  // pyramid sizes and scratch: D_k and B_k per level
  int w[kBloomMaxLevels + 1], h[kBloomMaxLevels + 1];
  w[0] = width;
  h[0] = height;
  size_t texels = 0;
  for (int k = 1; k <= levels; ++k) {
    w[k] = (w[k - 1] + 1) / 2;
    h[k] = (h[k - 1] + 1) / 2;
    texels += 2 * (size_t)w[k] * h[k];
  }
  const size_t need = std::max<size_t>(texels, 1) * sizeof(float4);
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
  if (!ctx->bloom_bar) {
    // arrivals and blocks done: zero now; every launch leaves them zero again
    BH_CUDA(cudaMalloc((void **)&ctx->bloom_bar, 2 * sizeof(unsigned)));
    BH_CUDA(cudaMemsetAsync(ctx->bloom_bar, 0, 2 * sizeof(unsigned), s));
  }
  static bool taps_ready[64] = {false};
  static int coop_blocks[64] = {0};
  if (ctx->device < 64 && !taps_ready[ctx->device]) {
    double t[4], sum = 0.0;
    for (int i = 0; i < 4; ++i) {
      t[i] = exp(-0.5 * i * i);
      sum += (i == 0 ? 1.0 : 2.0) * t[i];
    }
    float tf[4];
    for (int i = 0; i < 4; ++i) tf[i] = (float)(t[i] / sum);
    BH_CUDA(cudaMemcpyToSymbol(cBloomTaps, tf, sizeof tf));
    static_assert(kBloomSmem >= sizeof(float4) * (kBloomTile * kBloomTile + kBloomTile * kBloomTile / 4),
                  "the region ping-pong buffers fit in the blur tile's shared memory");
    BH_CUDA(cudaFuncSetAttribute(bloom_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBloomSmem));
    int per_sm = 0;
    BH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bloom_kernel, kBloomThreads, kBloomSmem));
    coop_blocks[ctx->device] = std::max(1, std::min(per_sm, 2)) * ctx->sm_count;
    taps_ready[ctx->device] = true;
  }
  BloomParams P;
  memset(&P, 0, sizeof P);
  P.in = reinterpret_cast<const float4 *>(in_device);
  P.out = reinterpret_cast<float4 *>(out_device);
  P.n = levels;
  float4 *cur = reinterpret_cast<float4 *>(ctx->bloom_dev);
  for (int k = 0; k <= levels; ++k) {
    P.w[k] = w[k];
    P.h[k] = h[k];
    P.wt[k] = (float)weights[k];
    if (k == 0) {
      P.D[0] = const_cast<float4 *>(P.in);
    } else {
      P.D[k] = cur;
      P.B[k] = cur + (size_t)w[k] * h[k];
      cur = P.B[k] + (size_t)w[k] * h[k];
    }
  }
  P.bar = ctx->bloom_bar;
  P.status = ctx->status_dev;
  P.wait_ns = 100000000ull;  // 0.1 s: a level takes microseconds
  if (ctx->inject_bloom_barrier) {
    P.inject = 1;
    P.wait_ns = 2000000ull;  // 2 ms
    ctx->inject_bloom_barrier = 0;
  }
  void *args[] = {&P};
  BH_CUDA(cudaLaunchCooperativeKernel((const void *)bloom_kernel, dim3(coop_blocks[ctx->device]),
                                      dim3(kBloomThreads), args, kBloomSmem, s));
  count_launch(ctx, 1);
  BH_CUDA(cudaGetLastError());
  return BH_OK;
}
