// Star cube map build (Sec. 3.3.2 "Emitted light", Sec. 4).
//
// Each texel holds the colour SUM of the stars it contains and their
// luminance-weighted mean position inside the texel; a mip texel sums the
// colours of its 4 children and averages their positions weighted by Y
// (Sec. 3.3.2).  The paper derives the in-texel position from a hash of the
// colour; here it is stored explicitly as two unorm8 (reading C15).
//
// Determinism: colours are accumulated as 64-bit fixed point (2^-20 units)
// with integer atomics, so the sums do not depend on the order in which
// threads arrive; the position averages are evaluated in FP64 in one fixed
// child order with round-to-nearest intrinsics (this file is compiled
// without multiply-add contraction).  The build is therefore bit-for-bit
// reproducible.
//
// Layout: records of 4 x 16 bit -- X, Y, Z (half or bfloat16 of the colour
// sum divided by 4^level, so that coarse levels stay in range) and the
// position word (s in the low byte, t in the high byte) -- level-major, then
// face (+x,-x,+y,-y,+z,-z), row t, column s.
#include <cmath>

#include "bh_colour.cuh"
#include "bh_internal.cuh"

namespace bh {

constexpr double kXyzScale = 1048576.0;  // 2^20

__global__ void cube_cmf_kernel(double *cmf) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < kNLambda) dcmf(360.0 + 5.0 * k, cmf + 3 * k);
}

// GL major-axis face and face coordinates (sc, tc, |ma|).
__device__ __forceinline__ int cube_face_d(double x, double y, double z, double &sc, double &tc,
                                           double &ma) {
  double ax = fabs(x), ay = fabs(y), az = fabs(z);
  if (ax >= ay && ax >= az) {
    ma = ax;
    if (x >= 0.0) { sc = -z; tc = -y; return 0; }
    sc = z; tc = -y; return 1;
  }
  if (ay >= az) {
    ma = ay;
    if (y >= 0.0) { sc = x; tc = z; return 2; }
    sc = x; tc = -z; return 3;
  }
  ma = az;
  if (z >= 0.0) { sc = x; tc = -y; return 4; }
  sc = -x; tc = -y; return 5;
}

// One thread per star: emitted XYZ (black body of the star's temperature,
// scaled to its luminosity X+Y+Z, rounded to float), fixed-point sums into
// the level-0 texel that contains its direction.
__global__ void star_bin_kernel(const bh_star *stars, long long n, int N, const double *cmf,
                                unsigned long long *acc) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= n) return;
  bh_star st = stars[k];
  double b[3];
  dblackbody_xyz(cmf, (double)st.temp_K, b);
  double s = __dadd_rn(__dadd_rn(b[0], b[1]), b[2]);
  double lum = (double)st.lum;
  long long q[3];
  for (int c = 0; c < 3; ++c) {
    float xf = (float)__ddiv_rn(__dmul_rn(lum, b[c]), s);
    q[c] = __double2ll_rn(__dmul_rn((double)xf, kXyzScale));
  }
  double sc, tc, ma;
  int f = cube_face_d((double)st.dir[0], (double)st.dir[1], (double)st.dir[2], sc, tc, ma);
  double S = __dmul_rn(__dmul_rn(__dadd_rn(__ddiv_rn(sc, ma), 1.0), 0.5), (double)N);
  double T = __dmul_rn(__dmul_rn(__dadd_rn(__ddiv_rn(tc, ma), 1.0), 0.5), (double)N);
  int i = (int)floor(S), j = (int)floor(T);
  i = min(max(i, 0), N - 1);
  j = min(max(j, 0), N - 1);
  long long s16 = (long long)floor(__dmul_rn(__dadd_rn(S, -(double)i), 65536.0));
  long long t16 = (long long)floor(__dmul_rn(__dadd_rn(T, -(double)j), 65536.0));
  s16 = min(max(s16, 0LL), 65535LL);
  t16 = min(max(t16, 0LL), 65535LL);
  unsigned long long *a = acc + (((long long)f * N + j) * N + i) * 5;
  atomicAdd(a + 0, (unsigned long long)q[0]);
  atomicAdd(a + 1, (unsigned long long)q[1]);
  atomicAdd(a + 2, (unsigned long long)q[2]);
  atomicAdd(a + 3, (unsigned long long)(q[1] * s16));
  atomicAdd(a + 4, (unsigned long long)(q[1] * t16));
}

__device__ __forceinline__ unsigned short enc16(double v, int dtype) {
  if (dtype == BH_BF16) return __bfloat16_as_ushort(__double2bfloat16(v));
  return __half_as_ushort(__double2half(fmin(v, 65504.0)));
}

// Level-0 records from the accumulators (X, Y, Z, Y*s16, Y*t16 per texel).
__global__ void level0_kernel(const unsigned long long *acc, long long ntex, int dtype,
                              uint2 *rec, long long *sums) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= ntex) return;
  const long long *a = (const long long *)(acc + t * 5);
  long long x = a[0], y = a[1], z = a[2];
  int ps = 128, pt = 128;
  if (y > 0) {
    double fs = __ddiv_rn(__dadd_rn(__ddiv_rn((double)a[3], (double)y), 0.5), 65536.0);
    double ft = __ddiv_rn(__dadd_rn(__ddiv_rn((double)a[4], (double)y), 0.5), 65536.0);
    ps = min((int)floor(__dmul_rn(fs, 256.0)), 255);
    pt = min((int)floor(__dmul_rn(ft, 256.0)), 255);
  }
  unsigned short X = enc16((double)x / kXyzScale, dtype), Y = enc16((double)y / kXyzScale, dtype),
                 Z = enc16((double)z / kXyzScale, dtype);
  rec[t] = make_uint2((unsigned)X | ((unsigned)Y << 16), (unsigned)Z | ((unsigned)(ps | (pt << 8)) << 16));
  sums[t * 3 + 0] = x;
  sums[t * 3 + 1] = y;
  sums[t * 3 + 2] = z;
}

// Mip level L from level L-1: colour sums of the 4 children (exact), and the
// Y-weighted mean of their positions, children in the order (a,b) = (0,0),
// (1,0), (0,1), (1,1) with a the column and b the row offset.
__global__ void mip_kernel(const long long *psums, const uint2 *prec, int Np, int L, int dtype,
                           long long *csums, uint2 *crec) {
  int Nc = Np >> 1;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long ntc = 6LL * Nc * Nc;
  if (t >= ntc) return;
  int f = (int)(t / ((long long)Nc * Nc));
  long long rem = t % ((long long)Nc * Nc);
  int j = (int)(rem / Nc), i = (int)(rem % Nc);
  long long sx = 0, sy = 0, sz = 0;
  double ns = 0.0, nt = 0.0;
  for (int b = 0; b < 2; ++b)
    for (int a = 0; a < 2; ++a) {
      long long ct = ((long long)f * Np + 2 * j + b) * Np + 2 * i + a;
      long long cy = psums[ct * 3 + 1];
      sx += psums[ct * 3 + 0];
      sy += cy;
      sz += psums[ct * 3 + 2];
      unsigned pp = prec[ct].y >> 16;
      double cs = __ddiv_rn((double)(pp & 255) + 0.5, 256.0), cq = __ddiv_rn((double)(pp >> 8) + 0.5, 256.0);
      ns = __dadd_rn(ns, __dmul_rn((double)cy, __dmul_rn(__dadd_rn((double)a, cs), 0.5)));
      nt = __dadd_rn(nt, __dmul_rn((double)cy, __dmul_rn(__dadd_rn((double)b, cq), 0.5)));
    }
  int ps = 128, pt = 128;
  if (sy > 0) {
    ps = min((int)floor(__dmul_rn(__ddiv_rn(ns, (double)sy), 256.0)), 255);
    pt = min((int)floor(__dmul_rn(__ddiv_rn(nt, (double)sy), 256.0)), 255);
  }
  double scale = ldexp(kXyzScale, 2 * L);
  unsigned short X = enc16((double)sx / scale, dtype), Y = enc16((double)sy / scale, dtype),
                 Z = enc16((double)sz / scale, dtype);
  crec[t] = make_uint2((unsigned)X | ((unsigned)Y << 16), (unsigned)Z | ((unsigned)(ps | (pt << 8)) << 16));
  csums[t * 3 + 0] = sx;
  csums[t * 3 + 1] = sy;
  csums[t * 3 + 2] = sz;
}

// Occupancy bits of one level: a texel is occupied when its colour is not
// zero.  The renderer walks only the occupied texels of a footprint row.
__global__ void occupancy_kernel(const uint2 *rec, int NL, unsigned *mask) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int wpr = (NL + 31) / 32;
  long long nw = 6LL * NL * wpr;
  if (t >= nw) return;
  long long row = t / wpr;  // face * NL + j
  int w = (int)(t % wpr);
  const uint2 *r = rec + row * NL;
  unsigned bits = 0;
  for (int b = 0; b < 32; ++b) {
    int i = 32 * w + b;
    if (i >= NL) break;
    uint2 v = r[i];
    if ((v.x | (v.y & 0xffffu)) != 0u) bits |= 1u << b;
  }
  mask[t] = bits;
}

}  // namespace bh

using namespace bh;

extern "C" long long bh_cubemap_records(int N) {
  if (N < 1 || (N & (N - 1))) return 0;
  return cube_level_offset(N, cube_levels(N));
}

extern "C" bh_status bh_build_star_cubemap(bh_ctx *ctx, const bh_star *stars, long long n, int N,
                                           bh_dtype storage, int on_device, void *stream,
                                           bh_cubemap **out) {
  TraceRange trace_("bh_build_star_cubemap");
  if (!ctx || !out || (n > 0 && !stars)) { set_error("bh_build_star_cubemap: NULL argument"); return BH_ERR_INVALID_ARG; }
  *out = nullptr;
  if (n < 0 || N < 1 || N > 8192 || (N & (N - 1))) {
    set_error("bh_build_star_cubemap: n = %lld, face_size = %d (power of two, 1..8192)", n, N);
    return BH_ERR_INVALID_ARG;
  }
  if (storage != BH_F16 && storage != BH_BF16) {
    set_error("bh_build_star_cubemap: storage must be BH_F16 or BH_BF16");
    return BH_ERR_INVALID_ARG;
  }
  BH_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  bh_cubemap *c = new bh_cubemap();
  c->ctx = ctx;
  c->n = N;
  c->levels = cube_levels(N);
  c->storage = storage;
  c->records = bh_cubemap_records(N);
  long long nt0 = 6LL * N * N;
  long long nt1 = N > 1 ? 6LL * (N / 2) * (N / 2) : 1;
  unsigned long long *acc = nullptr;
  long long *sums0 = nullptr, *sums1 = nullptr;
  double *cmf = nullptr;
  bh_star *dstars = nullptr;
  c->mask_words = mask_level_offset(N, c->levels);
  cudaError_t e = cudaMalloc((void **)&c->rec, sizeof(uint2) * c->records);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->mask, sizeof(unsigned) * c->mask_words);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&acc, sizeof(unsigned long long) * 5 * nt0, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&sums0, sizeof(long long) * 3 * nt0, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&sums1, sizeof(long long) * 3 * nt1, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&cmf, sizeof(double) * 3 * kNLambda, s);
  const bh_star *src = stars;
  if (e == cudaSuccess && n > 0 && !on_device) {
    e = cudaMallocAsync((void **)&dstars, sizeof(bh_star) * n, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dstars, stars, sizeof(bh_star) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host list may be freed on return
    src = dstars;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 5 * nt0, s);
  if (e == cudaSuccess) {
    cube_cmf_kernel<<<1, 128, 0, s>>>(cmf);
    if (n > 0) star_bin_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, n, N, cmf, acc);
    level0_kernel<<<(unsigned)((nt0 + 255) / 256), 256, 0, s>>>(acc, nt0, storage, c->rec, sums0);
    count_launch(ctx, n > 0 ? 3 : 2);
    long long *ps = sums0, *cs = sums1;
    for (int L = 1; L < c->levels; ++L) {
      int Np = N >> (L - 1);
      long long ntc = 6LL * (Np / 2) * (Np / 2);
      mip_kernel<<<(unsigned)((ntc + 255) / 256), 256, 0, s>>>(
          ps, c->rec + cube_level_offset(N, L - 1), Np, L, storage, cs, c->rec + cube_level_offset(N, L));
      count_launch(ctx);
      long long *tmp = ps;
      ps = cs;
      cs = tmp;
    }
    for (int L = 0; L < c->levels; ++L) {
      int NL = N >> L;
      long long nw = 6LL * NL * ((NL + 31) / 32);
      occupancy_kernel<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(c->rec + cube_level_offset(N, L), NL,
                                                                   c->mask + mask_level_offset(N, L));
      count_launch(ctx);
    }
    e = cudaGetLastError();
  }
  cudaFreeAsync(acc, s);
  cudaFreeAsync(sums0, s);
  cudaFreeAsync(sums1, s);
  cudaFreeAsync(cmf, s);
  if (dstars) cudaFreeAsync(dstars, s);
  if (e != cudaSuccess) {
    bh_cubemap_free(c);
    return cuda_fail(e, "bh_build_star_cubemap");
  }
  *out = c;
  return BH_OK;
}

extern "C" bh_status bh_cubemap_copy_out(const bh_cubemap *c, uint16_t *h, long long n) {
  if (!c || !h) { set_error("bh_cubemap_copy_out: NULL argument"); return BH_ERR_INVALID_ARG; }
  if (n != c->records) {
    set_error("bh_cubemap_copy_out: %lld records requested, map has %lld", n, c->records);
    return BH_ERR_INVALID_ARG;
  }
  BH_CUDA(cudaSetDevice(c->ctx->device));
  BH_CUDA(cudaDeviceSynchronize());
  BH_CUDA(cudaMemcpy(h, c->rec, sizeof(uint2) * n, cudaMemcpyDeviceToHost));
  return BH_OK;
}

namespace bh {
// An empty map of face size N (all levels and the occupancy mask allocated,
// contents undefined), for loading from a checkpoint.
bh_status cubemap_alloc_public(bh_ctx *ctx, int N, bh_dtype storage, bh_cubemap **out) {
  bh_cubemap *c = new bh_cubemap();
  c->ctx = ctx;
  c->n = N;
  c->levels = cube_levels(N);
  c->storage = storage;
  c->records = bh_cubemap_records(N);
  c->mask_words = mask_level_offset(N, c->levels);
  cudaError_t e = cudaMalloc((void **)&c->rec, sizeof(uint2) * c->records);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->mask, sizeof(unsigned) * c->mask_words);
  if (e != cudaSuccess) {
    cudaFree(c->rec);
    cudaFree(c->mask);
    delete c;
    return cuda_fail(e, "cube map allocation");
  }
  *out = c;
  return BH_OK;
}
}  // namespace bh

extern "C" void bh_cubemap_free(bh_cubemap *c) {
  if (!c) return;
  cudaSetDevice(c->ctx->device);
  cudaDeviceSynchronize();
  cudaFree(c->rec);
  cudaFree(c->mask);
  delete c;
}

// ---------------------------------------------------------------------------
// Allocation-free cube-map build
//
// For callers that may not allocate device memory themselves: applications
// that hand every byte of device memory to their own pool or arena (engines,
// plug-in hosts with a fixed memory budget), and real-time threads that must
// not call cudaMalloc/cudaFree, which can synchronise the device and take an
// unbounded time.  The scratch lives in one file-scope device array, sized for
// faces of up to kNoAllocMaxFace texels; every GPU that loads this library
// holds it (about 6.9 MB) until the process exits.
// ---------------------------------------------------------------------------
namespace bh {

constexpr int kNoAllocMaxFace = 128;
constexpr long long kNoAllocTexels0 = 6LL * kNoAllocMaxFace * kNoAllocMaxFace;
constexpr long long kNoAllocTexels1 = kNoAllocTexels0 / 4;
// accumulators (5 x 64 bit per level-0 texel), level sums (3 x 64 bit per
// texel of two consecutive levels), matching functions (3 x 95 doubles)
constexpr size_t kNoAllocScratchWords = 5 * kNoAllocTexels0 + 3 * kNoAllocTexels0 + 3 * kNoAllocTexels1 + 3 * kNLambda;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocScratchWords];

// Device address of the scratch array on the current device (the host-side
// name of a __device__ array is not a device address).  Looked up on every
// call that is not being captured into a CUDA graph, so that a device or
// primary-context reset between calls cannot leave a stale address behind;
// a call under stream capture uses the address its device's last uncaptured
// call found (cudaGetSymbolAddress may load the module, which capture forbids).
static bh_status noalloc_scratch(int device, bool capturing, unsigned long long **out) {
  static std::mutex mu;
  static unsigned long long *addr[64] = {nullptr};
  if (device < 0 || device >= 64) {
    set_error("bh_build_star_cubemap_noalloc: device %d out of range", device);
    return BH_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!capturing) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "bh_build_star_cubemap_noalloc: cudaGetSymbolAddress");
    addr[device] = static_cast<unsigned long long *>(p);
  } else if (!addr[device]) {
    set_error("bh_build_star_cubemap_noalloc: the first call on device %d is under stream capture; "
              "make one call before capturing", device);
    return BH_ERR_INVALID_ARG;
  }
  *out = addr[device];
  return BH_OK;
}

}  // namespace bh

extern "C" bh_status bh_build_star_cubemap_noalloc(const bh_star *stars_device, long long n,
                                                   int N, bh_dtype storage, uint16_t *records_device,
                                                   void *stream) {
  if ((n > 0 && !stars_device) || !records_device) {
    set_error("bh_build_star_cubemap_noalloc: NULL argument");
    return BH_ERR_INVALID_ARG;
  }
  if (N < 1 || (N & (N - 1)) || N > kNoAllocMaxFace) {
    set_error("bh_build_star_cubemap_noalloc: face_size %d must be a power of two <= %d (the size of "
              "its static scratch)", N, kNoAllocMaxFace);
    return BH_ERR_INVALID_ARG;
  }
  if (n < 0 || (storage != BH_F16 && storage != BH_BF16) || ((uintptr_t)records_device & 7)) {
    set_error("bh_build_star_cubemap_noalloc: n >= 0, storage BH_F16/BH_BF16 and 8-byte aligned records required");
    return BH_ERR_INVALID_ARG;
  }
  int dev = 0;
  BH_CUDA(cudaGetDevice(&dev));
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  BH_CUDA(cudaStreamIsCapturing(s, &cap));
  unsigned long long *scratch = nullptr;
  bh_status st = noalloc_scratch(dev, cap != cudaStreamCaptureStatusNone, &scratch);
  if (st) return st;
  long long nt0 = 6LL * N * N;
  unsigned long long *acc = scratch;
  long long *sums0 = reinterpret_cast<long long *>(scratch + 5 * kNoAllocTexels0);
  long long *sums1 = sums0 + 3 * kNoAllocTexels0;
  double *cmf = reinterpret_cast<double *>(sums1 + 3 * kNoAllocTexels1);
  uint2 *rec = reinterpret_cast<uint2 *>(records_device);
  int levels = cube_levels(N);
  // the array keeps the previous call's contents: the accumulators must start at zero
  BH_CUDA(cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 5 * nt0, s));
  cube_cmf_kernel<<<1, 128, 0, s>>>(cmf);
  if (n > 0) star_bin_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(stars_device, n, N, cmf, acc);
  level0_kernel<<<(unsigned)((nt0 + 255) / 256), 256, 0, s>>>(acc, nt0, storage, rec, sums0);
  long long *ps = sums0, *cs = sums1;
  for (int L = 1; L < levels; ++L) {
    int Np = N >> (L - 1);
    long long ntc = 6LL * (Np / 2) * (Np / 2);
    mip_kernel<<<(unsigned)((ntc + 255) / 256), 256, 0, s>>>(ps, rec + cube_level_offset(N, L - 1), Np, L,
                                                              storage, cs, rec + cube_level_offset(N, L));
    long long *tmp = ps;
    ps = cs;
    cs = tmp;
  }
  BH_CUDA(cudaGetLastError());
  return BH_OK;
}
