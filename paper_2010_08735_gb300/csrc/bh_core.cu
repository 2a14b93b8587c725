// libbh core: context, errors, and the GPU precompute of the tables.
//
//  * D(e,u) and U(e,phi) (Algorithm 1 PRECOMPUTE, Appendix A): instead of
//    Euler steps along each e row, every texel is an independent FP64
//    quadrature of the ray equation's first integral
//        phi(u) = int_0^u du' / sqrt(P(u')),  P(u) = e^2 - u^2 (1 - u)
//    (Eq. rayequation), after a substitution that removes the apsis
//    singularity and the near-double root at the photon sphere:
//      e^2 < mu:  P = (u_a - u) q(u), u = u_a - w^2, q = A + B w^2 - w^4,
//                 and near criticality w = sqrt(A/B) sinh t;
//      e^2 > mu:  P = (e^2 - mu) + v^2 (v + 1), v = u - 2/3 = sqrt(e^2-mu) sinh t.
//    Delta = phi - atan2(u, du/dphi) (Algorithm 1).  U inverts phi(u) by
//    safeguarded Newton iterations on the same quadrature, using the apsis
//    reflection phi -> 2 phi_a - phi past the apsis (Sec. 3.3.1).
//  * The colour tables (Sec. 3.4.2): C(xy, D) and the disc black-body table.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "bh_colour.cuh"
#include "bh_internal.cuh"

namespace bh {

static thread_local std::string g_last_error;

void set_error(const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

bh_status cuda_fail(cudaError_t e, const char *what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? BH_ERR_OOM : BH_ERR_CUDA;
}

void count_launch(bh_ctx *ctx, int n) { ctx->launches.fetch_add(n, std::memory_order_relaxed); }

bh_status check_status(bh_ctx *ctx, cudaStream_t s) {
  unsigned st = 0;
  BH_CUDA(cudaMemcpyAsync(&st, ctx->status_dev, sizeof st, cudaMemcpyDeviceToHost, s));
  BH_CUDA(cudaStreamSynchronize(s));
  if (st) {
    set_error("kernel status word 0x%x (%s%s%s)", st, (st & kStatusMbarTimeout) ? "table load timed out " : "",
              (st & kStatusBarrierTimeout) ? "grid barrier timed out " : "",
              (st & kStatusBadIndex) ? "index out of range" : "");
    BH_CUDA(cudaMemsetAsync(ctx->status_dev, 0, sizeof(unsigned), s));
    return (st & (kStatusMbarTimeout | kStatusBarrierTimeout)) ? BH_ERR_TIMEOUT : BH_ERR_DEVICE_STATUS;
  }
  return BH_OK;
}

// ---------------------------------------------------------------------------
// Gauss-Legendre nodes (16 points) computed once on the host by Newton's
// method on P_16 with its three-term recurrence.
// ---------------------------------------------------------------------------
constexpr int kGL = 16;
__constant__ double cGLx[kGL], cGLw[kGL];

static void gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(kPi * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// ---------------------------------------------------------------------------
// Device quadrature
// ---------------------------------------------------------------------------
struct Apsis {
  double ua, A, B;  // u_a (Eq. uapsis); q(w) = A + B w^2 - w^4
};

// From eta = 1 - e^2/mu in (0,1]: u_a = 1/3 + 2/3 sin(asin(2e^2/mu - 1)/3)
// with asin(1 - 2 eta) = pi/2 - 2 asin(sqrt(eta)), and
// A = u_a (2 - 3u_a) = 4 u_a cos(pi/12 + th/2) sin(asin(sqrt(eta))/3),
// B = 3 u_a - 1 = 2 sin(th), th = asin(2e^2/mu - 1)/3 -- free of cancellation
// near the photon sphere.
__device__ Apsis apsis_of_eta(double eta) {
  double s = asin(sqrt(eta));
  double th = (0.5 * kPi - 2.0 * s) / 3.0;
  Apsis a;
  a.ua = 1.0 / 3.0 + 2.0 / 3.0 * sin(th);
  a.A = 4.0 * a.ua * cos(kPi / 12.0 + 0.5 * th) * sin(s / 3.0);
  a.B = 2.0 * sin(th);
  return a;
}

__device__ __forceinline__ double qw(const Apsis &a, double w) {
  double w2 = w * w;
  return a.A + a.B * w2 - w2 * w2;
}

// The regularised time R = t + 1/u - ln(u/(1-u)) (reading C5) obeys
// dR/dphi = 1/(e + du/dphi), so every angle quadrature below has a time twin
// (TIME = true) whose integrand carries the extra factor 1/(e + du/dphi).

// int_{w0}^{w1} 2 dw / sqrt(q(w)) [/(e + w sqrt(q))], composite Gauss-Legendre
template <bool TIME>
__device__ double quad_w(const Apsis &a, double e, double w0, double w1, int panels) {
  double h = (w1 - w0) / panels, s = 0.0;
  for (int p = 0; p < panels; ++p) {
    double c = w0 + (p + 0.5) * h, r = 0.5 * h;
    for (int k = 0; k < kGL; ++k) {
      double w = c + r * cGLx[k], q = qw(a, w), rq = rsqrt(q);
      double f = 2.0 * rq;
      if (TIME) f /= e + w * q * rq;
      s += cGLw[k] * r * f;
    }
  }
  return s;
}

// same integral in t, w = c sinh t, c = sqrt(A/B): integrand 2 c cosh t / sqrt(q)
template <bool TIME>
__device__ double quad_t_scatter(const Apsis &a, double e, double c, double t0, double t1, int panels) {
  double h = (t1 - t0) / panels, s = 0.0;
  for (int p = 0; p < panels; ++p) {
    double m = t0 + (p + 0.5) * h, r = 0.5 * h;
    for (int k = 0; k < kGL; ++k) {
      double t = m + r * cGLx[k];
      double sh = sinh(t), w = c * sh, q = qw(a, w), rq = rsqrt(q);
      double f = 2.0 * c * sqrt(1.0 + sh * sh) * rq;
      if (TIME) f /= e + w * q * rq;
      s += cGLw[k] * r * f;
    }
  }
  return s;
}

// From infinity to u = u_a - w0^2: the angle (TIME = false) or the
// regularised time (TIME = true), int_{w0}^{sqrt(u_a)} in w.
template <bool TIME>
__device__ double scatter_integral(const Apsis &a, double e, double w0) {
  double w1 = sqrt(a.ua);
  if (a.ua > 0.6) {
    double c = sqrt(a.A / a.B);
    double wm = fmax(w0, fmin(w1, 0.35));
    return quad_t_scatter<TIME>(a, e, c, asinh(w0 / c), asinh(wm / c), 6) + quad_w<TIME>(a, e, wm, w1, 4);
  }
  return quad_w<TIME>(a, e, w0, w1, 4);
}

// Plunging rays: int_{ta}^{tb} dt / sqrt(1 + v tanh^2 t), v = se sinh t
// (du/dphi = se cosh t sqrt(1 + v tanh^2 t)).
template <bool TIME>
__device__ double plunge_integral(double se, double e, double ta, double tb) {
  const int panels = 6;
  double h = (tb - ta) / panels, s = 0.0;
  for (int p = 0; p < panels; ++p) {
    double m = ta + (p + 0.5) * h, r = 0.5 * h;
    for (int k = 0; k < kGL; ++k) {
      double t = m + r * cGLx[k];
      double th = tanh(t), g = 1.0 + se * sinh(t) * th * th, rg = rsqrt(g);
      double f = rg;
      if (TIME) f /= e + se * cosh(t) * g * rg;
      s += cGLw[k] * r * f;
    }
  }
  return s;
}

template <typename T>
__device__ __forceinline__ T to_storage(double v);
template <>
__device__ __forceinline__ float to_storage<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ __half to_storage<__half>(double v) { return __double2half(v); }

// D(e,u) per texel: texel (i,j) holds the Appendix A coordinates
// x = i/(n-1), y = j/(n-1) (reading C3).
__global__ void precompute_D_kernel(int n, double *D64, double *DT64, float *DTs) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y;
  if (i >= n || j >= n) return;
  double x = (double)i / (n - 1), y = (double)j / (n - 1);
  double Delta, R;
  if (i < n / 2) {
    // x = 1/2 - sqrt(-log(1 - e^2/mu)/50): eta = 1 - e^2/mu = exp(-50 (1/2 - x)^2)
    double a = 0.5 - x;
    double eta = exp(-50.0 * a * a);
    double e = sqrt(-kMu * expm1(-50.0 * a * a));
    Apsis ap = apsis_of_eta(eta);
    double w0 = sqrt(ap.ua) * (1.0 - y);  // y = 1 - sqrt(1 - u/u_a)
    double u = ap.ua - w0 * w0;
    double phi = scatter_integral<false>(ap, e, w0);
    double udot = w0 * sqrt(qw(ap, w0));
    Delta = phi - atan2(u, udot);
    R = scatter_integral<true>(ap, e, w0);
  } else {
    // x = 1/2 + sqrt(-log(1 - mu/e^2)/50): 1 - mu/e^2 = exp(-50 (x - 1/2)^2)
    double a = x - 0.5;
    double g = exp(-50.0 * a * a);
    double e2 = kMu / (-expm1(-50.0 * a * a));
    double em = e2 * g;  // e^2 - mu
    double se = sqrt(em);
    const double r23 = sqrt(2.0 / 3.0), r13 = sqrt(1.0 / 3.0);
    double z = y * (r23 + r13) - r23;
    double v = z >= 0.0 ? z * z : -z * z;  // u - 2/3
    double u = 2.0 / 3.0 + v;
    double ta = asinh(-2.0 / 3.0 / se), tb = asinh(v / se);
    double phi = plunge_integral<false>(se, 0.0, ta, tb);
    double udot = sqrt(em + v * v * (v + 1.0));
    Delta = phi - atan2(u, udot);
    R = plunge_integral<true>(se, sqrt(e2), ta, tb);
  }
  D64[(size_t)j * n + i] = Delta;
  DT64[(size_t)j * n + i] = R;
  DTs[(size_t)j * n + i] = (float)R;
}

// Warp-cooperative forms of the quadratures above: the 32 lanes of a warp
// share the Gauss-Legendre nodes of one integral and sum them with shuffles,
// so that the Newton iterations of one U texel run on a whole warp.
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <bool TIME>
__device__ double warp_quad_w(const Apsis &a, double e, double w0, double w1, int panels, int lane) {
  double h = (w1 - w0) / panels, s = 0.0;
  for (int idx = lane; idx < panels * kGL; idx += 32) {
    int p = idx / kGL, k = idx % kGL;
    double c = w0 + (p + 0.5) * h, r = 0.5 * h;
    double w = c + r * cGLx[k], q = qw(a, w), rq = rsqrt(q);
    double f = 2.0 * rq;
    if (TIME) f /= e + w * q * rq;
    s += cGLw[k] * r * f;
  }
  return warp_sum(s);
}

template <bool TIME>
__device__ double warp_quad_t_scatter(const Apsis &a, double e, double c, double t0, double t1, int panels,
                                      int lane) {
  double h = (t1 - t0) / panels, s = 0.0;
  for (int idx = lane; idx < panels * kGL; idx += 32) {
    int p = idx / kGL, k = idx % kGL;
    double m = t0 + (p + 0.5) * h, r = 0.5 * h;
    double sh = sinh(m + r * cGLx[k]), w = c * sh, q = qw(a, w), rq = rsqrt(q);
    double f = 2.0 * c * sqrt(1.0 + sh * sh) * rq;
    if (TIME) f /= e + w * q * rq;
    s += cGLw[k] * r * f;
  }
  return warp_sum(s);
}

template <bool TIME>
__device__ double warp_scatter_integral(const Apsis &a, double e, double w0, int lane) {
  double w1 = sqrt(a.ua);
  if (a.ua > 0.6) {
    double c = sqrt(a.A / a.B);
    double wm = fmax(w0, fmin(w1, 0.35));
    return warp_quad_t_scatter<TIME>(a, e, c, asinh(w0 / c), asinh(wm / c), 6, lane) +
           warp_quad_w<TIME>(a, e, wm, w1, 4, lane);
  }
  return warp_quad_w<TIME>(a, e, w0, w1, 4, lane);
}

template <bool TIME>
__device__ double warp_plunge_integral(double se, double e, double ta, double tb, int lane) {
  const int panels = 6;
  double h = (tb - ta) / panels, s = 0.0;
  for (int idx = lane; idx < panels * kGL; idx += 32) {
    int p = idx / kGL, k = idx % kGL;
    double t = ta + (p + 0.5) * h + 0.5 * h * cGLx[k];
    double th = tanh(t), g = 1.0 + se * sinh(t) * th * th, rg = rsqrt(g);
    double f = rg;
    if (TIME) f /= e + se * cosh(t) * g * rg;
    s += cGLw[k] * 0.5 * h * f;
  }
  return warp_sum(s);
}

// U(e,phi) per texel, one warp per texel: x = 1/(1 + 6 e^2),
// y = (phi/3)(1 + 6 e^3)/(1 + e^2).  UT gets the regularised time at the
// same point; past the apsis it follows from the time symmetry of the ray
// about its apsis, t(phi) = 2 t_a - t(2 phi_a - phi).
template <typename T>
__global__ void precompute_U_kernel(int ne, int nphi, double *U64, T *Us, double *UT64, float *UTs) {
  int lane = threadIdx.x & 31;
  int texel = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (texel >= ne * nphi) return;  // whole warps leave together
  int i = texel % ne, j = texel / ne;
  double u, R = 0.0;  // R = 0 where there is no ray or it was captured
  if (i == 0) {
    u = j == 0 ? 0.0 : 1.0;  // e -> infinity: radial ray, captured at once
  } else {
    double x = (double)i / (ne - 1), y = (double)j / (nphi - 1);
    double e2 = (1.0 / x - 1.0) / 6.0;
    double e = sqrt(e2);
    double phi = 3.0 * y * (1.0 + e2) / (1.0 + 6.0 * e2 * e);
    if (e2 <= 0.0 || phi <= 0.0) {
      u = 0.0;
    } else if (e2 < kMu) {
      Apsis ap = apsis_of_eta(1.0 - e2 / kMu);
      double phia = warp_scatter_integral<false>(ap, e, 0.0, lane);
      bool past = phi > phia;
      if (past) phi = 2.0 * phia - phi;  // past the apsis: reflection
      double lo = 0.0, hi = sqrt(ap.ua), w = 0.5 * (lo + hi);
      for (int it = 0; it < 80; ++it) {
        double F = warp_scatter_integral<false>(ap, e, w, lane) - phi;  // decreasing in w
        if (F > 0.0) lo = w; else hi = w;
        double dF = -2.0 * rsqrt(qw(ap, w));
        double wn = w - F / dF;
        if (!(wn > lo && wn < hi)) wn = 0.5 * (lo + hi);
        if (fabs(wn - w) < 1e-16) { w = wn; break; }
        w = wn;
      }
      u = ap.ua - w * w;
      R = warp_scatter_integral<true>(ap, e, w, lane);
      if (past) {
        if (u > 0.0) {
          double Ra = warp_scatter_integral<true>(ap, e, 0.0, lane);
          double l = 2.0 * log(u / (1.0 - u)), la = 2.0 * log(ap.ua / (1.0 - ap.ua));
          R = 2.0 * Ra - 2.0 / ap.ua + la - R + 2.0 / u - l;
        } else {
          R = 0.0;  // back at infinity: no texel of the mapping gets here
        }
      }
    } else {
      double se = sqrt(e2 - kMu);
      double ta = asinh(-2.0 / 3.0 / se), tb = asinh(1.0 / 3.0 / se);
      if (phi >= warp_plunge_integral<false>(se, e, ta, tb, lane)) {
        u = 1.0;  // reached the horizon before phi (reading C7)
      } else {
        double lo = ta, hi = tb, t = 0.5 * (lo + hi);
        for (int it = 0; it < 80; ++it) {
          double F = warp_plunge_integral<false>(se, e, ta, t, lane) - phi;  // increasing in t
          if (F < 0.0) lo = t; else hi = t;
          double th = tanh(t);
          double dF = rsqrt(1.0 + se * sinh(t) * th * th);
          double tn = t - F / dF;
          if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
          if (fabs(tn - t) < 1e-16) { t = tn; break; }
          t = tn;
        }
        u = 2.0 / 3.0 + se * sinh(t);
        R = warp_plunge_integral<true>(se, e, ta, t, lane);
      }
    }
  }
  if (lane == 0) {
    U64[(size_t)j * ne + i] = u;
    Us[(size_t)j * ne + i] = to_storage<T>(u);
    UT64[(size_t)j * ne + i] = R;
    UTs[(size_t)j * ne + i] = (float)R;
  }
}

// The render copy of D, row-paired: texel (j, i) holds D(j, i) and
// D(min(j+1, n-1), i) side by side, so a bilinear lookup is two loads.
template <typename T>
__global__ void pair_d_kernel(int n, const double *D64, T *Dp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= n || j >= n) return;
  const size_t o = (size_t)j * n + i;
  Dp[2 * o] = to_storage<T>(D64[o]);
  Dp[2 * o + 1] = to_storage<T>(D64[(size_t)min(j + 1, n - 1) * n + i]);
}

template <typename T>
__global__ void convert_kernel(const double *src, T *dst, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = to_storage<T>(src[i]);
}

// ---------------------------------------------------------------------------
// Colour tables (Sec. 3.4.2, reading C14)
// ---------------------------------------------------------------------------
__global__ void cmf_kernel(double *cmf) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < kNLambda) dcmf(360.0 + 5.0 * k, cmf + 3 * k);
}

__device__ __forceinline__ void uv1960(const double *xyz, double *uv) {
  double den = __dadd_rn(__dadd_rn(xyz[0], __dmul_rn(15.0, xyz[1])), __dmul_rn(3.0, xyz[2]));
  uv[0] = __ddiv_rn(__dmul_rn(4.0, xyz[0]), den);
  uv[1] = __ddiv_rn(__dmul_rn(6.0, xyz[1]), den);
}

__global__ void locus_kernel(const double *cmf, double *locus) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= kNLocus) return;
  double xyz[3];
  dblackbody_xyz(cmf, 1000.0 * pow(40.0, m / 4095.0), xyz);
  uv1960(xyz, locus + 2 * m);
}

// Nearest Planckian-locus temperature of each (x,y) cell in CIE 1960 uv.
__global__ void cct_kernel(const double *locus, double *cct) {
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= kCnx || j >= kCny) return;
  double x = 0.15 + 0.60 * (i + 0.5) / kCnx, y = 0.15 + 0.35 * (j + 0.5) / kCny;
  double c[3] = {__ddiv_rn(x, y), 1.0, __ddiv_rn(__dadd_rn(__dadd_rn(1.0, -x), -y), y)};
  double uv[2];
  uv1960(c, uv);
  int best = 0;
  double bd = INFINITY;
  for (int m = 0; m < kNLocus; ++m) {
    double du = __dadd_rn(uv[0], -locus[2 * m]), dv = __dadd_rn(uv[1], -locus[2 * m + 1]);
    double d = __dadd_rn(__dmul_rn(du, du), __dmul_rn(dv, dv));
    if (d < bd) { bd = d; best = m; }
  }
  cct[j * kCnx + i] = 1000.0 * pow(40.0, best / 4095.0);
}

// C(xy, D) = XYZ(B_{D T}) / (X+Y+Z)(B_T): D^5 I(D lambda) of a black body is
// the black body at temperature D T.
__global__ void ctable_kernel(const double *cmf, const double *cct, float4 *C) {
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  if (i >= kCnx) return;
  double T = cct[j * kCnx + i];
  double e[3], r[3];
  dblackbody_xyz(cmf, T, e);
  double es = e[0] + e[1] + e[2];
  double D = exp2(-4.0 + 8.0 * (k + 0.5) / kCnd);
  dblackbody_xyz(cmf, D * T, r);
  C[((size_t)k * kCny + j) * kCnx + i] =
      make_float4((float)(r[0] / es), (float)(r[1] / es), (float)(r[2] / es), 0.f);
}

// Disc table: ln Y, X/Y, Z/Y of B_T at log2 T = 8 + 12 (k + 1/2)/n (one
// exponential per lookup).
__global__ void disc_table_kernel(const double *cmf, float4 *out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kDiscN) return;
  double xyz[3];
  dblackbody_xyz(cmf, exp2(8.0 + 12.0 * (k + 0.5) / kDiscN), xyz);
  out[k] = make_float4((float)log(xyz[1]), (float)(xyz[0] / xyz[1]), (float)(xyz[2] / xyz[1]), 0.f);
}

bh_status colour_tables_launch(bh_ctx *ctx, bh_tables *t, cudaStream_t s) {
  double *scratch = nullptr;
  size_t n = 3 * kNLambda + 2 * kNLocus + kCnx * kCny;
  BH_CUDA(cudaMallocAsync((void **)&scratch, n * sizeof(double), s));
  double *cmf = scratch, *locus = scratch + 3 * kNLambda, *cct = locus + 2 * kNLocus;
  cmf_kernel<<<1, 128, 0, s>>>(cmf);
  locus_kernel<<<(kNLocus + 127) / 128, 128, 0, s>>>(cmf, locus);
  cct_kernel<<<dim3(1, kCny), kCnx, 0, s>>>(locus, cct);
  ctable_kernel<<<dim3(1, kCny, kCnd), kCnx, 0, s>>>(cmf, cct, t->C);
  disc_table_kernel<<<(kDiscN + 127) / 128, 128, 0, s>>>(cmf, t->disc);
  count_launch(ctx, 5);
  BH_CUDA(cudaGetLastError());
  BH_CUDA(cudaFreeAsync(scratch, s));
  return BH_OK;
}

}  // namespace bh

using namespace bh;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" const char *bh_last_error(void) { return g_last_error.c_str(); }

extern "C" bh_status bh_create(int device, size_t budget, bh_ctx **out) {
  if (!out) { set_error("bh_create: out is NULL"); return BH_ERR_INVALID_ARG; }
  *out = nullptr;
  int ndev = 0;
  BH_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) {
    set_error("bh_create: device %d not in [0, %d)", device, ndev);
    return BH_ERR_INVALID_ARG;
  }
  BH_CUDA(cudaSetDevice(device));
  bh_ctx *c = new bh_ctx();
  c->device = device;
  c->budget = budget;
  cudaError_t e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->status_dev, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(c->status_dev, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->sched_dev, sizeof(unsigned) * 2 * kSchedRing);
  if (e == cudaSuccess) e = cudaMemset(c->sched_dev, 0, sizeof(unsigned) * 2 * kSchedRing);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    bh_destroy(c);
    return cuda_fail(e, "bh_create");
  }
  static bool gl_ready[64] = {false};
  static std::mutex gl_mu;
  {
    std::lock_guard<std::mutex> lk(gl_mu);
    if (device < 64 && !gl_ready[device]) {
      double x[kGL], w[kGL];
      gauss_legendre(kGL, x, w);
      e = cudaMemcpyToSymbol(cGLx, x, sizeof x);
      if (e == cudaSuccess) e = cudaMemcpyToSymbol(cGLw, w, sizeof w);
      if (e != cudaSuccess) {
        bh_destroy(c);
        return cuda_fail(e, "bh_create: Gauss-Legendre nodes");
      }
      gl_ready[device] = true;
    }
  }
  *out = c;
  return BH_OK;
}

namespace bh {
void serve_destroy(bh_ctx *ctx);
}

extern "C" void bh_destroy(bh_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  bh::serve_destroy(c);
  cudaDeviceSynchronize();
  c->graph.reset();
  if (c->status_dev) cudaFree(c->status_dev);
  if (c->sched_dev) cudaFree(c->sched_dev);
  if (c->aux) cudaStreamDestroy(c->aux);
  if (c->cam_host) cudaFreeHost(c->cam_host);
  if (c->cam_dev) cudaFree(c->cam_dev);
  if (c->frame_dev) cudaFree(c->frame_dev);
  for (int k = 0; k < 2; ++k) {
    if (c->ring_dev[k]) cudaFree(c->ring_dev[k]);
    if (c->ring_ready[k]) cudaEventDestroy(c->ring_ready[k]);
    if (c->ring_done[k]) cudaEventDestroy(c->ring_done[k]);
  }
  if (c->ring_copy) cudaStreamDestroy(c->ring_copy);
  if (c->bloom_dev) cudaFree(c->bloom_dev);
  if (c->bloom_bar) cudaFree(c->bloom_bar);
  if (c->orb_outs_host) cudaFreeHost(c->orb_outs_host);
  if (c->orb_outs_dev) cudaFree(c->orb_outs_dev);
  if (c->orb_cams_dev) cudaFree(c->orb_cams_dev);
  delete c;
}

extern "C" long long bh_kernel_launches(const bh_ctx *ctx) {
  return ctx ? ctx->launches.load() : 0;
}

static bool valid_desc(const bh_table_desc *d) {
  if (!d) { set_error("table desc is NULL"); return false; }
  if (d->d_n < 4 || d->d_n > 4096 || (d->d_n & 1)) {
    set_error("d_n = %d: must be even, 4..4096", d->d_n);
    return false;
  }
  if (d->u_ne < 2 || d->u_nphi < 2 || d->u_ne * d->u_nphi > kMaxUTexels) {
    set_error("U table %d x %d: each >= 2 and at most %d texels", d->u_ne, d->u_nphi, kMaxUTexels);
    return false;
  }
  if (d->storage != BH_F32 && d->storage != BH_F16) {
    set_error("table storage must be BH_F32 or BH_F16");
    return false;
  }
  return true;
}

static bh_status tables_alloc(bh_ctx *ctx, const bh_table_desc *desc, cudaStream_t s,
                              bh_tables **out) {
  bh_tables *t = new bh_tables();
  t->ctx = ctx;
  t->desc = *desc;
  size_t nd = (size_t)desc->d_n * desc->d_n, nu = (size_t)desc->u_ne * desc->u_nphi;
  size_t es = desc->storage == BH_F32 ? 4 : 2;
  cudaError_t e = cudaMalloc((void **)&t->D64, nd * 8);
  if (e == cudaSuccess) e = cudaMalloc((void **)&t->U64, nu * 8);
  if (e == cudaSuccess) e = cudaMalloc(&t->D, 2 * nd * es);  // row-paired render copy
  if (e == cudaSuccess) e = cudaMalloc(&t->U, ((nu * es + 15) / 16) * 16);
  if (e == cudaSuccess) e = cudaMalloc((void **)&t->DT64, nd * 8);
  if (e == cudaSuccess) e = cudaMalloc((void **)&t->UT64, nu * 8);
  if (e == cudaSuccess) e = cudaMalloc((void **)&t->DT, nd * 4);
  if (e == cudaSuccess) e = cudaMalloc((void **)&t->UT, nu * 4);
  if (e == cudaSuccess) e = cudaMalloc((void **)&t->C, sizeof(float4) * kCnx * kCny * kCnd);
  if (e == cudaSuccess) e = cudaMalloc((void **)&t->disc, sizeof(float4) * kDiscN);
  if (e != cudaSuccess) {
    bh_tables_free(t);
    return cuda_fail(e, "table allocation");
  }
  (void)s;
  *out = t;
  return BH_OK;
}

extern "C" bh_status bh_precompute_tables(bh_ctx *ctx, const bh_table_desc *desc, void *stream,
                                          bh_tables **out) {
  TraceRange trace_("bh_precompute_tables");
  if (!ctx || !out) { set_error("bh_precompute_tables: NULL argument"); return BH_ERR_INVALID_ARG; }
  *out = nullptr;
  if (!valid_desc(desc)) return BH_ERR_INVALID_ARG;
  BH_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  bh_tables *t = nullptr;
  bh_status st = tables_alloc(ctx, desc, s, &t);
  if (st) return st;
  int n = desc->d_n;
  dim3 gd((n + 127) / 128, n);
  unsigned gu = (unsigned)((desc->u_ne * desc->u_nphi + 3) / 4);  // 4 warps (texels) per block
  precompute_D_kernel<<<gd, 128, 0, s>>>(n, t->D64, t->DT64, t->DT);
  if (desc->storage == BH_F32) {
    pair_d_kernel<float><<<gd, 128, 0, s>>>(n, t->D64, (float *)t->D);
    precompute_U_kernel<float><<<gu, 128, 0, s>>>(desc->u_ne, desc->u_nphi, t->U64, (float *)t->U, t->UT64,
                                                 t->UT);
  } else {
    pair_d_kernel<__half><<<gd, 128, 0, s>>>(n, t->D64, (__half *)t->D);
    precompute_U_kernel<__half><<<gu, 128, 0, s>>>(desc->u_ne, desc->u_nphi, t->U64, (__half *)t->U, t->UT64,
                                                  t->UT);
  }
  count_launch(ctx, 3);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { bh_tables_free(t); return cuda_fail(e, "precompute launch"); }
  st = colour_tables_launch(ctx, t, s);
  if (st) { bh_tables_free(t); return st; }
  *out = t;
  return BH_OK;
}

namespace bh {
bh_status tables_alloc_public(bh_ctx *ctx, const bh_table_desc *desc, bh_tables **out) {
  return tables_alloc(ctx, desc, nullptr, out);
}

// Storage copies of D and U (the table's storage type) and FP32 copies of the
// time channels from the FP64 values already on the device.
bh_status tables_convert_storage(bh_ctx *ctx, bh_tables *t, cudaStream_t s) {
  size_t nd = (size_t)t->desc.d_n * t->desc.d_n, nu = (size_t)t->desc.u_ne * t->desc.u_nphi;
  const int n = t->desc.d_n;
  const dim3 gd((n + 127) / 128, n);
  if (t->desc.storage == BH_F32) {
    pair_d_kernel<float><<<gd, 128, 0, s>>>(n, t->D64, (float *)t->D);
    convert_kernel<float><<<(nu + 255) / 256, 256, 0, s>>>(t->U64, (float *)t->U, nu);
  } else {
    pair_d_kernel<__half><<<gd, 128, 0, s>>>(n, t->D64, (__half *)t->D);
    convert_kernel<__half><<<(nu + 255) / 256, 256, 0, s>>>(t->U64, (__half *)t->U, nu);
  }
  convert_kernel<float><<<(nd + 255) / 256, 256, 0, s>>>(t->DT64, t->DT, nd);
  convert_kernel<float><<<(nu + 255) / 256, 256, 0, s>>>(t->UT64, t->UT, nu);
  count_launch(ctx, 4);
  BH_CUDA(cudaGetLastError());
  return BH_OK;
}
}  // namespace bh

extern "C" bh_status bh_tables_upload(bh_ctx *ctx, const bh_table_desc *desc, const double *Dh,
                                      const double *Uh, void *stream, bh_tables **out) {
  TraceRange trace_("bh_tables_upload");
  if (!ctx || !out || !Dh || !Uh) { set_error("bh_tables_upload: NULL argument"); return BH_ERR_INVALID_ARG; }
  *out = nullptr;
  if (!valid_desc(desc)) return BH_ERR_INVALID_ARG;
  BH_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  bh_tables *t = nullptr;
  bh_status st = tables_alloc(ctx, desc, s, &t);
  if (st) return st;
  size_t nd = (size_t)desc->d_n * desc->d_n, nu = (size_t)desc->u_ne * desc->u_nphi;
  cudaError_t e = cudaMemcpyAsync(t->D64, Dh, nd * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(t->U64, Uh, nu * 8, cudaMemcpyHostToDevice, s);
  // no time channel until bh_tables_upload_time: all-ones bytes read as NaN
  if (e == cudaSuccess) e = cudaMemsetAsync(t->DT64, 0xff, nd * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->UT64, 0xff, nu * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->DT, 0xff, nd * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->UT, 0xff, nu * 4, s);
  if (e == cudaSuccess) {
    const int n = desc->d_n;
    const dim3 gd((n + 127) / 128, n);
    if (desc->storage == BH_F32) {
      pair_d_kernel<float><<<gd, 128, 0, s>>>(n, t->D64, (float *)t->D);
      convert_kernel<float><<<(nu + 255) / 256, 256, 0, s>>>(t->U64, (float *)t->U, nu);
    } else {
      pair_d_kernel<__half><<<gd, 128, 0, s>>>(n, t->D64, (__half *)t->D);
      convert_kernel<__half><<<(nu + 255) / 256, 256, 0, s>>>(t->U64, (__half *)t->U, nu);
    }
    count_launch(ctx, 2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    st = colour_tables_launch(ctx, t, s);
    if (st) { bh_tables_free(t); return st; }
    e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) { bh_tables_free(t); return cuda_fail(e, "bh_tables_upload"); }
  *out = t;
  return BH_OK;
}

extern "C" bh_status bh_tables_copy_out(const bh_tables *t, double *Dh, double *Uh) {
  if (!t) { set_error("bh_tables_copy_out: NULL tables"); return BH_ERR_INVALID_ARG; }
  BH_CUDA(cudaSetDevice(t->ctx->device));
  BH_CUDA(cudaDeviceSynchronize());
  if (Dh) BH_CUDA(cudaMemcpy(Dh, t->D64, sizeof(double) * t->desc.d_n * t->desc.d_n, cudaMemcpyDeviceToHost));
  if (Uh) BH_CUDA(cudaMemcpy(Uh, t->U64, sizeof(double) * t->desc.u_ne * t->desc.u_nphi, cudaMemcpyDeviceToHost));
  return BH_OK;
}

extern "C" bh_status bh_tables_upload_time(bh_tables *t, const double *DTh, const double *UTh, void *stream) {
  if (!t || !DTh || !UTh) { set_error("bh_tables_upload_time: NULL argument"); return BH_ERR_INVALID_ARG; }
  BH_CUDA(cudaSetDevice(t->ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  size_t nd = (size_t)t->desc.d_n * t->desc.d_n, nu = (size_t)t->desc.u_ne * t->desc.u_nphi;
  BH_CUDA(cudaMemcpyAsync(t->DT64, DTh, nd * 8, cudaMemcpyHostToDevice, s));
  BH_CUDA(cudaMemcpyAsync(t->UT64, UTh, nu * 8, cudaMemcpyHostToDevice, s));
  convert_kernel<float><<<(nd + 255) / 256, 256, 0, s>>>(t->DT64, t->DT, nd);
  convert_kernel<float><<<(nu + 255) / 256, 256, 0, s>>>(t->UT64, t->UT, nu);
  count_launch(t->ctx, 2);
  BH_CUDA(cudaGetLastError());
  BH_CUDA(cudaStreamSynchronize(s));
  return BH_OK;
}

extern "C" bh_status bh_tables_copy_time(const bh_tables *t, double *DTh, double *UTh) {
  if (!t) { set_error("bh_tables_copy_time: NULL tables"); return BH_ERR_INVALID_ARG; }
  BH_CUDA(cudaSetDevice(t->ctx->device));
  BH_CUDA(cudaDeviceSynchronize());
  if (DTh) BH_CUDA(cudaMemcpy(DTh, t->DT64, sizeof(double) * t->desc.d_n * t->desc.d_n, cudaMemcpyDeviceToHost));
  if (UTh)
    BH_CUDA(cudaMemcpy(UTh, t->UT64, sizeof(double) * t->desc.u_ne * t->desc.u_nphi, cudaMemcpyDeviceToHost));
  return BH_OK;
}

extern "C" bh_status bh_tables_copy_colour(const bh_tables *t, float *Ch, float *dh) {
  if (!t) { set_error("bh_tables_copy_colour: NULL tables"); return BH_ERR_INVALID_ARG; }
  BH_CUDA(cudaSetDevice(t->ctx->device));
  BH_CUDA(cudaDeviceSynchronize());
  if (Ch) BH_CUDA(cudaMemcpy(Ch, t->C, sizeof(float4) * kCnx * kCny * kCnd, cudaMemcpyDeviceToHost));
  if (dh) BH_CUDA(cudaMemcpy(dh, t->disc, sizeof(float4) * kDiscN, cudaMemcpyDeviceToHost));
  return BH_OK;
}

extern "C" void bh_tables_free(bh_tables *t) {
  if (!t) return;
  cudaSetDevice(t->ctx->device);
  cudaDeviceSynchronize();
  cudaFree(t->D64);
  cudaFree(t->U64);
  cudaFree(t->D);
  cudaFree(t->U);
  cudaFree(t->DT64);
  cudaFree(t->UT64);
  cudaFree(t->DT);
  cudaFree(t->UT);
  cudaFree(t->C);
  cudaFree(t->disc);
  delete t;
}
