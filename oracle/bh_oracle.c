/*
 * bh_oracle.c -- plain FP64 CPU oracle for the table-driven Schwarzschild
 * beam tracer of E. Bruneton, "Real-time High-Quality Rendering of
 * Non-Rotating Black Holes" (2020).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously correct reference
 * the CUDA library is checked against.  Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg load it; the product library never links,
 * includes or calls anything in this directory, and this file includes
 * nothing from the product.
 *
 * Every step follows the paper's equations in the paper's order, in double
 * precision, one pixel at a time:
 *   - tables D(e,u) and U(e,phi): Algorithm 1 PRECOMPUTE, but the ray
 *     equation (Eq. rayequation, u'' = 3/2 u^2 - u) is integrated with the
 *     classical fixed-step Runge-Kutta 4 instead of Euler (Sec. 3.3.2 leaves
 *     the integrator open), sampled exactly at the texel
 *     coordinates i/(n-1) of the Appendix A mappings (reading C3), with the
 *     retarded-time channel of Algorithm 1 carried as the regularised time
 *     R = t + 1/u - ln(u/(1-u)) (reading C5);
 *   - camera basis and beam direction: Eq. staticbasis, Eq. camerabasis,
 *     Eq. d, Eq. raybasis, Eq. alpha;
 *   - Algorithm 1 TRACERAY with bilinear table lookups;
 *   - disc emission (Sec. 3.3.3), Doppler and beaming (Sec. 3.4.2),
 *     lensing amplification (Sec. 3.4.1);
 *   - the manually filtered star cube map (Sec. 3.3.2, "Emitted light"):
 *     build with colour sums and luminance-weighted positions, mip level
 *     with at most 9x9 texels, tent weights f(w)f(h);
 *   - C(xy,D) colour-shift table (Sec. 3.4.2);
 *   - the animated disc of linear particles on precessing orbits, shaded at
 *     the retarded time of each crossing (Appendix B);
 *   - free-fall camera orbits (Appendix C).
 * Where the paper is silent the reading used is listed in the design notes
 * of the repository (readings C1..C26); each is restated at its use below.
 *
 * A brute-force, table-free integrator of the 3D photon orbit (carrying the
 * coordinate time along it) is included for the table-method error report
 * (Sec. 4: TRACERAY's results within 1e-3 of values computed without
 * intermediate textures).
 *
 * Parity notes: the colour observer (piecewise-Gaussian colour matching
 * functions) is pinned to the published Planckian locus through the black
 * body's chromaticity; the C(xy,D) chromaticity-to-spectrum choice is a
 * project definition, "parity unpinned" for that choice itself.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Counting hooks (no-ops here).  The counting build (op_count.cpp, test
 * infrastructure) compiles this file as C++ with every double replaced by a
 * counting double and defines these to tally the per-pixel work: operations
 * by class, table texels read, and the cube-map records touched. */
#ifndef ORC_COUNTING
#define ORC_COUNT_PAUSE()
#define ORC_COUNT_RESUME()
#define ORC_COUNT_FLUSH()
#define ORC_FETCH(cls, k)
#define ORC_TOUCH(rec, occupied)
#endif

#define MU (4.0 / 27.0) /* max of u^2 (1-u) on [0,1], at the photon sphere u = 2/3 (Sec. 3.3.1) */
#define PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Ray equation and its Runge-Kutta 4 step (Eq. rayequation)                 */
/* ------------------------------------------------------------------------ */

static double accel(double u) { return 1.5 * u * u - u; } /* d2u/dphi2 */

static void rk4_step(double u, double ud, double h, double *uo, double *udo) {
  double k1u = ud, k1v = accel(u);
  double u2 = u + 0.5 * h * k1u, v2 = ud + 0.5 * h * k1v;
  double k2u = v2, k2v = accel(u2);
  double u3 = u + 0.5 * h * k2u, v3 = ud + 0.5 * h * k2v;
  double k3u = v3, k3v = accel(u3);
  double u4 = u + h * k3u, v4 = ud + h * k3v;
  double k4u = v4, k4v = accel(u4);
  *uo = u + h / 6.0 * (k1u + 2.0 * k2u + 2.0 * k3u + k4u);
  *udo = ud + h / 6.0 * (k1v + 2.0 * k2v + 2.0 * k3v + k4v);
}

/* The same step carrying the regularised time R = t + 1/u - ln(u/(1-u)) of
 * the ray: with dt/dphi = e/(u^2 (1-u)) (Eq. motionconstants) and the first
 * integral (du/dphi)^2 = e^2 - u^2 (1-u), dR/dphi = 1/(e + du/dphi), finite
 * from u = 0 (where R = 0) through the apsis up to phi < pi. */
static void rk4_step_t(double e, double u, double ud, double R, double h, double *uo, double *udo,
                       double *Ro) {
  double k1u = ud, k1v = accel(u), k1r = 1.0 / (e + ud);
  double u2 = u + 0.5 * h * k1u, v2 = ud + 0.5 * h * k1v;
  double k2u = v2, k2v = accel(u2), k2r = 1.0 / (e + v2);
  double u3 = u + 0.5 * h * k2u, v3 = ud + 0.5 * h * k2v;
  double k3u = v3, k3v = accel(u3), k3r = 1.0 / (e + v3);
  double u4 = u + h * k3u, v4 = ud + h * k3v;
  double k4u = v4, k4v = accel(u4), k4r = 1.0 / (e + v4);
  *uo = u + h / 6.0 * (k1u + 2.0 * k2u + 2.0 * k3u + k4u);
  *udo = ud + h / 6.0 * (k1v + 2.0 * k2v + 2.0 * k3v + k4v);
  *Ro = R + h / 6.0 * (k1r + 2.0 * k2r + 2.0 * k3r + k4r);
}

/* Coordinate time from the regularised time: t = R - 1/u + ln(u/(1-u)). */
double orc_time_of_R(double R, double u) { return R - 1.0 / u + log(u / (1.0 - u)); }

/* Apsis of a scattered ray, Eq. uapsis (valid for e^2 < mu). */
double orc_apsis(double e2) {
  return 1.0 / 3.0 + 2.0 / 3.0 * sin(asin(2.0 * e2 / MU - 1.0) / 3.0);
}

/* Inverse of the Appendix A mapping of D's first coordinate: texel x -> e^2.
 * x < 1/2: e^2 < mu,  x = 1/2 - sqrt(-log(1 - e^2/mu)/50).
 * x > 1/2: e^2 > mu,  x = 1/2 + sqrt(-log(1 - mu/e^2)/50).            */
double orc_d_e2_of_x(double x) {
  double a = x - 0.5;
  if (a < 0.0) return MU * (1.0 - exp(-50.0 * a * a));
  return MU / (1.0 - exp(-50.0 * a * a));
}

/* Inverse of the Appendix A mapping of D's second coordinate: (e^2, y) -> u. */
double orc_d_u_of_y(double e2, double y) {
  if (e2 < MU) {
    double ua = orc_apsis(e2);
    return ua * (1.0 - (1.0 - y) * (1.0 - y)); /* y = 1 - sqrt(1 - u/ua) */
  }
  double z = y * (sqrt(2.0 / 3.0) + sqrt(1.0 / 3.0)) - sqrt(2.0 / 3.0);
  return 2.0 / 3.0 + (z >= 0.0 ? z * z : -z * z); /* y = (sqrt(2/3) +- sqrt|u-2/3|)/(...) */
}

/* Inverse of the Appendix A mapping of U: texel (x,y) -> (e^2, phi). */
double orc_u_e2_of_x(double x) { return (1.0 / x - 1.0) / 6.0; }
double orc_u_phi_of_y(double e2, double y) {
  double e = sqrt(e2);
  return 3.0 * y * (1.0 + e2) / (1.0 + 6.0 * e2 * e);
}

/* ------------------------------------------------------------------------ */
/* PRECOMPUTE (Algorithm 1) with RK4 sampled at texel centres                */
/* ------------------------------------------------------------------------ */

/* Partial RK4 step of length s solving u(s) = target on [0, smax], where u
 * is increasing on that interval.  Bisection to full double precision. */
static double solve_step_for_u(double u, double ud, double smax, double target) {
  double lo = 0.0, hi = smax;
  for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    double um, udm;
    rk4_step(u, ud, mid, &um, &udm);
    if (um < target) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* Length s in [0, smax] of the partial step at which du/dphi = 0 (apsis),
 * given ud > 0 at s = 0 and ud < 0 at s = smax. */
static double solve_step_for_apsis(double u, double ud, double smax) {
  double lo = 0.0, hi = smax;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    double um, udm;
    rk4_step(u, ud, mid, &um, &udm);
    if (udm > 0.0) lo = mid; else hi = mid;
  }
  return lo;
}

/* One column (fixed e) of D: Delta(e, u_j) = phi - atan2(u, du/dphi) on the
 * ray coming from infinity (u = 0, du/dphi = e, phi = 0), for the n texel
 * coordinates y_j = j/(n-1) of the Appendix A mapping (reading C3: the first
 * and last texels hold the ends of the [0,1] range, so y = 1 is the apsis or
 * the horizon exactly).  out[j*stride]. */
static void d_column(double e2, int n, double h0, double *out, double *outR, int stride) {
  double e = sqrt(e2);
  double h = h0 / (e > 1.0 ? e : 1.0);
  double u = 0.0, ud = e, phi = 0.0, R = 0.0;
  int j = 0;
  double target = orc_d_u_of_y(e2, 0.0);
  while (j < n) {
    double u1, ud1, R1;
    rk4_step_t(e, u, ud, R, h, &u1, &ud1, &R1);
    if (e2 < MU && ud1 <= 0.0) {
      /* The apsis lies inside this step: the remaining texels are between
       * the current point and the apsis, where u increases. */
      double sa = solve_step_for_apsis(u, ud, h);
      double ua, uda;
      rk4_step(u, ud, sa, &ua, &uda);
      while (j < n) {
        /* y = 1 is the apsis itself; elsewhere find u(s) = target */
        double s = (j == n - 1 || target > ua) ? sa : solve_step_for_u(u, ud, sa, target);
        double us, uds, Rs;
        rk4_step_t(e, u, ud, R, s, &us, &uds, &Rs);
        if (uds < 0.0) uds = 0.0;
        out[(long)j * stride] = phi + s - atan2(us, uds);
        if (outR) outR[(long)j * stride] = Rs;
        ++j;
        if (j < n) target = orc_d_u_of_y(e2, (double)j / (n - 1));
      }
      break;
    }
    while (j < n && target <= u1) {
      double s = solve_step_for_u(u, ud, h, target);
      double us, uds, Rs;
      rk4_step_t(e, u, ud, R, s, &us, &uds, &Rs);
      out[(long)j * stride] = phi + s - atan2(us, uds);
      if (outR) outR[(long)j * stride] = Rs;
      ++j;
      if (j < n) target = orc_d_u_of_y(e2, (double)j / (n - 1));
    }
    u = u1; ud = ud1; R = R1; phi += h;
  }
}

/* One column (fixed e) of U: u(phi_j) on the ray from infinity for the
 * texel coordinates y_j = j/(n-1), or 1 once the ray has reached the horizon
 * u = 1 (reading C7).  Algorithm 1 writes U for phi < pi only; every texel of
 * the Appendix A mapping has phi < pi. */
static void u_column(double e2, int n, double h0, double *out, double *outR, int stride) {
  double e = sqrt(e2);
  double h = h0 / (e > 1.0 ? e : 1.0);
  double u = 0.0, ud = e, phi = 0.0, R = 0.0;
  int captured = 0;
  for (int j = 0; j < n; ++j) {
    double phij = orc_u_phi_of_y(e2, (double)j / (n - 1));
    while (!captured && phi + h <= phij) {
      double u1, ud1, R1;
      rk4_step_t(e, u, ud, R, h, &u1, &ud1, &R1);
      u = u1; ud = ud1; R = R1; phi += h;
      if (u >= 1.0) captured = 1;
    }
    if (captured) {
      out[(long)j * stride] = 1.0;
      if (outR) outR[(long)j * stride] = 0.0;
      continue;
    }
    double us, uds, Rs;
    rk4_step_t(e, u, ud, R, phij - phi, &us, &uds, &Rs);
    out[(long)j * stride] = us >= 1.0 ? 1.0 : us;
    if (outR) outR[(long)j * stride] = us >= 1.0 ? 0.0 : Rs;
  }
}

/* Exact tables.  D: d_n x d_n doubles, D[j*d_n + i], i indexes e (x), j
 * indexes u (y).  U: u_nphi x u_ne doubles, U[j*u_ne + i], i indexes e, j
 * indexes phi.  Texel i of n holds coordinate i/(n-1) (reading C3).  h0 is
 * the RK4 step in phi (scaled down by e for e > 1).  U's column x = 0 is the
 * limit e -> infinity, a radial ray, captured at once (u = 1 for phi > 0).
 * DT, UT (may be NULL): the regularised time R = t + 1/u - ln(u/(1-u)) of the
 * same texels (reading C5); 0 where u = 0 or the ray is captured. */
int orc_tables_exact2(int d_n, int u_ne, int u_nphi, double h0, double *D, double *U, double *DT,
                      double *UT) {
  if (d_n < 4 || (d_n & 1) || u_ne < 2 || u_nphi < 2 || !(h0 > 0.0)) return 1;
  for (int i = 0; i < d_n; ++i) {
    double e2 = orc_d_e2_of_x((double)i / (d_n - 1));
    d_column(e2, d_n, h0, D + i, DT ? DT + i : NULL, d_n);
  }
  for (int j = 0; j < u_nphi; ++j) {
    U[(long)j * u_ne] = j == 0 ? 0.0 : 1.0;
    if (UT) UT[(long)j * u_ne] = 0.0;
  }
  for (int i = 1; i < u_ne; ++i) {
    double e2 = orc_u_e2_of_x((double)i / (u_ne - 1));
    if (e2 <= 0.0) { /* e = 0: no ray */
      for (int j = 0; j < u_nphi; ++j) {
        U[(long)j * u_ne + i] = 0.0;
        if (UT) UT[(long)j * u_ne + i] = 0.0;
      }
      continue;
    }
    u_column(e2, u_nphi, h0, U + i, UT ? UT + i : NULL, u_ne);
  }
  return 0;
}

int orc_tables_exact(int d_n, int u_ne, int u_nphi, double h0, double *D, double *U) {
  return orc_tables_exact2(d_n, u_ne, u_nphi, h0, D, U, NULL, NULL);
}

/* u(phi) on the ray from infinity with constant e (RK4, step h0); 1 once
 * captured.  Exposed for the symmetry and closed-form checks. */
double orc_u_of_phi(double e2, double phi, double h0) {
  double out;
  double e = sqrt(e2);
  double h = h0 / (e > 1.0 ? e : 1.0);
  double u = 0.0, ud = e, p = 0.0;
  while (p + h <= phi) {
    double u1, ud1;
    rk4_step(u, ud, h, &u1, &ud1);
    u = u1; ud = ud1; p += h;
    if (u >= 1.0) return 1.0;
  }
  double us, uds;
  rk4_step(u, ud, phi - p, &us, &uds);
  out = us;
  return out;
}

/* Deflection at the apsis, Delta_a = phi_a - pi/2, of the ray from infinity
 * with e^2 < mu (RK4 to the point where du/dphi changes sign). */
double orc_apsis_deflection(double e2, double h0) {
  double e = sqrt(e2);
  double h = h0 / (e > 1.0 ? e : 1.0);
  double u = 0.0, ud = e, p = 0.0;
  if (!(e2 < MU)) return INFINITY;
  for (;;) {
    double u1, ud1;
    rk4_step(u, ud, h, &u1, &ud1);
    if (ud1 <= 0.0) return p + solve_step_for_apsis(u, ud, h) - PI / 2.0;
    u = u1; ud = ud1; p += h;
  }
}

/* Coordinate time t(phi) on the ray from infinity, from the regularised time
 * (RK4, step h0): out[0] = u, out[1] = du/dphi, out[2] = R, out[3] = t. */
void orc_time_at_phi(double e2, double phi, double h0, double *out) {
  double e = sqrt(e2);
  double h = h0 / (e > 1.0 ? e : 1.0);
  double u = 0.0, ud = e, R = 0.0, p = 0.0;
  while (p + h <= phi) {
    double u1, ud1, R1;
    rk4_step_t(e, u, ud, R, h, &u1, &ud1, &R1);
    u = u1; ud = ud1; R = R1; p += h;
  }
  rk4_step_t(e, u, ud, R, phi - p, &out[0], &out[1], &out[2]);
  out[3] = orc_time_of_R(out[2], out[0]);
}

/* State (u, du/dphi) after integrating to angle phi (for the first-integral
 * check).  out[0] = u, out[1] = du/dphi. */
void orc_state_at_phi(double e2, double phi, double h0, double *out) {
  double e = sqrt(e2);
  double h = h0 / (e > 1.0 ? e : 1.0);
  double u = 0.0, ud = e, p = 0.0;
  while (p + h <= phi) {
    double u1, ud1;
    rk4_step(u, ud, h, &u1, &ud1);
    u = u1; ud = ud1; p += h;
  }
  rk4_step(u, ud, phi - p, &out[0], &out[1]);
}

/* ------------------------------------------------------------------------ */
/* Table lookups (readings C2, C3): coordinate x in [0,1] reads texel          */
/* x (n-1), bilinear, D's first coordinate clamped inside its own branch.    */
/* ------------------------------------------------------------------------ */

static double lerp(double a, double b, double t) { return a + (b - a) * t; }

static double bilinear(const double *T, int nx, int ny, double fx, double fy,
                       int xlo, int xhi) {
  if (fx < xlo) fx = xlo;
  if (fx > xhi) fx = xhi;
  if (fy < 0.0) fy = 0.0;
  if (fy > ny - 1) fy = ny - 1;
  int i0 = (int)floor(fx), j0 = (int)floor(fy);
  int i1 = i0 + 1 > xhi ? xhi : i0 + 1;
  int j1 = j0 + 1 > ny - 1 ? ny - 1 : j0 + 1;
  double tx = fx - i0, ty = fy - j0;
  double a = lerp(T[(long)j0 * nx + i0], T[(long)j0 * nx + i1], tx);
  double b = lerp(T[(long)j1 * nx + i0], T[(long)j1 * nx + i1], tx);
  return lerp(a, b, ty);
}

/* D(e,u) at the Appendix A texel coordinates. */
double orc_d_lookup(const double *D, int n, double e2, double u) {
  double x, y;
  int xlo, xhi;
  if (e2 < MU) {
    double ua = orc_apsis(e2);
    x = 0.5 - sqrt(-log(1.0 - e2 / MU) / 50.0);
    double a = 1.0 - u / ua;
    y = 1.0 - sqrt(a > 0.0 ? a : 0.0);
    xlo = 0; xhi = n / 2 - 1;
  } else {
    x = 0.5 + sqrt(-log(1.0 - MU / e2) / 50.0);
    double s = sqrt(fabs(u - 2.0 / 3.0));
    y = (sqrt(2.0 / 3.0) + (u >= 2.0 / 3.0 ? s : -s)) / (sqrt(2.0 / 3.0) + sqrt(1.0 / 3.0));
    xlo = n / 2; xhi = n - 1;
  }
  ORC_FETCH(kFetchD, 4);
  return bilinear(D, n, n, x * (n - 1), y * (n - 1), xlo, xhi);
}

/* U(e,phi) at the Appendix A texel coordinates. */
double orc_u_lookup(const double *U, int ne, int nphi, double e2, double phi) {
  double e = sqrt(e2);
  double x = 1.0 / (1.0 + 6.0 * e2);
  double y = phi / 3.0 * (1.0 + 6.0 * e2 * e) / (1.0 + e2);
  ORC_FETCH(kFetchU, 4);
  return bilinear(U, ne, nphi, x * (ne - 1), y * (nphi - 1), 0, ne - 1);
}

/* ------------------------------------------------------------------------ */
/* TRACERAY (Algorithm 1)                                                     */
/* out: [0] delta' (INFINITY if captured), [1] number of disc hits,           */
/*      [2] u0, [3] angle of hit 0, [4] u1, [5] angle of hit 1, [6] e^2,      */
/*      [7] hit slots: 1 if slot 0 is the pre-apsis hit, 2 if slot holds the  */
/*      post-apsis hit only (see below).                                      */
/* Hits are returned in the order met along the backward ray.                 */
/* ------------------------------------------------------------------------ */
void orc_trace_ray2(const double *D, const double *DT, int dn, const double *U, const double *UT,
                    int une, int unphi, double pr, double delta, double alpha, int alpha_valid,
                    double u_ic, double u_oc, double *out) {
  double u = 1.0 / pr;
  double ud = -u * cos(delta) / sin(delta); /* du/dphi = -u cot(delta) */
  double e2 = ud * ud + u * u * (1.0 - u);
  out[0] = INFINITY; out[1] = 0; out[2] = 0; out[3] = 0; out[4] = 0; out[5] = 0;
  out[6] = e2; out[7] = 0; out[8] = 0; out[9] = 0;
  if (e2 < MU && u > 2.0 / 3.0) return; /* trapped inside the photon sphere */
  int s = ud > 0.0 ? 1 : -1;
  double Dl = orc_d_lookup(D, dn, e2, u);
  double Da = 0.0, phia = INFINITY;           /* reading C6: no apsis if e^2 >= mu */
  double ua = 0.0;
  if (e2 < MU) {
    ua = orc_apsis(e2);
    Da = orc_d_lookup(D, dn, e2, ua);
    phia = Da + PI / 2.0;
  }
  /* retarded times (Algorithm 1): coordinate time of the camera point and of
   * the apsis on the ray from infinity, from the regularised time channel */
  double tc = 0.0, ta = 0.0;
  if (DT) {
    tc = orc_time_of_R(orc_d_lookup(DT, dn, e2, u), u);
    if (e2 < MU) ta = orc_time_of_R(orc_d_lookup(DT, dn, e2, ua), ua);
  }
  int nh = 0;
  if (alpha_valid) {
    double phi = Dl + (s == 1 ? PI - delta : delta) + s * alpha;
    double phi0 = phi - PI * floor(phi / PI);
    double u0 = orc_u_lookup(U, une, unphi, e2, phi0);
    if (phi0 < phia && u_oc <= u0 && u0 <= u_ic &&
        ((s == 1 && u0 > u) || (s == -1 && u0 < u))) {
      out[2 + 2 * nh] = u0;
      out[3 + 2 * nh] = alpha + phi - phi0;
      if (UT) out[8 + nh] = s * (orc_time_of_R(orc_u_lookup(UT, une, unphi, e2, phi0), u0) - tc);
      ++nh;
    }
    if (e2 < MU && s == 1) {
      phi = 2.0 * phia - phi;
      double phi1 = phi - PI * floor(phi / PI);
      double u1 = orc_u_lookup(U, une, unphi, e2, phi1);
      if (phi1 < phia && u_oc <= u1 && u1 <= u_ic) {
        out[2 + 2 * nh] = u1;
        out[3 + 2 * nh] = alpha + phi - phi1;
        if (UT) out[8 + nh] = 2.0 * ta - tc - orc_time_of_R(orc_u_lookup(UT, une, unphi, e2, phi1), u1);
        ++nh;
      }
    }
  }
  out[1] = nh;
  double Delta = Dl;
  if (ud > 0.0) Delta = e2 < MU ? 2.0 * Da - Dl : INFINITY;
  out[0] = delta + Delta;
}

/* TRACERAY without the time channels; out as orc_trace_ray2 (10 doubles). */
void orc_trace_ray(const double *D, int dn, const double *U, int une, int unphi, double pr,
                   double delta, double alpha, int alpha_valid, double u_ic, double u_oc,
                   double *out) {
  orc_trace_ray2(D, NULL, dn, U, NULL, une, unphi, pr, delta, alpha, alpha_valid, u_ic, u_oc, out);
}

/* ------------------------------------------------------------------------ */
/* Colour: project-defined observer, black bodies, XYZ -> linear sRGB         */
/* ------------------------------------------------------------------------ */

#define NLAMBDA 95 /* 360..830 nm, 5 nm trapezoid */
static double lobe(double l, double m, double s1, double s2) {
  double t = (l - m) / (l < m ? s1 : s2);
  return exp(-0.5 * t * t);
}
/* Piecewise-Gaussian colour matching functions (project-defined observer,
 * after the functional form of Wyman, Sloan and Shirley, JCGT 2(2), 2013). */
void orc_cmf(double l, double *xyz) {
  xyz[0] = 1.056 * lobe(l, 599.8, 37.9, 31.0) + 0.362 * lobe(l, 442.0, 16.0, 26.7) -
           0.065 * lobe(l, 501.1, 20.4, 26.2);
  xyz[1] = 0.821 * lobe(l, 568.8, 46.9, 40.5) + 0.286 * lobe(l, 530.9, 16.3, 31.1);
  xyz[2] = 1.217 * lobe(l, 437.0, 11.8, 36.0) + 0.681 * lobe(l, 459.0, 26.0, 13.8);
}
/* Planck spectral radiance up to a constant factor, lambda in nm. */
double orc_planck(double l, double T) {
  const double c2 = 1.4387769e7; /* h c / k in nm K */
  return 1.0 / (l * l * l * l * l * expm1(c2 / (l * T)));
}
/* XYZ of a black body at temperature T (trapezoid over the 5 nm grid). */
void orc_blackbody_xyz(double T, double *xyz) {
  xyz[0] = xyz[1] = xyz[2] = 0.0;
  if (!(T > 0.0)) return;
  for (int k = 0; k < NLAMBDA; ++k) {
    double l = 360.0 + 5.0 * k;
    double w = (k == 0 || k == NLAMBDA - 1) ? 2.5 : 5.0;
    double c[3];
    orc_cmf(l, c);
    double b = orc_planck(l, T) * w;
    xyz[0] += b * c[0]; xyz[1] += b * c[1]; xyz[2] += b * c[2];
  }
}

/* XYZ -> linear sRGB, derived from the Rec.709 primaries and D65 white. */
void orc_xyz_to_rgb_matrix(double *m) {
  const double px[3] = {0.64, 0.30, 0.15}, py[3] = {0.33, 0.60, 0.06};
  const double wx = 0.3127, wy = 0.3290;
  double P[9]; /* columns: XYZ of each primary with Y = 1 */
  for (int c = 0; c < 3; ++c) {
    P[0 * 3 + c] = px[c] / py[c];
    P[1 * 3 + c] = 1.0;
    P[2 * 3 + c] = (1.0 - px[c] - py[c]) / py[c];
  }
  double W[3] = {wx / wy, 1.0, (1.0 - wx - wy) / wy};
  /* invert P (3x3, cofactors) */
  double det = P[0] * (P[4] * P[8] - P[5] * P[7]) - P[1] * (P[3] * P[8] - P[5] * P[6]) +
               P[2] * (P[3] * P[7] - P[4] * P[6]);
  double I[9];
  I[0] = (P[4] * P[8] - P[5] * P[7]) / det; I[1] = (P[2] * P[7] - P[1] * P[8]) / det;
  I[2] = (P[1] * P[5] - P[2] * P[4]) / det; I[3] = (P[5] * P[6] - P[3] * P[8]) / det;
  I[4] = (P[0] * P[8] - P[2] * P[6]) / det; I[5] = (P[2] * P[3] - P[0] * P[5]) / det;
  I[6] = (P[3] * P[7] - P[4] * P[6]) / det; I[7] = (P[1] * P[6] - P[0] * P[7]) / det;
  I[8] = (P[0] * P[4] - P[1] * P[3]) / det;
  double S[3]; /* primary scales so that RGB = (1,1,1) maps to W */
  for (int r = 0; r < 3; ++r) S[r] = I[r * 3 + 0] * W[0] + I[r * 3 + 1] * W[1] + I[r * 3 + 2] * W[2];
  /* M = P diag(S); return inverse(M) = diag(1/S) inverse(P) */
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) m[r * 3 + c] = I[r * 3 + c] / S[r];
}

/* Disc colour table: ln Y, X/Y and Z/Y of B_T at log2 T = 8 + 12 (k+1/2)/n. */
int orc_disc_colour_table(int n, double *out) {
  for (int k = 0; k < n; ++k) {
    double T = exp2(8.0 + 12.0 * (k + 0.5) / n);
    double xyz[3];
    orc_blackbody_xyz(T, xyz);
    out[3 * k + 0] = log(xyz[1]);
    out[3 * k + 1] = xyz[0] / xyz[1];
    out[3 * k + 2] = xyz[2] / xyz[1];
  }
  return 0;
}

/* XYZ of B_T from the disc colour table: ln Y, X/Y and Z/Y linear in log2 T,
 * clamped to the table's range; 0 below 2^8 K. */
static void disc_xyz(const double *tab, int n, double T, double *xyz) {
  if (!(T >= 256.0)) { xyz[0] = xyz[1] = xyz[2] = 0.0; return; }
  double f = (log2(T) - 8.0) / 12.0 * n - 0.5;
  if (f < 0.0) f = 0.0;
  if (f > n - 1) f = n - 1;
  int k0 = (int)floor(f);
  int k1 = k0 + 1 > n - 1 ? n - 1 : k0 + 1;
  double t = f - k0;
  ORC_FETCH(kFetchDisc, 2);
  double Y = exp(lerp(tab[3 * k0], tab[3 * k1], t));
  xyz[0] = Y * lerp(tab[3 * k0 + 1], tab[3 * k1 + 1], t);
  xyz[1] = Y;
  xyz[2] = Y * lerp(tab[3 * k0 + 2], tab[3 * k1 + 2], t);
}

/* For tests: the disc colour table lookup the render uses. */
void orc_disc_xyz(const double *tab, int n, double T, double *xyz) { disc_xyz(tab, n, T, xyz); }

/* CIE 1960 uv of an XYZ colour. */
static void uv1960(const double *xyz, double *uv) {
  double den = xyz[0] + 15.0 * xyz[1] + 3.0 * xyz[2];
  uv[0] = 4.0 * xyz[0] / den;
  uv[1] = 6.0 * xyz[1] / den;
}

#define NLOCUS 4096
/* Temperature of the Planckian-locus point nearest to chromaticity (x,y) in
 * CIE 1960 uv, over T_m = 1000 * 40^(m/4095) (reading C14). */
static double cct_of_xy(const double *locus_uv, double x, double y) {
  double X = x / y, Z = (1.0 - x - y) / y;
  double c[3] = {X, 1.0, Z}, uv[2];
  uv1960(c, uv);
  int best = 0;
  double bd = INFINITY;
  for (int m = 0; m < NLOCUS; ++m) {
    double du = uv[0] - locus_uv[2 * m], dv = uv[1] - locus_uv[2 * m + 1];
    double d = du * du + dv * dv;
    if (d < bd) { bd = d; best = m; }
  }
  return 1000.0 * pow(40.0, best / 4095.0);
}

/* C(xy, D) table (Sec. 3.4.2) with a1 = a2 = 0 (reading C14): the spectrum
 * of chromaticity xy is the black body at its nearest-locus temperature T,
 * and D^5 I(D lambda) of a black body is B_{D T}(lambda); so
 * C = XYZ(B_{DT}) / (X+Y+Z)(B_T).  Layout [k][j][i][3], i: x, j: y, k: log2 D. */
int orc_colour_table(int nx, int ny, int nd, double *C) {
  double *locus = (double *)malloc(sizeof(double) * 2 * NLOCUS);
  if (!locus) return 1;
  for (int m = 0; m < NLOCUS; ++m) {
    double xyz[3];
    orc_blackbody_xyz(1000.0 * pow(40.0, m / 4095.0), xyz);
    uv1960(xyz, locus + 2 * m);
  }
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double x = 0.15 + 0.60 * (i + 0.5) / nx, y = 0.15 + 0.35 * (j + 0.5) / ny;
      double T = cct_of_xy(locus, x, y);
      double e[3];
      orc_blackbody_xyz(T, e);
      double es = e[0] + e[1] + e[2];
      for (int k = 0; k < nd; ++k) {
        double D = exp2(-4.0 + 8.0 * (k + 0.5) / nd);
        double r[3];
        orc_blackbody_xyz(D * T, r);
        double *o = C + (((long)k * ny + j) * nx + i) * 3;
        o[0] = r[0] / es; o[1] = r[1] / es; o[2] = r[2] / es;
      }
    }
  free(locus);
  return 0;
}

/* Trilinear C(xy, D) lookup, texel centres, clamped. */
static void c_lookup(const double *C, int nx, int ny, int nd, double x, double y, double D,
                     double *out) {
  double f[3] = {(x - 0.15) / 0.60 * nx - 0.5, (y - 0.15) / 0.35 * ny - 0.5,
                 (log2(D) + 4.0) / 8.0 * nd - 0.5};
  int n[3] = {nx, ny, nd}, i0[3], i1[3];
  double t[3];
  for (int a = 0; a < 3; ++a) {
    if (f[a] < 0.0) f[a] = 0.0;
    if (f[a] > n[a] - 1) f[a] = n[a] - 1;
    i0[a] = (int)floor(f[a]);
    i1[a] = i0[a] + 1 > n[a] - 1 ? n[a] - 1 : i0[a] + 1;
    t[a] = f[a] - i0[a];
  }
  out[0] = out[1] = out[2] = 0.0;
  ORC_FETCH(kFetchC, 8);
  for (int c = 0; c < 8; ++c) {
    int ii = (c & 1) ? i1[0] : i0[0], jj = (c & 2) ? i1[1] : i0[1], kk = (c & 4) ? i1[2] : i0[2];
    double w = ((c & 1) ? t[0] : 1.0 - t[0]) * ((c & 2) ? t[1] : 1.0 - t[1]) *
               ((c & 4) ? t[2] : 1.0 - t[2]);
    const double *v = C + (((long)kk * ny + jj) * nx + ii) * 3;
    out[0] += w * v[0]; out[1] += w * v[1]; out[2] += w * v[2];
  }
}

/* ------------------------------------------------------------------------ */
/* Star cube map (Sec. 3.3.2 "Emitted light", reading C15)                    */
/* ------------------------------------------------------------------------ */

/* GL major-axis cube face selection.  Returns face (+x,-x,+y,-y,+z,-z) and
 * the face coordinates sc, tc and |ma|. */
static int cube_face(const double *d, double *sc, double *tc, double *ma) {
  double ax = fabs(d[0]), ay = fabs(d[1]), az = fabs(d[2]);
  if (ax >= ay && ax >= az) {
    *ma = ax;
    if (d[0] >= 0.0) { *sc = -d[2]; *tc = -d[1]; return 0; }
    *sc = d[2]; *tc = -d[1]; return 1;
  }
  if (ay >= az) {
    *ma = ay;
    if (d[1] >= 0.0) { *sc = d[0]; *tc = d[2]; return 2; }
    *sc = d[0]; *tc = -d[2]; return 3;
  }
  *ma = az;
  if (d[2] >= 0.0) { *sc = d[0]; *tc = -d[1]; return 4; }
  *sc = -d[0]; *tc = -d[1]; return 5;
}

/* Round a non-negative double to IEEE half (RNE), saturating at 65504. */
static uint16_t to_half(double v) {
  if (!(v > 0.0)) return 0;
  if (v >= 65504.0) return 0x7bff;
  int e;
  (void)frexp(v, &e); /* v = m 2^e, m in [0.5,1) */
  int E = e - 1;           /* v = (2m) 2^E, 2m in [1,2) */
  if (E < -14) {
    /* subnormal: units of 2^-24 */
    double q = nearbyint(ldexp(v, 24));
    return (uint16_t)q; /* q <= 1024 rolls into the smallest normal exactly */
  }
  double q = nearbyint(ldexp(v, 10 - E)); /* in [1024, 2048] */
  int exp_field = E + 15;
  if (q >= 2048.0) { q = 1024.0; exp_field += 1; }
  if (exp_field >= 31) return 0x7bff;
  return (uint16_t)((exp_field << 10) | ((int)q - 1024));
}
/* Round a non-negative double to bfloat16 (RNE). */
static uint16_t to_bf16(double v) {
  if (!(v > 0.0)) return 0;
  int e;
  (void)frexp(v, &e);
  int E = e - 1;
  if (E < -126) {
    double q = nearbyint(ldexp(v, 133)); /* units of 2^-133 */
    return (uint16_t)q;
  }
  double q = nearbyint(ldexp(v, 7 - E)); /* in [128, 256] */
  int exp_field = E + 127;
  if (q >= 256.0) { q = 128.0; exp_field += 1; }
  if (exp_field >= 255) return 0x7f7f;
  return (uint16_t)((exp_field << 7) | ((int)q - 128));
}
static double from_half(uint16_t h) {
  int ex = (h >> 10) & 31, m = h & 1023;
  if (ex == 0) return ldexp((double)m, -24);
  if (ex == 31) return m ? NAN : INFINITY;
  return ldexp((double)(m + 1024), ex - 25);
}
static double from_bf16(uint16_t h) {
  uint32_t b = (uint32_t)h << 16;
  float f;
  memcpy(&f, &b, 4);
  return (double)f;
}
double orc_decode16(uint16_t h, int dtype) { return dtype == 2 ? from_bf16(h) : from_half(h); }
uint16_t orc_encode16(double v, int dtype) { return dtype == 2 ? to_bf16(v) : to_half(v); }

long long orc_cube_level_offset(int N, int L) {
  long long off = 0;
  for (int l = 0; l < L; ++l) off += 6LL * (N >> l) * (N >> l);
  return off;
}
int orc_cube_levels(int N) {
  int L = 0;
  while ((1 << L) < N) ++L;
  return L + 1;
}

#define XYZ_SCALE 1048576.0 /* fixed point 2^20 for per-star XYZ sums */

/* Emitted XYZ of a synthetic star: luminosity lum (= X+Y+Z) with the
 * chromaticity of a black body at temp_K, rounded to float. */
void orc_star_xyz(double lum, double temp_K, float *xyz) {
  double b[3];
  orc_blackbody_xyz(temp_K, b);
  double s = b[0] + b[1] + b[2];
  for (int c = 0; c < 3; ++c) xyz[c] = (float)(lum * b[c] / s);
}

/* One occupied texel of one level: key = (face*N_L + row)*N_L + column,
 * exact fixed-point X, Y, Z sums and its stored position word.  sub orders
 * the entries of a group: star index at level 0, child number (2 b + a) in
 * the mips, so that every floating-point sum runs in one fixed order. */
typedef struct {
  long long key, sub;
  int64_t x, y, z;
  int64_t ys, yt; /* level 0: sums of Y * (16-bit in-texel position) */
  uint16_t pos;
} cube_entry;

static int entry_cmp(const void *pa, const void *pb) {
  const cube_entry *a = (const cube_entry *)pa, *b = (const cube_entry *)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  if (a->sub != b->sub) return a->sub < b->sub ? -1 : 1;
  return 0;
}

/* Build the star cube map: stars[5*k] = dir x,y,z, luminosity, temperature.
 * Records: 4 uint16 per texel (X, Y, Z as half or bfloat16 of the colour sum
 * divided by 4^L, then the texel-relative position as two unorm8, s in the
 * low byte), all mip levels, level-major, then face, row t, column s.
 * Empty texels: zero colour, position (128, 128). */
int orc_build_cubemap(const float *stars, long long n, int N, int dtype, uint16_t *rec) {
  if (N < 1 || (N & (N - 1))) return 1;
  int nl = orc_cube_levels(N);
  long long total = orc_cube_level_offset(N, nl);
  for (long long t = 0; t < total; ++t) {
    rec[4 * t] = rec[4 * t + 1] = rec[4 * t + 2] = 0;
    rec[4 * t + 3] = (uint16_t)(128 | (128 << 8));
  }
  cube_entry *ent = (cube_entry *)malloc(sizeof(cube_entry) * (size_t)(n > 0 ? n : 1));
  if (!ent) return 2;
  for (long long k = 0; k < n; ++k) {
    const float *st = stars + 5 * k;
    double d[3] = {st[0], st[1], st[2]};
    double sc, tc, ma;
    int f = cube_face(d, &sc, &tc, &ma);
    double S = (sc / ma + 1.0) * 0.5 * N, T = (tc / ma + 1.0) * 0.5 * N;
    int i = (int)floor(S), j = (int)floor(T);
    if (i > N - 1) i = N - 1;
    if (j > N - 1) j = N - 1;
    if (i < 0) i = 0;
    if (j < 0) j = 0;
    double fs = S - i, ft = T - j;
    int64_t s16 = (int64_t)floor(fs * 65536.0), t16 = (int64_t)floor(ft * 65536.0);
    if (s16 > 65535) s16 = 65535;
    if (t16 > 65535) t16 = 65535;
    if (s16 < 0) s16 = 0;
    if (t16 < 0) t16 = 0;
    float xyz[3];
    orc_star_xyz(st[3], st[4], xyz);
    cube_entry *e = ent + k;
    e->key = ((long long)f * N + j) * N + i;
    e->sub = k;
    e->x = (int64_t)nearbyint((double)xyz[0] * XYZ_SCALE);
    e->y = (int64_t)nearbyint((double)xyz[1] * XYZ_SCALE);
    e->z = (int64_t)nearbyint((double)xyz[2] * XYZ_SCALE);
    e->ys = e->y * s16;
    e->yt = e->y * t16;
  }
  qsort(ent, (size_t)n, sizeof(cube_entry), entry_cmp);
  /* level 0: merge each texel's stars */
  long long m = 0;
  for (long long k = 0; k < n;) {
    cube_entry g = ent[k];
    long long q = k + 1;
    for (; q < n && ent[q].key == g.key; ++q) {
      g.x += ent[q].x; g.y += ent[q].y; g.z += ent[q].z;
      g.ys += ent[q].ys; g.yt += ent[q].yt;
    }
    int ps = 128, pt = 128;
    if (g.y > 0) {
      double fs = ((double)g.ys / (double)g.y + 0.5) / 65536.0;
      double ft = ((double)g.yt / (double)g.y + 0.5) / 65536.0;
      ps = (int)floor(fs * 256.0); pt = (int)floor(ft * 256.0);
      if (ps > 255) ps = 255;
      if (pt > 255) pt = 255;
    }
    g.pos = (uint16_t)(ps | (pt << 8));
    uint16_t *r = rec + g.key * 4;
    r[0] = orc_encode16((double)g.x / XYZ_SCALE, dtype);
    r[1] = orc_encode16((double)g.y / XYZ_SCALE, dtype);
    r[2] = orc_encode16((double)g.z / XYZ_SCALE, dtype);
    r[3] = g.pos;
    ent[m++] = g;
    k = q;
  }
  /* mips: colour sum of the 4 children, Y-weighted mean of their positions,
   * children taken in the order (a,b) = (0,0), (1,0), (0,1), (1,1) */
  for (int L = 1; L < nl; ++L) {
    int Np = N >> (L - 1), Nc = N >> L;
    for (long long k = 0; k < m; ++k) {
      long long key = ent[k].key;
      long long f = key / ((long long)Np * Np), rem = key % ((long long)Np * Np);
      long long j = rem / Np, i = rem % Np;
      ent[k].sub = (j & 1) * 2 + (i & 1);
      ent[k].key = (f * Nc + (j >> 1)) * Nc + (i >> 1);
    }
    qsort(ent, (size_t)m, sizeof(cube_entry), entry_cmp);
    double scale = XYZ_SCALE * ldexp(1.0, 2 * L);
    uint16_t *rc = rec + orc_cube_level_offset(N, L) * 4;
    long long mm = 0;
    for (long long k = 0; k < m;) {
      cube_entry g = ent[k];
      double ns = 0.0, nt = 0.0;
      long long q = k;
      g.x = g.y = g.z = 0;
      for (; q < m && ent[q].key == g.key; ++q) {
        const cube_entry *c = ent + q;
        int a = (int)(c->sub & 1), b = (int)(c->sub >> 1);
        double cs = ((c->pos & 255) + 0.5) / 256.0, cq = ((c->pos >> 8) + 0.5) / 256.0;
        ns = ns + (double)c->y * ((a + cs) * 0.5);
        nt = nt + (double)c->y * ((b + cq) * 0.5);
        g.x += c->x; g.y += c->y; g.z += c->z;
      }
      int ps = 128, pt = 128;
      if (g.y > 0) {
        ps = (int)floor(ns / (double)g.y * 256.0);
        pt = (int)floor(nt / (double)g.y * 256.0);
        if (ps > 255) ps = 255;
        if (pt > 255) pt = 255;
      }
      g.pos = (uint16_t)(ps | (pt << 8));
      uint16_t *r = rc + g.key * 4;
      r[0] = orc_encode16((double)g.x / scale, dtype);
      r[1] = orc_encode16((double)g.y / scale, dtype);
      r[2] = orc_encode16((double)g.z / scale, dtype);
      r[3] = g.pos;
      ent[mm++] = g;
      k = q;
    }
    m = mm;
  }
  free(ent);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Camera (Eq. staticbasis, Eq. camerabasis, Eq. d) and the beam (Eq.         */
/* raybasis, Eq. alpha)                                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
  double r, theta, phi;
  double v[3];      /* velocity wrt the static observer, (e_r, e_theta, e_phi) */
  double orient[9]; /* rows: e_w, e_h, e_d in the boosted (r', theta', phi') axes */
  double fov_y;     /* vertical field of view, radians */
  int width, height;
} orc_camera;

typedef struct {
  double r_in, r_out, t_peak, density;
  int enabled;
  /* animated disc (Appendix B): n_particles linear particles, 3 doubles each
   * (u1, u2, phi0), and the coordinate time of the frame at the camera */
  const double *particles;
  int n_particles;
  double time;
} orc_disc;

typedef struct {
  const double *D; int d_n;
  const double *U; int u_ne, u_nphi;
  const double *DT, *UT; /* regularised time channels (may be NULL) */
  const double *C; int c_nx, c_ny, c_nd;
  const double *disc_ln; int disc_n;
  const uint16_t *cube; int cube_n, cube_dtype;
} orc_scene;

typedef struct {
  double u;          /* 1/r of the camera */
  double rhat[3], that[3], phat[3];
  double gamma;
  double E[4][4];    /* E[i] = 4-vector (t,r,theta,phi static components) of e_tau, e_w, e_h, e_d */
  double f;          /* focal length in pixels */
} cam_frame;

static void camera_frame(const orc_camera *c, cam_frame *F) {
  double st = sin(c->theta), ct = cos(c->theta), sp = sin(c->phi), cp = cos(c->phi);
  F->u = 1.0 / c->r;
  F->rhat[0] = st * cp; F->rhat[1] = st * sp; F->rhat[2] = ct;
  F->that[0] = ct * cp; F->that[1] = ct * sp; F->that[2] = -st;
  F->phat[0] = -sp; F->phat[1] = cp; F->phat[2] = 0.0;
  double v2 = c->v[0] * c->v[0] + c->v[1] * c->v[1] + c->v[2] * c->v[2];
  double g = 1.0 / sqrt(1.0 - v2);
  F->gamma = g;
  /* Lorentz boost B(v): e_t' = g (e_t + v.e), e_j' = g v_j e_t + (delta_jk +
   * (g-1) v_j v_k / v^2) e_k. */
  double B[4][4];
  B[0][0] = g;
  for (int k = 0; k < 3; ++k) B[0][1 + k] = g * c->v[k];
  for (int j = 0; j < 3; ++j) {
    B[1 + j][0] = g * c->v[j];
    for (int k = 0; k < 3; ++k)
      B[1 + j][1 + k] = (j == k ? 1.0 : 0.0) + (v2 > 0.0 ? (g - 1.0) * c->v[j] * c->v[k] / v2 : 0.0);
  }
  for (int a = 0; a < 4; ++a) F->E[0][a] = B[0][a];
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < 4; ++a) {
      double s = 0.0;
      for (int j = 0; j < 3; ++j) s += c->orient[i * 3 + j] * B[1 + j][a];
      F->E[1 + i][a] = s;
    }
  F->f = 0.5 * c->height / tan(0.5 * c->fov_y);
}

typedef struct {
  double q[3];      /* normalised [q^w, q^h, -f] */
  double dcart[3];  /* beam direction, pseudo-Cartesian */
  double dcam;      /* gamma (1 + beta . d^) of the camera (energy ratio camera / static) */
  double delta;
  double ey[3], ez[3];
  double alpha;
  int alpha_valid;
} beam;

/* Beam through screen point (qw, qh) (Eq. d, Eq. raybasis, Eq. alpha). */
static void beam_init(const orc_camera *c, const cam_frame *F, double qw, double qh, beam *b) {
  double n = sqrt(qw * qw + qh * qh + F->f * F->f);
  b->q[0] = qw / n; b->q[1] = qh / n; b->q[2] = -F->f / n;
  double k[4];
  for (int a = 0; a < 4; ++a)
    k[a] = -F->E[0][a] + b->q[0] * F->E[1][a] + b->q[1] * F->E[2][a] + b->q[2] * F->E[3][a];
  /* spatial part in the static orthonormal frame; then pseudo-Cartesian */
  double dn = sqrt(k[1] * k[1] + k[2] * k[2] + k[3] * k[3]);
  double vd = c->v[0] * k[1] + c->v[1] * k[2] + c->v[2] * k[3];
  b->dcam = F->gamma * (1.0 + vd / dn);
  double sr = sqrt(1.0 - F->u) * k[1];
  for (int a = 0; a < 3; ++a) b->dcart[a] = sr * F->rhat[a] + k[2] * F->that[a] + k[3] * F->phat[a];
  const double *x = F->rhat;
  const double *d = b->dcart;
  double cr[3] = {x[1] * d[2] - x[2] * d[1], x[2] * d[0] - x[0] * d[2], x[0] * d[1] - x[1] * d[0]};
  double cn = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
  double dd = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  double cosd = x[0] * d[0] + x[1] * d[1] + x[2] * d[2];
  b->delta = atan2(cn, cosd);
  if (cn < 1e-7 * dd) {
    /* reading C8: radial beam, any plane through the radius will do */
    double ax[3] = {0, 0, 0};
    int m = fabs(x[0]) <= fabs(x[1]) ? (fabs(x[0]) <= fabs(x[2]) ? 0 : 2) : (fabs(x[1]) <= fabs(x[2]) ? 1 : 2);
    ax[m] = 1.0;
    cr[0] = x[1] * ax[2] - x[2] * ax[1]; cr[1] = x[2] * ax[0] - x[0] * ax[2];
    cr[2] = x[0] * ax[1] - x[1] * ax[0];
    cn = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
  }
  for (int a = 0; a < 3; ++a) b->ez[a] = cr[a] / cn;
  const double *z = b->ez;
  b->ey[0] = z[1] * x[2] - z[2] * x[1];
  b->ey[1] = z[2] * x[0] - z[0] * x[2];
  b->ey[2] = z[0] * x[1] - z[1] * x[0];
  /* t = +- e_z ^ e_z' / |.|, with t . e_y' >= 0; alpha = arccos(e_x' . t) */
  double t[3] = {-z[1], z[0], 0.0};
  double tn = sqrt(t[0] * t[0] + t[1] * t[1]);
  if (tn < 1e-12) { b->alpha_valid = 0; b->alpha = 0.0; return; } /* reading C9 */
  for (int a = 0; a < 3; ++a) t[a] /= tn;
  if (t[0] * b->ey[0] + t[1] * b->ey[1] + t[2] * b->ey[2] < 0.0)
    for (int a = 0; a < 3; ++a) t[a] = -t[a];
  double ca = x[0] * t[0] + x[1] * t[1] + x[2] * t[2];
  if (ca > 1.0) ca = 1.0;
  if (ca < -1.0) ca = -1.0;
  b->alpha = acos(ca);
  b->alpha_valid = 1;
}

/* For tests: the beam quantities of screen point (qw, qh).
 * out: [0..2] q, [3..5] dcart, [6] dcam, [7] delta, [8..10] ey, [11..13] ez,
 * [14] alpha, [15] alpha_valid. */
void orc_beam(const orc_camera *c, double qw, double qh, double *out) {
  cam_frame F;
  camera_frame(c, &F);
  beam b;
  beam_init(c, &F, qw, qh, &b);
  for (int a = 0; a < 3; ++a) { out[a] = b.q[a]; out[3 + a] = b.dcart[a]; }
  out[6] = b.dcam; out[7] = b.delta;
  for (int a = 0; a < 3; ++a) { out[8 + a] = b.ey[a]; out[11 + a] = b.ez[a]; }
  out[14] = b.alpha; out[15] = b.alpha_valid;
}

/* Doppler factor nu/nu' for a disc hit at u' (reading C12, local form):
 * D = gamma (1 + beta . d^) / (gamma' (1 + beta' . d^')) sqrt(1-u')/sqrt(1-u),
 * beta' = sqrt(u'/(2(1-u'))) along e_phi (prograde circular orbit, Eq. k_prime),
 * beta' . d^' = beta' (u' sqrt(1-u')/e) (e_z . e_z'). */
double orc_disc_doppler(double dcam, double ucam, double e, double up, double ezz) {
  double bp = sqrt(up / (2.0 * (1.0 - up)));
  double gp = 1.0 / sqrt(1.0 - bp * bp);
  double bd = bp * (up * sqrt(1.0 - up) / e) * ezz;
  return dcam / (gp * (1.0 + bd)) * sqrt(1.0 - up) / sqrt(1.0 - ucam);
}

/* Disc temperature, T^4 proportional to u^3 (1 - sqrt(3u)), normalised so
 * that the maximum (at u = 12/49) is t_peak. */
double orc_disc_temperature(double t_peak, double u) {
  double fmax = pow(12.0 / 49.0, 3) * (1.0 - sqrt(36.0 / 49.0));
  double f = u * u * u * (1.0 - sqrt(3.0 * u));
  if (f <= 0.0) return 0.0;
  return t_peak * pow(f / fmax, 0.25);
}

/* ------------------------------------------------------------------------ */
/* Animated disc (Appendix B)                                                 */
/* ------------------------------------------------------------------------ */

/* Complete elliptic integral of the first kind,
 * K(k) = int_0^1 dx / sqrt((1 - x^2)(1 - k^2 x^2)), by the arithmetic-geometric
 * mean (Gauss): K(k) = pi / (2 AGM(1, sqrt(1 - k^2))). */
double orc_ellipk(double k) {
  double a = 1.0, b = sqrt(1.0 - k * k);
  for (int it = 0; it < 64 && fabs(a - b) > 1e-16 * a; ++it) {
    double an = 0.5 * (a + b);
    b = sqrt(a * b);
    a = an;
  }
  return PI / (2.0 * a);
}

/* Point a of the linear particle p = (u1, u2, phi0) at coordinate time t, by
 * the quasi-circular approximation of the precessing massive-particle orbit:
 * phi_a(t) = a + sqrt(ubar^3 / 2) t + phi0, ubar = (u1 + u2) / 2, and
 * u_a(t) = u1 + (u2 - u1) sin^2(pi / (4 K) phi_a(t) sqrt(u3 - u1)),
 * u3 = 1 - u1 - u2, K = K(kappa), kappa^2 = (u2 - u1) / (u3 - u1). */
void orc_particle_point(const double *p, double t, double a, double *u, double *phi) {
  double u1 = p[0], u2 = p[1], u3 = 1.0 - u1 - u2;
  double ub = 0.5 * (u1 + u2);
  double K = orc_ellipk(sqrt((u2 - u1) / (u3 - u1)));
  double ph = a + sqrt(0.5 * ub * ub * ub) * t + p[2];
  double sn = sin(PI / (4.0 * K) * ph * sqrt(u3 - u1));
  *u = u1 + (u2 - u1) * sn * sn;
  *phi = ph;
}

/* Disc density at a hit of coordinate time ht, radius hr and azimuth hphi
 * (Appendix B, readings C23-C24): for every particle, the parameter of the
 * nearest point a = (hphi - phi(ht)) mod 2 pi, the "distance" to the
 * particle centre d^2 = (a/pi - 1)^2 + (hr - 1/u_a(ht))^2 and its
 * contribution (1 - d^2)^2 for d < 1; the density is rho times the sum,
 * clamped to 1. */
double orc_disc_density(const double *particles, int n, double rho, double ht, double hr,
                        double hphi) {
  double sum = 0.0;
  for (int k = 0; k < n; ++k) {
    const double *p = particles + 3 * k;
    double u0, ph0;
    orc_particle_point(p, ht, 0.0, &u0, &ph0); /* ph0 = phi(ht) */
    double a = fmod(hphi - ph0, 2.0 * PI);
    if (a < 0.0) a += 2.0 * PI;
    double ua, pha;
    orc_particle_point(p, ht, a, &ua, &pha);
    double x = a / PI - 1.0, y = hr - 1.0 / ua;
    double d2 = x * x + y * y;
    if (d2 < 1.0) sum += (1.0 - d2) * (1.0 - d2);
  }
  double r = rho * sum;
  return r < 1.0 ? r : 1.0;
}

/* ------------------------------------------------------------------------ */
/* Per-pixel render                                                          */
/* ------------------------------------------------------------------------ */

#define NDBG 29
typedef struct {
  const orc_camera *cam;
  const orc_disc *disc;
  double exposure_disc, exposure_stars;
  const orc_scene *sc;
  cam_frame F;
  double rgbm[9];
  double y_peak;
  int y0, y1, force_level, nthreads;
  double *out, *dbg;
  long long texels[64];
} render_job;

typedef struct {
  beam b;
  double dprime[3];
  int captured;
  double tr[10];
} pix;

static void trace_pixel(render_job *J, int i, int j, pix *p) {
  const orc_camera *c = J->cam;
  double qw = i + 0.5 - 0.5 * c->width, qh = 0.5 * c->height - j - 0.5;
  beam_init(c, &J->F, qw, qh, &p->b);
  double uic = 1.0 / J->disc->r_in, uoc = 1.0 / J->disc->r_out;
  orc_trace_ray2(J->sc->D, J->sc->DT, J->sc->d_n, J->sc->U, J->sc->UT, J->sc->u_ne, J->sc->u_nphi,
                 c->r, p->b.delta, p->b.alpha, p->b.alpha_valid && J->disc->enabled, uic, uoc, p->tr);
  p->captured = isinf(p->tr[0]);
  if (!p->captured) {
    double cd = cos(p->tr[0]), sd = sin(p->tr[0]);
    for (int a = 0; a < 3; ++a) p->dprime[a] = cd * J->F.rhat[a] + sd * p->b.ey[a];
  } else {
    p->dprime[0] = p->dprime[1] = p->dprime[2] = 0.0;
  }
}

static void cross3(const double *a, const double *b, double *o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double *a) { return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

/* Star light gathered over the beam footprint (Sec. 3.3.2), for the pixel
 * whose quad neighbours give the screen-space derivatives (reading C16).
 * Returns XYZ sum in xyz, the mip level, face, and Omega/Omega'. */
static void star_gather(render_job *J, const pix *P, const pix *Pw0, const pix *Pw1,
                        const pix *Ph0, const pix *Ph1, double *xyz, double *dbg,
                        long long *texels) {
  const orc_scene *sc = J->sc;
  xyz[0] = xyz[1] = xyz[2] = 0.0;
  dbg[6] = -1; dbg[7] = -1; dbg[8] = 0; dbg[15] = 0;
  double dw[3], dh[3], qw[3], qh[3];
  for (int a = 0; a < 3; ++a) {
    dw[a] = Pw1->dprime[a] - Pw0->dprime[a];
    dh[a] = Ph0->dprime[a] - Ph1->dprime[a];
    qw[a] = Pw1->b.q[a] - Pw0->b.q[a];
    qh[a] = Ph0->b.q[a] - Ph1->b.q[a];
  }
  double cq[3], cd[3];
  cross3(qw, qh, cq);
  cross3(dw, dh, cd);
  double den = norm3(cd);
  if (!(den > 0.0)) return;
  double omega = norm3(cq) / den; /* Omega / Omega' (Sec. 3.4.1) */
  dbg[8] = omega;
  double sc_, tc_, ma;
  int face = cube_face(P->dprime, &sc_, &tc_, &ma);
  const double *d = P->dprime;
  /* derivative of the major-axis coordinate and of sc, tc along w and h */
  double dmaw, dmah, dscw, dsch, dtcw, dtch;
  switch (face) {
    case 0: dmaw = dw[0]; dmah = dh[0]; dscw = -dw[2]; dsch = -dh[2]; dtcw = -dw[1]; dtch = -dh[1]; break;
    case 1: dmaw = -dw[0]; dmah = -dh[0]; dscw = dw[2]; dsch = dh[2]; dtcw = -dw[1]; dtch = -dh[1]; break;
    case 2: dmaw = dw[1]; dmah = dh[1]; dscw = dw[0]; dsch = dh[0]; dtcw = dw[2]; dtch = dh[2]; break;
    case 3: dmaw = -dw[1]; dmah = -dh[1]; dscw = dw[0]; dsch = dh[0]; dtcw = -dw[2]; dtch = -dh[2]; break;
    case 4: dmaw = dw[2]; dmah = dh[2]; dscw = dw[0]; dsch = dh[0]; dtcw = -dw[1]; dtch = -dh[1]; break;
    default: dmaw = -dw[2]; dmah = -dh[2]; dscw = -dw[0]; dsch = -dh[0]; dtcw = -dw[1]; dtch = -dh[1]; break;
  }
  int N = sc->cube_n;
  double hN = 0.5 * N;
  double S = (sc_ / ma + 1.0) * hN, T = (tc_ / ma + 1.0) * hN;
  /* level-0 texels per screen pixel: J = [dS/dw dS/dh; dT/dw dT/dh] */
  double Jsw = hN * (dscw - sc_ / ma * dmaw) / ma, Jsh = hN * (dsch - sc_ / ma * dmah) / ma;
  double Jtw = hN * (dtcw - tc_ / ma * dmaw) / ma, Jth = hN * (dtch - tc_ / ma * dmah) / ma;
  double hs = fabs(Jsw) + fabs(Jsh), ht = fabs(Jtw) + fabs(Jth);
  double hm = hs > ht ? hs : ht;
  int nl = orc_cube_levels(N);
  {
    /* decision margins, for masking comparisons at discontinuities */
    ORC_COUNT_PAUSE();
    double a[3] = {fabs(d[0]), fabs(d[1]), fabs(d[2])}, mx = a[0], sd = -1.0;
    for (int k = 1; k < 3; ++k) if (a[k] > mx) mx = a[k];
    for (int k = 0; k < 3; ++k) if (a[k] < mx && a[k] > sd) sd = a[k];
    int nmax = (a[0] == mx) + (a[1] == mx) + (a[2] == mx);
    dbg[16] = hm;
    dbg[17] = nmax > 1 ? 0.0 : 1.0 - sd / mx;
    ORC_COUNT_RESUME();
  }
  int L = 0;
  if (J->force_level >= 0) L = J->force_level;
  else
    while (L < nl - 1 && 2.0 * hm > 8.0 * ldexp(1.0, L)) ++L; /* reading C17 */
  dbg[6] = L; dbg[7] = face;
  double sL = ldexp(1.0, -L);
  int NL = N >> L;
  double cS = S * sL, cT = T * sL, hsL = hs * sL, htL = ht * sL;
  double a11 = Jsw * sL, a12 = Jsh * sL, a21 = Jtw * sL, a22 = Jth * sL;
  double det = a11 * a22 - a12 * a21;
  /* reading C18: skip a degenerate footprint */
  ORC_COUNT_PAUSE();
  dbg[18] = fabs(det) / sqrt((a11 * a11 + a21 * a21) * (a12 * a12 + a22 * a22));
  ORC_COUNT_RESUME();
  if (!(fabs(det) > 1e-6 * sqrt((a11 * a11 + a21 * a21) * (a12 * a12 + a22 * a22)))) return;
  double i11 = a22 / det, i12 = -a12 / det, i21 = -a21 / det, i22 = a11 / det;
  int i0 = (int)floor(cS - hsL), i1 = (int)floor(cS + hsL);
  int j0 = (int)floor(cT - htL), j1 = (int)floor(cT + htL);
  if (i0 < 0) i0 = 0;
  if (j0 < 0) j0 = 0;
  if (i1 > NL - 1) i1 = NL - 1;
  if (j1 > NL - 1) j1 = NL - 1;
  const uint16_t *rec = sc->cube + (orc_cube_level_offset(N, L) + (long long)face * NL * NL) * 4;
  double lscale = ldexp(1.0, 2 * L);
  long long cnt = 0;
  double gw = 0.0, gh = 0.0, ysum = 0.0; /* for the sensitivity to a footprint shift */
  for (int jj = j0; jj <= j1; ++jj)
    for (int ii = i0; ii <= i1; ++ii) {
      ++cnt;
      const uint16_t *r = rec + ((long long)jj * NL + ii) * 4;
      ORC_FETCH(kFetchCube, 1);
      ORC_TOUCH(orc_cube_level_offset(N, L) + (long long)face * NL * NL + (long long)jj * NL + ii,
                (r[0] | r[1] | r[2]) != 0);
      ORC_COUNT_PAUSE(); /* decoding a record is bit work, not arithmetic */
      double X = orc_decode16(r[0], sc->cube_dtype), Y = orc_decode16(r[1], sc->cube_dtype),
             Z = orc_decode16(r[2], sc->cube_dtype);
      ORC_COUNT_RESUME();
      if (X + Y + Z <= 0.0) continue;
      double ps = ((r[3] & 255) + 0.5) / 256.0, pt = ((r[3] >> 8) + 0.5) / 256.0;
      double ds = ii + ps - cS, dt = jj + pt - cT;
      double w = i11 * ds + i12 * dt, h = i21 * ds + i22 * dt;
      double fw = 1.0 - fabs(w), fh = 1.0 - fabs(h);
      if (fw <= 0.0 || fh <= 0.0) continue;
      double wt = fw * fh * lscale;
      xyz[0] += wt * X; xyz[1] += wt * Y; xyz[2] += wt * Z;
      ORC_COUNT_PAUSE();
      ysum += wt * Y;
      gw += (w > 0.0 ? 1.0 : -1.0) * fh * lscale * Y; /* d/d(shift in w) of the Y sum */
      gh += (h > 0.0 ? 1.0 : -1.0) * fw * lscale * Y;
      ORC_COUNT_RESUME();
    }
  ORC_COUNT_PAUSE();
  dbg[15] = (double)cnt;
  dbg[19] = ysum > 0.0 ? sqrt(gw * gw + gh * gh) / ysum : 0.0;
  ORC_COUNT_RESUME();
  *texels += cnt;
}

static void render_pixel(render_job *J, int i, int j, pix *quad[2][2], double *out, double *dbg,
                         long long *texels) {
  /* quad[b][a]: a = column parity, b = row parity */
  int a = i & 1, b = j & 1;
  const pix *P = quad[b][a];
  const orc_camera *c = J->cam;
  double d[NDBG];
  for (int k = 0; k < NDBG; ++k) d[k] = 0.0;
  d[0] = P->tr[6];
  d[1] = P->b.delta;
  d[2] = P->captured ? INFINITY : P->tr[0];
  d[3] = P->tr[1];
  d[4] = P->tr[2];
  d[5] = P->tr[4];
  d[23] = P->tr[8]; /* retarded time (camera minus emission) of hit slot 0 */
  d[24] = P->tr[9];
  /* disc hits, front to back (Sec. 3.3.3, reading C13) */
  double L[3] = {0, 0, 0};
  double trans = 1.0;
  double e = sqrt(P->tr[6]);
  for (int h = 0; h < (int)P->tr[1]; ++h) {
    double up = P->tr[2 + 2 * h];
    /* the hit point: at angle psi from e_x' towards e_y' in the ray plane
     * (its azimuth is needed only by the animated disc) */
    double rho = J->disc->density, hphi = 0.0;
    if (J->disc->n_particles <= 0) ORC_COUNT_PAUSE();
    double psi = P->tr[3 + 2 * h], hd[3];
    for (int k = 0; k < 3; ++k) hd[k] = cos(psi) * J->F.rhat[k] + sin(psi) * P->b.ey[k];
    hphi = atan2(hd[1], hd[0]);
    if (J->disc->n_particles <= 0) ORC_COUNT_RESUME();
    if (J->disc->n_particles > 0) /* animated disc: emitted at the retarded time (App. B) */
      rho = orc_disc_density(J->disc->particles, J->disc->n_particles, J->disc->density,
                             J->disc->time - P->tr[8 + h], 1.0 / up, hphi);
    d[25 + h] = rho;
    d[27 + h] = hphi;
    double T = orc_disc_temperature(J->disc->t_peak, up);
    double D = orc_disc_doppler(P->b.dcam, J->F.u, e, up, P->b.ez[2]);
    d[13 + h] = D;
    double xyz[3];
    disc_xyz(J->sc->disc_ln, J->sc->disc_n, D * T, xyz);
    double s = rho * J->exposure_disc / J->y_peak;
    for (int k = 0; k < 3; ++k) L[k] += trans * s * xyz[k];
    trans *= 1.0 - rho;
  }
  /* stars: zero if any quad member is captured (reading C16) */
  int anycap = quad[0][0]->captured || quad[0][1]->captured || quad[1][0]->captured ||
               quad[1][1]->captured;
  if (!anycap && J->sc->cube) {
    double sxyz[3];
    star_gather(J, P, quad[b][0], quad[b][1], quad[0][a], quad[1][a], sxyz, d, texels);
    d[10] = sxyz[0]; d[11] = sxyz[1]; d[12] = sxyz[2];
    double S = sxyz[0] + sxyz[1] + sxyz[2];
    double Dst = P->b.dcam / sqrt(1.0 - J->F.u); /* static star, u' = 0 */
    d[9] = Dst;
    if (S > 0.0) {
      double cc[3];
      c_lookup(J->sc->C, J->sc->c_nx, J->sc->c_ny, J->sc->c_nd, sxyz[0] / S, sxyz[1] / S, Dst, cc);
      double s = S * d[8] * J->exposure_stars;
      for (int k = 0; k < 3; ++k) L[k] += trans * s * cc[k];
      /* bound on the change of each linear-RGB channel per screen pixel of
       * footprint shift: |d sum/d shift| / sum (channel 19) times the star
       * light seen through |M| (the XYZ -> RGB matrix mixes signs) */
      ORC_COUNT_PAUSE();
      for (int c = 0; c < 3; ++c)
        d[20 + c] = d[19] * trans * s *
                    (fabs(J->rgbm[c * 3 + 0] * cc[0]) + fabs(J->rgbm[c * 3 + 1] * cc[1]) +
                     fabs(J->rgbm[c * 3 + 2] * cc[2]));
      ORC_COUNT_RESUME();
    }
  } else {
    d[6] = -1; d[7] = -1;
  }
  for (int r = 0; r < 3; ++r)
    out[r] = J->rgbm[r * 3 + 0] * L[0] + J->rgbm[r * 3 + 1] * L[1] + J->rgbm[r * 3 + 2] * L[2];
  out[3] = 1.0;
  if (dbg)
    for (int k = 0; k < NDBG; ++k) dbg[k] = d[k];
  (void)c;
}

typedef struct { render_job *J; int tid; } worker_arg;

static void *render_worker(void *argp) {
  worker_arg *w = (worker_arg *)argp;
  render_job *J = w->J;
  const orc_camera *c = J->cam;
  int W = c->width;
  long long texels = 0;
  pix *row[2][2];
  pix *buf = (pix *)malloc(sizeof(pix) * 4);
  for (int qy = J->y0 / 2 + w->tid; 2 * qy < J->y1; qy += J->nthreads) {
    for (int qx = 0; 2 * qx < W; ++qx) {
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          row[b][a] = buf + b * 2 + a;
          trace_pixel(J, 2 * qx + a, 2 * qy + b, row[b][a]);
        }
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          int i = 2 * qx + a, j = 2 * qy + b;
          if (i >= W || j >= c->height || j < J->y0 || j >= J->y1) continue;
          long long o = (long long)(j - J->y0) * W + i;
          render_pixel(J, i, j, row, J->out + 4 * o, J->dbg ? J->dbg + NDBG * o : NULL, &texels);
        }
    }
  }
  free(buf);
  J->texels[w->tid] = texels;
  ORC_COUNT_FLUSH();
  return NULL;
}

/* Render image rows [y0, y1) (y0 even) into out (rows y0.. first; RGBA
 * doubles) and optionally per-pixel debug values (NDBG doubles per pixel):
 *  0 e^2, 1 delta, 2 delta' (inf if captured), 3 hits, 4 u0, 5 u1,
 *  6 mip level (-1: no star term), 7 face, 8 Omega/Omega', 9 star Doppler,
 *  10..12 gathered star XYZ, 13 hit-0 Doppler, 14 hit-1 Doppler,
 *  15 texels visited, 16 footprint half extent (level-0 texels),
 *  17 face margin 1 - second/major axis, 18 |det J| / (|J_w| |J_h|),
 *  19 |gradient| of the star sum's Y per pixel of footprint shift, relative
 *     to that sum, 20..22 resulting bound on the change of R, G, B per pixel
 *     of footprint shift, 23..24 retarded times of the two hit slots,
 *  25..26 disc density of the two hit slots, 27..28 their azimuths.
 * force_level >= 0 forces the mip level (for the flat-space checks). */
int orc_render(const orc_camera *cam, const orc_disc *disc, double exposure_disc,
               double exposure_stars, const orc_scene *sc, int y0, int y1, int force_level,
               int nthreads, double *out, double *dbg, long long *texels_visited) {
  if (y0 < 0 || (y0 & 1) || y1 > cam->height || y1 <= y0) return 1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 64) nthreads = 64;
  render_job J;
  memset(&J, 0, sizeof(J));
  J.cam = cam; J.disc = disc; J.exposure_disc = exposure_disc; J.exposure_stars = exposure_stars;
  J.sc = sc; J.y0 = y0; J.y1 = y1; J.force_level = force_level; J.nthreads = nthreads;
  J.out = out; J.dbg = dbg;
  ORC_COUNT_PAUSE(); /* per-frame constants: not per-pixel work */
  camera_frame(cam, &J.F);
  orc_xyz_to_rgb_matrix(J.rgbm);
  double yp[3];
  disc_xyz(sc->disc_ln, sc->disc_n, disc->t_peak, yp);
  J.y_peak = yp[1] > 0.0 ? yp[1] : 1.0;
  ORC_COUNT_RESUME();
  pthread_t th[64];
  worker_arg args[64];
  for (int t = 0; t < nthreads; ++t) {
    args[t].J = &J; args[t].tid = t;
    if (nthreads == 1) render_worker(&args[t]);
    else pthread_create(&th[t], NULL, render_worker, &args[t]);
  }
  if (nthreads > 1)
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  long long tot = 0;
  for (int t = 0; t < nthreads; ++t) tot += J.texels[t];
  if (texels_visited) *texels_visited = tot;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Brute-force ray: table-free integration of the 3D photon orbit            */
/* x'' = -3/2 h^2 x / |x|^5, h = |x ^ x'| (Cartesian form of Eq. rayequation) */
/* ------------------------------------------------------------------------ */

/* State: position (0..2), velocity (3..5) with respect to the affine
 * parameter lambda, and coordinate time (6): along a null geodesic
 * dt/dlambda = E / (1 - 1/r), with E^2 = |x'|^2 - h^2 / r^3 conserved. */
static void orbit_deriv(const double *s, double h2, double E, double *ds) {
  double r2 = s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
  double r = sqrt(r2);
  double k = -1.5 * h2 / (r2 * r2 * r);
  ds[0] = s[3]; ds[1] = s[4]; ds[2] = s[5];
  ds[3] = k * s[0]; ds[4] = k * s[1]; ds[5] = k * s[2];
  ds[6] = E / (1.0 - 1.0 / r);
}
static void orbit_rk4(const double *s, double h2, double E, double dl, double *o) {
  double k1[7], k2[7], k3[7], k4[7], t[7];
  orbit_deriv(s, h2, E, k1);
  for (int a = 0; a < 7; ++a) t[a] = s[a] + 0.5 * dl * k1[a];
  orbit_deriv(t, h2, E, k2);
  for (int a = 0; a < 7; ++a) t[a] = s[a] + 0.5 * dl * k2[a];
  orbit_deriv(t, h2, E, k3);
  for (int a = 0; a < 7; ++a) t[a] = s[a] + dl * k3[a];
  orbit_deriv(t, h2, E, k4);
  for (int a = 0; a < 7; ++a) o[a] = s[a] + dl / 6.0 * (k1[a] + 2 * k2[a] + 2 * k3[a] + k4[a]);
}

/* x0: pseudo-Cartesian position, d0: pseudo-Cartesian direction.
 * out (17 doubles): [0..2] escape direction (0 if captured), [3] captured,
 * [4] number of disc crossings with r_in <= r <= r_out (at most 4 recorded),
 * [5..8] their u, [9..12] the coordinate time from the camera back to each
 * crossing, [13..16] the crossing's azimuth atan2(y, x). */
int orc_bruteforce_ray(const double *x0, const double *d0, double r_in, double r_out,
                       double step, double *out) {
  double s[7];
  double dn = norm3(d0);
  for (int a = 0; a < 3; ++a) { s[a] = x0[a]; s[3 + a] = d0[a] / dn; }
  s[6] = 0.0;
  double hv[3];
  cross3(s, s + 3, hv);
  double h2 = hv[0] * hv[0] + hv[1] * hv[1] + hv[2] * hv[2];
  double r0 = norm3(x0);
  double E = sqrt(1.0 - h2 / (r0 * r0 * r0)); /* |x'| = 1 at the start */
  for (int a = 0; a < 17; ++a) out[a] = 0.0;
  int nh = 0;
  for (long it = 0; it < 50000000L; ++it) {
    double r = norm3(s);
    if (r < 1.0 + 1e-9) { out[3] = 1.0; break; }
    double rd = (s[0] * s[3] + s[1] * s[4] + s[2] * s[5]) / r;
    if (r > 1e7 && rd > 0.0) {
      double vn = norm3(s + 3);
      for (int a = 0; a < 3; ++a) out[a] = s[3 + a] / vn;
      break;
    }
    double dl = step * r;
    if (r < 2.0 && dl > step * (r - 1.0) + 1e-6) dl = step * (r - 1.0) + 1e-6;
    double n[7];
    orbit_rk4(s, h2, E, dl, n);
    if ((s[2] > 0.0) != (n[2] > 0.0) && s[2] != 0.0) {
      /* disc plane crossing: bisection on the step length */
      double lo = 0.0, hi = dl, m[7];
      for (int k = 0; k < 100; ++k) {
        double mid = 0.5 * (lo + hi);
        orbit_rk4(s, h2, E, mid, m);
        if ((m[2] > 0.0) == (s[2] > 0.0)) lo = mid; else hi = mid;
      }
      orbit_rk4(s, h2, E, 0.5 * (lo + hi), m);
      double rc = norm3(m);
      if (rc >= r_in && rc <= r_out) {
        if (nh < 4) {
          out[5 + nh] = 1.0 / rc;
          out[9 + nh] = m[6];
          out[13 + nh] = atan2(m[1], m[0]);
        }
        ++nh;
      }
    }
    for (int a = 0; a < 7; ++a) s[a] = n[a];
  }
  out[4] = nh;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Free-fall camera orbit (Appendix C)                                        */
/* ------------------------------------------------------------------------ */

typedef struct {
  double t, r, psi, rdot; /* coordinate time, radius, angle in the orbital plane, dr/dtau */
  double e, l;            /* constants of motion */
  double chi;             /* inclination of the orbital plane */
} orc_orbit;

/* Constants of motion from the initial radius, direction and speed (App. C):
 * e^2 = (1 - u0)/(1 - v0^2), l^2 = (e^2 + u0 - 1)/(u0^2 (1 - u0 + cot^2 delta0));
 * dr/dtau from (dr/dtau)^2 = e^2 + l^2 u^3 - l^2 u^2 + u - 1, outward if
 * delta0 < pi/2. */
int orc_orbit_init(double r0, double delta0, double v0, double chi, orc_orbit *o) {
  if (!(r0 > 1.0) || !(v0 >= 0.0 && v0 < 1.0)) return 1;
  double u = 1.0 / r0;
  double e2 = (1.0 - u) / (1.0 - v0 * v0);
  double cot = cos(delta0) / sin(delta0);
  double l2 = (e2 + u - 1.0) / (u * u * (1.0 - u + cot * cot));
  o->t = 0.0; o->r = r0; o->psi = 0.0; o->chi = chi;
  o->e = sqrt(e2);
  o->l = sqrt(l2 > 0.0 ? l2 : 0.0);
  double rd2 = e2 + l2 * u * u * u - l2 * u * u + u - 1.0;
  o->rdot = (delta0 < PI / 2 ? 1.0 : -1.0) * sqrt(rd2 > 0.0 ? rd2 : 0.0);
  return 0;
}

static void orbit_rhs(const orc_orbit *o, const double *y, double *dy) {
  double u = 1.0 / y[1], l2 = o->l * o->l;
  dy[0] = o->e / (1.0 - u);
  dy[1] = y[3];
  dy[2] = o->l * u * u;
  dy[3] = 0.5 * (2.0 * l2 * u * u * u - 3.0 * l2 * u * u * u * u - u * u);
}

/* Advance by dtau of proper time in n RK4 steps (App. C: d^2r/dtau^2 =
 * (2 l^2 u^3 - 3 l^2 u^4 - u^2)/2, dpsi/dtau = l u^2, dt/dtau = e/(1-u)). */
void orc_orbit_advance(orc_orbit *o, double dtau, int n) {
  double h = dtau / n;
  for (int s = 0; s < n; ++s) {
    double y[4] = {o->t, o->r, o->psi, o->rdot}, k1[4], k2[4], k3[4], k4[4], z[4];
    orbit_rhs(o, y, k1);
    for (int a = 0; a < 4; ++a) z[a] = y[a] + 0.5 * h * k1[a];
    orbit_rhs(o, z, k2);
    for (int a = 0; a < 4; ++a) z[a] = y[a] + 0.5 * h * k2[a];
    orbit_rhs(o, z, k3);
    for (int a = 0; a < 4; ++a) z[a] = y[a] + h * k3[a];
    orbit_rhs(o, z, k4);
    o->t = y[0] + h / 6.0 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0]);
    o->r = y[1] + h / 6.0 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1]);
    o->psi = y[2] + h / 6.0 * (k1[2] + 2 * k2[2] + 2 * k3[2] + k4[2]);
    o->rdot = y[3] + h / 6.0 * (k1[3] + 2 * k2[3] + 2 * k3[3] + k4[3]);
  }
}

/* Camera of an orbit state (App. C): position from
 * r (cos chi cos psi, sin psi, sin chi cos psi), velocity wrt the static
 * observer v = [ (dr/dtau)/e , 0 , l u sqrt(1-u)/e ] on (e_r, e_chi, e_psi),
 * and the rotation to (e_r, e_theta, e_phi): e_chi = a e_theta + b e_phi,
 * e_psi = -b e_theta + a e_phi, with e_chi the unit normal e_psi ^ e_r =
 * (sin chi, 0, -cos chi), so a = sin chi cos theta cos phi + cos chi sin theta
 * and b = -sin chi sin phi (reading C22).  The user rotation O is given on the
 * boosted (r', chi', psi') axes and is returned on (r', theta', phi').
 * out: [0] r, [1] theta, [2] phi, [3..5] v on (e_r, e_theta, e_phi),
 * [6..14] orientation rows on (r', theta', phi'). */
void orc_orbit_camera(const orc_orbit *o, const double *orient_rcp, double *out) {
  double th = acos(cos(o->psi) * sin(o->chi));
  double ph = atan2(sin(o->psi), cos(o->chi) * cos(o->psi));
  double u = 1.0 / o->r;
  double a = sin(o->chi) * cos(th) * cos(ph) + cos(o->chi) * sin(th);
  double b = -sin(o->chi) * sin(ph);
  double vr = o->rdot / o->e, vpsi = o->l * u * sqrt(1.0 - u) / o->e;
  out[0] = o->r; out[1] = th; out[2] = ph;
  out[3] = vr; out[4] = -b * vpsi; out[5] = a * vpsi;
  for (int i = 0; i < 3; ++i) {
    const double *Or = orient_rcp + 3 * i; /* (r', chi', psi') components */
    out[6 + 3 * i + 0] = Or[0];
    out[6 + 3 * i + 1] = a * Or[1] - b * Or[2];
    out[6 + 3 * i + 2] = b * Or[1] + a * Or[2];
  }
}
