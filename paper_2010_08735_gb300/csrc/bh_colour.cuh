// Colour definitions on the device, FP64 (Sec. 3.4.2).
//
// The observer is this project's piecewise-Gaussian colour matching
// functions (in the functional form of Wyman, Sloan and Shirley, JCGT 2013);
// black bodies are integrated on a 5 nm trapezoid grid from 360 to 830 nm.
// The arithmetic is written with explicit round-to-nearest intrinsics where
// the result feeds an integer decision (star binning), so that no
// multiply-add contraction changes the rounding.
#pragma once

#include "bh_internal.cuh"

namespace bh {

__device__ __forceinline__ double dlobe(double l, double m, double s1, double s2) {
  double t = __ddiv_rn(__dadd_rn(l, -m), l < m ? s1 : s2);
  return exp(__dmul_rn(-0.5, __dmul_rn(t, t)));
}

__device__ __forceinline__ void dcmf(double l, double *c) {
  c[0] = __dadd_rn(__dadd_rn(__dmul_rn(1.056, dlobe(l, 599.8, 37.9, 31.0)),
                             __dmul_rn(0.362, dlobe(l, 442.0, 16.0, 26.7))),
                   -__dmul_rn(0.065, dlobe(l, 501.1, 20.4, 26.2)));
  c[1] = __dadd_rn(__dmul_rn(0.821, dlobe(l, 568.8, 46.9, 40.5)),
                   __dmul_rn(0.286, dlobe(l, 530.9, 16.3, 31.1)));
  c[2] = __dadd_rn(__dmul_rn(1.217, dlobe(l, 437.0, 11.8, 36.0)),
                   __dmul_rn(0.681, dlobe(l, 459.0, 26.0, 13.8)));
}

// Planck's law up to a constant factor; lambda in nm.
__device__ __forceinline__ double dplanck(double l, double T) {
  const double c2 = 1.4387769e7;  // h c / k, nm K
  double l2 = __dmul_rn(l, l);
  double l5 = __dmul_rn(__dmul_rn(l2, l2), l);
  return __ddiv_rn(1.0, __dmul_rn(l5, expm1(__ddiv_rn(c2, __dmul_rn(l, T)))));
}

// XYZ of a black body; cmf[3*k..] holds the matching functions at 360 + 5k nm.
__device__ __forceinline__ void dblackbody_xyz(const double *cmf, double T, double *xyz) {
  xyz[0] = xyz[1] = xyz[2] = 0.0;
  if (!(T > 0.0)) return;
  for (int k = 0; k < kNLambda; ++k) {
    double l = 360.0 + 5.0 * k;
    double w = (k == 0 || k == kNLambda - 1) ? 2.5 : 5.0;
    double b = __dmul_rn(dplanck(l, T), w);
    xyz[0] = __dadd_rn(xyz[0], __dmul_rn(b, cmf[3 * k + 0]));
    xyz[1] = __dadd_rn(xyz[1], __dmul_rn(b, cmf[3 * k + 1]));
    xyz[2] = __dadd_rn(xyz[2], __dmul_rn(b, cmf[3 * k + 2]));
  }
}

}  // namespace bh
