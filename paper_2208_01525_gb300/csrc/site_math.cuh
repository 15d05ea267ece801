// Per-site arithmetic of the U(1)xU(1) leapfrog (Sec. III, Eqs. 17-26), of
// the gauge-invariant plaquette windings (Sec. III.A) and of the diagnostic
// densities (Eqs. 33, 36-37), shared by every kernel variant.  The callers
// gather the neighbourhood values (from global memory, shared memory or
// registers) and these functions only compute.
#pragma once

#include <math.h>

#include "sincos_table.cuh"
#include "u1u1_internal.cuh"

namespace u1u1 {

template <typename T> __device__ __forceinline__ void sincos_t(T x, T* s, T* c);
template <> __device__ __forceinline__ void sincos_t<float>(float x, float* s, float* c) { sincosf(x, s, c); }
template <> __device__ __forceinline__ void sincos_t<double>(double x, double* s, double* c) { sincos(x, s, c); }

// cos and sin of a link angle theta = dx A.  FP32: reduction to
// r = theta - 2 pi k, k = rint(theta / 2 pi), |r| <= pi, with 2 pi split into
// two floats (Cody & Waite 1980) and fused multiply-adds, then the hardware
// sine and cosine (__sincosf, documented absolute error below 2^-21.41 on
// [-pi, pi]; measured 3.6e-7 here).  That is about 6 ulp at 1: the step's
// FP32 tolerance (field max-rel 1e-5 against FP64 after 20 steps) leaves
// room for it, and the Gauss constraint does not depend on it (the same U is
// used in the Laplacian and in the current).  It made the step 3% and a
// measuring step 8% faster than a Taylor series on [-pi/4, pi/4].  FP64 uses
// the library sincos.
template <typename T> __device__ __forceinline__ void link_sincos(T x, T* s, T* c);
template <> __device__ __forceinline__ void link_sincos<float>(float x, float* s, float* c) {
  const float k = rintf(x * 0.159154943091895335769f);
  float r = fmaf(-k, 6.28318548202514648f, x);  // fl(2 pi)
  r = fmaf(-k, -1.74845553e-07f, r);            // 2 pi - fl(2 pi)
  __sincosf(r, s, c);
}
// FP64: the table-driven method (Tang 1989).  theta = m h + r with
// h = 2 pi / 1024, m = rint(theta / h) and |r| <= h / 2 (h split in two
// doubles so that m h1 is exact); sin(m h) and cos(m h) from the table of
// sincos_table.cuh, indexed by m mod 1024; sin r = r - r^3/6 + r^5/120 and
// cos r - 1 = -r^2/2 + r^4/24 (truncation below 6e-22 and 1.2e-18 at
// |r| <= 3.1e-3), combined by the angle-addition formulas with cos r - 1
// kept apart so that nothing cancels.  About 14 FP64 operations against the
// library sincos' larger count, on a step that is bound by GB300's FP64
// rate; within two ulp of the exact values (tested against a correctly
// rounded reference).  Arguments beyond the exact range of the reduction
// (|theta| > 5e4, far outside any link angle of a run) take the library
// sincos.
template <> __device__ __forceinline__ void link_sincos<double>(double x, double* s, double* c) {
  if (fabs(x) > SINCOS_TAB_MAX_ARG) {
    sincos(x, s, c);
    return;
  }
  const double m = rint(x * SINCOS_TAB_INV_H);
  double r = fma(-m, SINCOS_TAB_H1, x);
  r = fma(-m, SINCOS_TAB_H2, r);
  const int j = (int)((long long)m & (SINCOS_TAB_N - 1));
  const double2 t = __ldg(&k_sincos_tab[j]);  // {sin(m h), cos(m h)}
  const double r2 = r * r;
  const double sr = fma(r * r2, fma(r2, 1.0 / 120.0, -1.0 / 6.0), r);
  const double cm1 = r2 * fma(r2, 1.0 / 24.0, -0.5);
  *s = fma(t.y, sr, fma(t.x, cm1, t.x));
  *c = fma(-t.x, sr, fma(t.y, cm1, t.y));
}


template <typename T> __device__ __forceinline__ T rint_t(T x);
template <> __device__ __forceinline__ float rint_t<float>(float x) { return rintf(x); }
template <> __device__ __forceinline__ double rint_t<double>(double x) { return rint(x); }

template <typename T> struct Consts;
template <> struct Consts<float> {
  static __device__ __forceinline__ float pi() { return 3.14159265358979323846f; }
  static __device__ __forceinline__ float inv_two_pi() { return 0.159154943091895335769f; }
};
template <> struct Consts<double> {
  static __device__ __forceinline__ double pi() { return 3.14159265358979323846; }
  static __device__ __forceinline__ double inv_two_pi() { return 0.159154943091895335769; }
};

// U phi with U = exp(-i theta) = (c, -s):  (c + (-s) i)(a + b i)
template <typename T>
__device__ __forceinline__ void transport_fwd(T c, T s, T a, T b, T* re, T* im) {
  *re = c * a + s * b;
  *im = c * b - s * a;
}
// conj(U) phi = (c + s i)(a + b i)
template <typename T>
__device__ __forceinline__ void transport_bwd(T c, T s, T a, T b, T* re, T* im) {
  *re = c * a - s * b;
  *im = c * b + s * a;
}

// Everything one sector's site update needs.
template <typename T>
struct SectorIn {
  T fr, fi;            // phi(x)
  T fwr[3], fwi[3];    // U_i(x) phi(x+i)
  T bwr[3], bwi[3];    // conj(U_i(x-i)) phi(x-i)
  T F[3];              // dx F_01, dx F_02, dx F_12 at x
  T Fm[6];             // dx F at: 01(x-y), 01(x-x), 02(x-z), 02(x-x), 12(x-z), 12(x-y)
  T A[3];              // A_i(x)
};

// plaquette curl dx*F_ij(x) = A_j(x+i) - A_j(x) - A_i(x+j) + A_i(x)
template <typename T>
__device__ __forceinline__ T curl_ft(T Aj_xpi, T Aj_x, T Ai_xpj, T Ai_x) {
  return (Aj_xpi - Aj_x) - (Ai_xpj - Ai_x);
}

// Scalar kick, Eq. 17/18, for sector s; r_self and r_other are
// |phi_s|^2 - sigma_s^2 and |phi_o|^2 - sigma_o^2.
template <typename T>
__device__ __forceinline__ void scalar_kick(const SectorIn<T>& in, T r_self, T r_other, T pr, T pi,
                                            const Coef<T>& c, int s, T* pr_new, T* pi_new) {
  T sr = (in.fwr[0] + in.bwr[0]) + (in.fwr[1] + in.bwr[1]) + (in.fwr[2] + in.bwr[2]) - T(6) * in.fr;
  T si = (in.fwi[0] + in.bwi[0]) + (in.fwi[1] + in.bwi[1]) + (in.fwi[2] + in.bwi[2]) - T(6) * in.fi;
  T g = c.kgl[s] * r_self - c.kgk * r_other;
  *pr_new = c.kPa * pr + c.kP1 * sr - g * in.fr;
  *pi_new = c.kPa * pi + c.kP1 * si - g * in.fi;
}

// Im[phi^*(x) U_i(x) phi(x+i)] for each direction.
template <typename T>
__device__ __forceinline__ T current_im(const SectorIn<T>& in, int i) {
  return in.fr * in.fwi[i] - in.fi * in.fwr[i];
}
template <typename T>
__device__ __forceinline__ T current_re(const SectorIn<T>& in, int i) {
  return in.fr * in.fwr[i] + in.fi * in.fwi[i];
}

// Gauge kick, Eq. 20/21, for sector s.
template <typename T>
__device__ __forceinline__ void gauge_kick(const SectorIn<T>& in, const T E[3], const Coef<T>& c,
                                           int s, T En[3]) {
  T C0 = (in.F[0] - in.Fm[0]) + (in.F[1] - in.Fm[2]);
  T C1 = (in.F[2] - in.Fm[4]) - (in.F[0] - in.Fm[1]);
  T C2 = -(in.F[1] - in.Fm[3]) - (in.F[2] - in.Fm[5]);
  En[0] = c.kEa * E[0] - c.kE1 * C0 + c.kE2[s] * current_im(in, 0);
  En[1] = c.kEa * E[1] - c.kE1 * C1 + c.kE2[s] * current_im(in, 1);
  En[2] = c.kEa * E[2] - c.kE1 * C2 + c.kE2[s] * current_im(in, 2);
}

// arg(re + i im) in [-pi, pi] in FP32 for the edge phases.  Octant
// reduction t = min(|re|, |im|) / max(|re|, |im|) in [0, 1], the minimax
// odd polynomial atan(t) ~ t P(t^2) of degree 15 (Remez exchange, derived by
// fit_atan.py; 3.7e-8 in exact arithmetic, 3.1e-7 rad measured in FP32),
// then the octant, half-plane and sign fix-ups: pi/2 - r when |im| > |re|,
// pi - r when re carries a minus sign (so arg(+-0 - 0 i) = +-pi), and the
// sign of im.  A winding only needs the four edge phases of a plaquette to
// within pi in total, and the branch is decided by the signs of re and im
// exactly; the accuracy kept here makes the cut flag agree with a
// correctly rounded arctangent except within rounding of its threshold.
__device__ __forceinline__ float edge_phase_f32(float re, float im) {
  const float ax = fabsf(re), ay = fabsf(im);
  const float mn = fminf(ax, ay), mx = fmaxf(ax, ay);
  const float t = mx > 0.0f ? __fdividef(mn, mx) : 0.0f;
  const float s = t * t;
  float p = fmaf(s, -4.054567212e-03f, 2.186295787e-02f);
  p = fmaf(s, p, -5.591232676e-02f);
  p = fmaf(s, p, 9.642197328e-02f);
  p = fmaf(s, p, -1.390862955e-01f);
  p = fmaf(s, p, 1.994656565e-01f);
  p = fmaf(s, p, -3.332986078e-01f);
  p = fmaf(s, p, 9.999993356e-01f);
  float r = t * p;
  r = ay > ax ? 1.57079632679489662f - r : r;
  r = signbit(re) ? 3.14159265358979324f - r : r;
  return copysignf(r, im);
}

template <typename T> __device__ __forceinline__ T edge_phase(T re, T im);
template <> __device__ __forceinline__ float edge_phase<float>(float re, float im) { return edge_phase_f32(re, im); }
template <> __device__ __forceinline__ double edge_phase<double>(double re, double im) { return atan2(im, re); }

// Edge phase chi = arg(Re + i Im) and its branch-cut flag (pi - |chi| < 1e-4
// or a zero product).
template <typename T>
__device__ __forceinline__ T edge_chi(T re, T im, bool* cut) {
  T chi = edge_phase<T>(re, im);
  if (Consts<T>::pi() - fabs(chi) < T(1e-4) || (re == T(0) && im == T(0))) *cut = true;
  return chi;
}

// Winding of one plaquette from its four edge phases and dx F.
template <typename T>
__device__ __forceinline__ int plaquette_winding(T chi_i_x, T chi_j_xpi, T chi_i_xpj, T chi_j_x,
                                                 T dx, T Ft) {
  T tot = (chi_i_x + chi_j_xpi) - (chi_i_xpj + chi_j_x) + dx * Ft;
  return (int)rint_t<T>(tot * Consts<T>::inv_two_pi());
}

// Diagnostic densities of one sector (Sec. III.A):
// kin = (|pi-|^2 + |pi+|^2)/2, grad = sum |D+ phi|^2,
// el = sum (E-^2 + E+^2)/2 / (2 e^2 c), mag = sum F^2 / (2 e^2 c).
template <typename T>
struct SectorDiag {
  T kin, grad, el, mag;
};
template <typename T>
__device__ __forceinline__ SectorDiag<T> sector_diag(const SectorIn<T>& in, T pr, T pi, T prn,
                                                     T pin, const T E[3], const T En[3],
                                                     const Coef<T>& c, int s) {
  SectorDiag<T> d;
  d.kin = T(0.5) * ((pr * pr + pi * pi) + (prn * prn + pin * pin));
  T g = T(0);
  for (int i = 0; i < 3; ++i) {
    T a = in.fwr[i] - in.fr, b = in.fwi[i] - in.fi;
    g += a * a + b * b;
  }
  d.grad = c.inv_dx2 * g;
  T e2 = T(0.5) * ((E[0] * E[0] + En[0] * En[0]) + (E[1] * E[1] + En[1] * En[1]) +
                   (E[2] * E[2] + En[2] * En[2]));
  d.el = c.el_f[s] * e2;
  d.mag = c.mag_f[s] * (in.F[0] * in.F[0] + in.F[1] * in.F[1] + in.F[2] * in.F[2]);
  return d;
}

}  // namespace u1u1
