// phase_eval.cuh -- FP64 device evaluation of the phase and amplitude of the
// FIO kernel a(x, xi) exp(2 pi i Phi(x, xi)) (Eq. dfio) and of the residual
// kernel entries A_{x,xi} of one wedge (Eq. probform).  Shared by the plan's
// kernels and by the regeneration of gamma^x in the recompute storage mode, so
// that both form the same entries.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "fio_internal.h"

namespace fio {
namespace pe {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kMmax = kTauMmax;  // tau modes: m in [-8, 8]
constexpr int kNm = 2 * kMmax + 1;

static __device__ __forceinline__ int imodp(long long a, int n) {
  long long r = a % n;
  return (int)(r < 0 ? r + n : r);
}

// Per-x phase data: ellipse axes (c1, c2), or the tau modes grouped by m:
// C_m(x) = sum_{j : m_j = m} a_j exp(i (2 pi k_j.x + p_j)), so that
// tau(x, theta) = Re sum_m C_m(x) exp(i m theta) (an exact regrouping).
struct XView {
  const double2 *ell;   // [x] (c1, c2)
  const double2 *Cm;    // [x][kNm]
};

static __device__ __forceinline__ XView xview(const PhaseDev &ph, const void *xd) {
  XView v{nullptr, nullptr};
  if (ph.kind == FIO_PHASE_ELLIPSE) v.ell = (const double2 *)xd;
  if (ph.kind == FIO_PHASE_TAU_MODES) v.Cm = (const double2 *)xd;
  return v;
}

// sum_m C_m e^{i m theta} and sum_m m C_m e^{i m theta}, with e = e^{i theta}.
static __device__ __forceinline__ void tau_sums(const double2 *C, double ec, double es, double2 &S,
                                         double2 &Sm) {
  S = C[kMmax];
  Sm = make_double2(0.0, 0.0);
  double pc = 1.0, ps = 0.0;  // e^{i m theta}
  for (int m = 1; m <= kMmax; ++m) {
    const double nc = pc * ec - ps * es, ns = pc * es + ps * ec;
    pc = nc;
    ps = ns;
    const double2 Cp = C[kMmax + m], Cn = C[kMmax - m];
    // C_m e^{i m th} + C_{-m} e^{-i m th}
    const double2 tp = make_double2(Cp.x * pc - Cp.y * ps, Cp.x * ps + Cp.y * pc);
    const double2 tn = make_double2(Cn.x * pc + Cn.y * ps, Cn.y * pc - Cn.x * ps);
    S.x += tp.x + tn.x;
    S.y += tp.y + tn.y;
    Sm.x += m * (tp.x - tn.x);
    Sm.y += m * (tp.y - tn.y);
  }
}

// Psi(x, xi) = Phi(x, xi) - x.xi
static __device__ __forceinline__ double psi(const PhaseDev &ph, const XView &xv, long long x, int k1,
                                      int k2) {
  if (k1 == 0 && k2 == 0) return 0.0;
  const double d1 = k1, d2 = k2;
  const double r = sqrt(d1 * d1 + d2 * d2);
  switch (ph.kind) {
    case FIO_PHASE_SHIFT_WAVE:
      return -(ph.p[0] * d1 + ph.p[1] * d2) + ph.p[2] * r;
    case FIO_PHASE_ELLIPSE: {
      const double2 c = xv.ell[x];
      return sqrt(c.x * c.x * d1 * d1 + c.y * c.y * d2 * d2);
    }
    case FIO_PHASE_TAU_MODES: {
      double2 S, Sm;
      tau_sums(xv.Cm + x * kNm, d1 / r, d2 / r, S, Sm);
      return r * S.x;
    }
  }
  return 0.0;
}

// grad_xi Psi at the unit vector (ct, st).
static __device__ __forceinline__ void grad_psi_unit(const PhaseDev &ph, const XView &xv, long long x,
                                              double ct, double st, double &g1, double &g2) {
  switch (ph.kind) {
    case FIO_PHASE_SHIFT_WAVE:
      g1 = -ph.p[0] + ph.p[2] * ct;
      g2 = -ph.p[1] + ph.p[2] * st;
      return;
    case FIO_PHASE_ELLIPSE: {
      const double2 c = xv.ell[x];
      const double a = c.x * c.x, b = c.y * c.y;
      const double rho = sqrt(a * ct * ct + b * st * st);
      g1 = a * ct / rho;
      g2 = b * st / rho;
      return;
    }
    case FIO_PHASE_TAU_MODES: {
      // grad(|xi| tau) = tau xihat + (d tau / d theta) xihat_perp
      double2 S, Sm;
      tau_sums(xv.Cm + x * kNm, ct, st, S, Sm);
      const double tau = S.x, dtau = -Sm.y;  // Re(i sum m C_m e^{i m th}) = -Im(sum m ...)
      g1 = tau * ct - dtau * st;
      g2 = tau * st + dtau * ct;
      return;
    }
  }
  g1 = g2 = 0.0;
}

// a(x, xi) as a complex number; ps = Phi(x, xi) - x.xi (read by the Hankel kind).
// Hankel (Appendix A, Eq. ellipses_amp): s = a1, rho = s ps,
// a = (J0(2 pi rho) + i s Y0(2 pi rho)) exp(-2 pi i s rho) / (4 pi), without the
// Y0 term where rho <= 0 (xi = 0, where Y0 is singular).
static __device__ __forceinline__ double2 amp(const PhaseDev &ph, double x1, int k1, int k2, double ps) {
  if (ph.amp_kind == FIO_AMP_SEPARABLE) {
    const double r = sqrt((double)k1 * k1 + (double)k2 * k2);
    const double cth = r > 0 ? k1 / r : 1.0;
    return make_double2((1.0 + ph.a1 * sinpi(2.0 * x1)) * (1.0 + ph.a2 * cth), 0.0);
  }
  if (ph.amp_kind == FIO_AMP_HANKEL) {
    const double s = ph.a1, rho = s * ps;
    const double z = 2.0 * 3.141592653589793238462643383279502884 * rho;
    const double jr = j0(z), yi = rho > 0 ? s * y0(z) : 0.0;
    double sn, cn;
    sincospi(-2.0 * s * rho, &sn, &cn);
    const double k = 1.0 / (4.0 * 3.141592653589793238462643383279502884);
    return make_double2(k * (jr * cn - yi * sn), k * (jr * sn + yi * cn));
  }
  return make_double2(1.0, 0.0);
}

// A_{x,xi} = a(x,xi) exp(2 pi i [Phi(x,xi) - y'.(M xi)]) with y' the 32-bit
// fraction Y / 2^32 (its integer part only adds integers to the phase).
// x.xi mod 1 and y'.(M xi) mod 1 are formed exactly in integer arithmetic.
static __device__ __forceinline__ double2 entry(const PhaseDev &ph, const XView &xv, int N,
                                         const WedgeDev &w, long long x, uint2 Y, int k1,
                                         int k2) {
  const int n1 = (int)(x / N), n2 = (int)(x % N);
  const int xx = imodp((long long)n1 * k1 + (long long)n2 * k2, N);
  const int kk1 = w.M[0] * k1 + w.M[1] * k2, kk2 = w.M[2] * k1 + w.M[3] * k2;
  const uint32_t yk = Y.x * (uint32_t)kk1 + Y.y * (uint32_t)kk2;  // mod 2^32
  const double frac = (double)xx / N - (double)yk * 2.3283064365386962890625e-10;
  const double ps = psi(ph, xv, x, k1, k2);
  const double phase = frac + ps;
  double s, c;
  sincospi(2.0 * phase, &s, &c);
  const double2 a = amp(ph, (double)n1 / N, k1, k2, ps);
  return make_double2(a.x * c - a.y * s, a.x * s + a.y * c);
}

}  // namespace pe
}  // namespace fio
