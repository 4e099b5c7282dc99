// alpha_regen.cu -- the recompute storage mode (Sec. 3.2, Eq. probnewfac):
// gamma^x_t(x) = exp(2 pi i y'.xi_c) / N * sum_c A(x, xi_c) (V S^-1)[c][t] is
// formed again in every apply from the sampled columns xi_c of each wedge and
// the r x q matrix V S^-1 that the plan keeps, instead of being stored for
// every x (L N^2 q values).  The result has the stored mode's layout, so the
// interpolation and spread kernels read it unchanged.
//
// A(x, xi) = a(x, xi) exp(2 pi i Phi_l(x, xi)), with the residual phase
// Phi_l(x, xi) = Psi(x, xi) - grad Psi(x, xihat_l) . xi (Psi = Phi - x.xi).  The
// plan forms it in FP64 as Phi(x, xi) - y'.M xi mod 1, which cancels O(N)
// cycles.  Complex64 plans here use forms of Phi_l in which nothing cancels, so
// that single precision keeps its relative accuracy (ct, st: the wedge's
// centre direction xihat_l; d = theta - theta_l):
//  - ellipse, Psi = sqrt(a xi1^2 + b xi2^2), (a, b) = (c1^2, c2^2): with
//    rho_l = sqrt(a ct^2 + b st^2), Psi^2 rho_l^2 - (a ct xi1 + b st xi2)^2 =
//    a b (ct xi2 - st xi1)^2, so
//    Phi_l = a b (ct xi2 - st xi1)^2 / (rho_l (Psi rho_l + a ct xi1 + b st xi2));
//  - tau modes, Psi = |xi| Re sum_m C_m(x) e^{i m theta}:
//    Phi_l = Re sum_m C_m(x) G_m(xi), G_m = |xi| e^{i m theta_l}
//    (e^{i m d} - cos d - i m sin d), made per column in FP64 on the host;
//  - shift / wave multiplier: Phi_l = c (ct xi2 - st xi1)^2 / (|xi| + ct xi1 + st xi2),
//    which does not depend on x (made on the host).
// Beyond single-precision rounding, the one difference from the plan's entries
// is the 32-bit rounding of the warped point y' the plan used (at most
// 2^-33 |M xi| cycles, 1e-6 rad at N = 2048).
//
// FP64 plans form the plan's own entries (phase_eval.cuh) in the plan's order.
#include <cuda_runtime.h>

#include <cstdint>

#include "fio_internal.h"
#include "phase_eval.cuh"

namespace fio {

namespace {

constexpr int kRgThreads = 256;

// Terms t0 .. t0 + QC - 1 of every point: acc_t = sum_k A(x, xi_k) W[k][t].
// KIND: the phase kind (only the tau kind holds the 17 C_m(x) in registers).
template <int QC, int KIND>
__global__ void __launch_bounds__(kRgThreads, 2)
k_regen_f32(PhaseDev ph, int N, const WedgeDev *__restrict__ Wd, int l0, int L,
            const uint2 *__restrict__ warps, const uint32_t *__restrict__ perm,
            const RcCol *__restrict__ cols, const float2 *__restrict__ G,
            const float2 *__restrict__ Wm, const float2 *__restrict__ xf,
            float2 *__restrict__ alpha) {
  const int l = l0 + blockIdx.y;
  const WedgeDev &w = Wd[l];
  const long long NN = (long long)N * N;
  const long long pos = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= NN) return;
  const long long x = perm[(long long)l * NN + pos];
  const uint2 Y = warps[(long long)l * NN + pos];
  // centre factor exp(2 pi i y'.xi_c) / N from the exact 32-bit product
  const uint32_t yk = Y.x * (uint32_t)w.xc1 + Y.y * (uint32_t)w.xc2;
  float cs, cc;
  sincospif(2.0f * ((float)yk * 2.3283064365386962890625e-10f), &cs, &cc);
  const float invN = 1.0f / (float)N;
  const float2 ctr = make_float2(cc * invN, cs * invN);
  // per-x data
  float ax = 1.0f;
  if (ph.amp_kind == FIO_AMP_SEPARABLE)
    ax = 1.0f + (float)ph.a1 * sinpif(2.0f * (float)(x / N) / (float)N);
  float ea = 0.f, eb = 0.f, rho = 0.f;
  float2 C[KIND == FIO_PHASE_TAU_MODES ? pe::kNm : 1];
  if constexpr (KIND == FIO_PHASE_ELLIPSE) {
    const float2 v = xf[x];
    ea = v.x;
    eb = v.y;
    float st, ct;
    sincospif(2.0f * (float)l / (float)L, &st, &ct);
    rho = sqrtf(ea * ct * ct + eb * st * st);
  } else if constexpr (KIND == FIO_PHASE_TAU_MODES) {
#pragma unroll
    for (int m = 0; m < pe::kNm; ++m) C[m] = xf[x * pe::kNm + m];
  }
  const RcCol *cl = cols + w.rc_col_off;
  const float2 *gl = G ? G + w.rc_col_off * pe::kNm : nullptr;
  float2 *out = alpha + w.alpha_off + pos * w.qp;
  // A(x, xi_k) for column k: amplitude times exp(2 pi i Phi_l)
  auto entry = [&](int k) -> float2 {
    const RcCol c = cl[k];
    float R = 0.f;
    if constexpr (KIND == FIO_PHASE_ELLIPSE) {
      const float psi = sqrtf(ea * c.fk1 * c.fk1 + eb * c.fk2 * c.fk2);
      const float den = rho * (psi * rho + ea * c.ctk1 + eb * c.stk2);
      R = den > 0.f ? __fdividef(ea * eb * c.cross2, den) : 0.f;  // xi = 0: Phi_l = 0
    } else if constexpr (KIND == FIO_PHASE_TAU_MODES) {
      const float2 *gk = gl + (long long)k * pe::kNm;
#pragma unroll
      for (int m = 0; m < pe::kNm; ++m) {
        const float2 g = gk[m];
        R = fmaf(C[m].x, g.x, fmaf(-C[m].y, g.y, R));
      }
    } else {
      R = c.rsw;
    }
    float s, co;
    sincospif(2.0f * R, &s, &co);
    const float amp = ax * c.ampc;
    return make_float2(amp * co, amp * s);
  };
  for (int t0 = 0; t0 < w.qp; t0 += QC) {
    float2 acc[QC];
#pragma unroll
    for (int j = 0; j < QC; ++j) acc[j] = make_float2(0.f, 0.f);
    // two columns per step, so that one entry's phase and sine overlap the other's
    int k = 0;
    for (; k + 1 < w.rc_r; k += 2) {
      const float2 e0 = entry(k), e1 = entry(k + 1);
      const float2 *wr = Wm + w.rc_w_off + (long long)k * w.qp + t0;
#pragma unroll
      for (int j = 0; j < QC; ++j) {
        if (t0 + j < w.qp) {
          const float2 v0 = wr[j], v1 = wr[w.qp + j];
          acc[j].x = fmaf(e0.x, v0.x, fmaf(-e0.y, v0.y, acc[j].x));
          acc[j].y = fmaf(e0.x, v0.y, fmaf(e0.y, v0.x, acc[j].y));
          acc[j].x = fmaf(e1.x, v1.x, fmaf(-e1.y, v1.y, acc[j].x));
          acc[j].y = fmaf(e1.x, v1.y, fmaf(e1.y, v1.x, acc[j].y));
        }
      }
    }
    if (k < w.rc_r) {
      const float2 e = entry(k);
      const float2 *wr = Wm + w.rc_w_off + (long long)k * w.qp + t0;
#pragma unroll
      for (int j = 0; j < QC; ++j) {
        if (t0 + j < w.qp) {
          const float2 v = wr[j];
          acc[j].x = fmaf(e.x, v.x, fmaf(-e.y, v.y, acc[j].x));
          acc[j].y = fmaf(e.x, v.y, fmaf(e.y, v.x, acc[j].y));
        }
      }
    }
#pragma unroll
    for (int j = 0; j < QC; ++j)
      if (t0 + j < w.qp)
        out[t0 + j] = make_float2(acc[j].x * ctr.x - acc[j].y * ctr.y,
                                  acc[j].x * ctr.y + acc[j].y * ctr.x);
  }
}

// FP64 plans: the plan's own entries and order (as the plan forms A_[C] and then
// gamma^x), terms in chunks of QC.
template <int QC>
__global__ void __launch_bounds__(kRgThreads)
k_regen_f64(PhaseDev ph, int N, const WedgeDev *__restrict__ Wd, int l0,
            const uint2 *__restrict__ warps, const uint32_t *__restrict__ perm,
            const RcCol *__restrict__ cols, const double2 *__restrict__ Wm, const void *xd,
            double2 *__restrict__ alpha) {
  const int l = l0 + blockIdx.y;
  const WedgeDev &w = Wd[l];
  const long long NN = (long long)N * N;
  const long long pos = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= NN) return;
  const long long x = perm[(long long)l * NN + pos];
  const uint2 Y = warps[(long long)l * NN + pos];
  const uint32_t yk = Y.x * (uint32_t)w.xc1 + Y.y * (uint32_t)w.xc2;
  double s, c;
  sincospi(2.0 * ((double)yk * 2.3283064365386962890625e-10), &s, &c);
  const double invN = 1.0 / N;
  const double2 ctr = make_double2(c * invN, s * invN);
  const pe::XView xv = pe::xview(ph, xd);
  const RcCol *cl = cols + w.rc_col_off;
  double2 *out = alpha + w.alpha_off + pos * w.qp;
  for (int t0 = 0; t0 < w.qp; t0 += QC) {
    double2 acc[QC];
#pragma unroll
    for (int j = 0; j < QC; ++j) acc[j] = make_double2(0.0, 0.0);
    for (int k = 0; k < w.rc_r; ++k) {
      const double2 a = pe::entry(ph, xv, N, w, x, Y, cl[k].k1, cl[k].k2);
      const double2 *wr = Wm + w.rc_w_off + (long long)k * w.qp + t0;
#pragma unroll
      for (int j = 0; j < QC; ++j) {
        if (t0 + j < w.qp) {
          const double2 b = wr[j];
          acc[j].x += a.x * b.x - a.y * b.y;
          acc[j].y += a.x * b.y + a.y * b.x;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < QC; ++j)
      if (t0 + j < w.qp)
        out[t0 + j] = make_double2(acc[j].x * ctr.x - acc[j].y * ctr.y,
                                   acc[j].x * ctr.y + acc[j].y * ctr.x);
  }
}

__global__ void k_xdata_f32(PhaseDev ph, long long NN, const double2 *__restrict__ xd,
                            float2 *__restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (ph.kind == FIO_PHASE_ELLIPSE) {
    if (i >= NN) return;
    const double2 c = xd[i];
    out[i] = make_float2((float)(c.x * c.x), (float)(c.y * c.y));
  } else if (ph.kind == FIO_PHASE_TAU_MODES) {
    if (i >= NN * pe::kNm) return;
    out[i] = make_float2((float)xd[i].x, (float)xd[i].y);
  }
}

}  // namespace

cudaError_t regen_alpha(const fio_plan_s *p, int g, cudaStream_t s) {
  const int l0 = p->grp_first[g], nw = p->grp_first[g + 1] - l0;
  const long long NN = (long long)p->N * p->N;
  const dim3 grid((unsigned)((NN + kRgThreads - 1) / kRgThreads), (unsigned)nw);
  if (p->precision == FIO_FP64)
    k_regen_f64<8><<<grid, kRgThreads, 0, s>>>(p->phase, p->N, p->d_wedges_rc, l0, p->d_warps,
                                              p->d_perm, p->d_rc_col, (const double2 *)p->d_rc_w,
                                              p->d_rc_x, (double2 *)p->d_alpha);
  else {
    auto go = [&](auto kern) {
      kern<<<grid, kRgThreads, 0, s>>>(p->phase, p->N, p->d_wedges_rc, l0, p->L, p->d_warps,
                                        p->d_perm, p->d_rc_col, (const float2 *)p->d_rc_g,
                                        (const float2 *)p->d_rc_w, (const float2 *)p->d_rc_x,
                                        (float2 *)p->d_alpha);
    };
    if (p->phase.kind == FIO_PHASE_ELLIPSE) go(k_regen_f32<24, FIO_PHASE_ELLIPSE>);
    else if (p->phase.kind == FIO_PHASE_TAU_MODES) go(k_regen_f32<24, FIO_PHASE_TAU_MODES>);
    else go(k_regen_f32<24, FIO_PHASE_SHIFT_WAVE>);
  }
  return cudaGetLastError();
}

cudaError_t rc_xdata_f32(const PhaseDev &ph, const void *d_xdata64, int N, void *d_out,
                         cudaStream_t s) {
  const long long NN = (long long)N * N;
  const long long n = ph.kind == FIO_PHASE_TAU_MODES ? NN * pe::kNm : NN;
  if (ph.kind != FIO_PHASE_ELLIPSE && ph.kind != FIO_PHASE_TAU_MODES) return cudaSuccess;
  k_xdata_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ph, NN, (const double2 *)d_xdata64,
                                                         (float2 *)d_out);
  return cudaGetLastError();
}

}  // namespace fio
