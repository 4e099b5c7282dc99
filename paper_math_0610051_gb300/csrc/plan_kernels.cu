// plan_kernels.cu -- FP64 device kernels of the preprocessing step (Sec. 3.2):
// warped points y_l(x) = grad_xi Phi(x, xihat_l) (Sec. 1.4), entries of the
// residual kernel A_{x,xi} = a(x,xi) exp(2 pi i Phi_l(x,xi)) (Eq. probform) at
// sampled columns and rows, the triangular factor of A_[C] (Householder TSQR),
// and the factors gamma^x = U = A_[C] V S^-1 and gamma^xi = T = U_[R]^+ A_[R].
//
// Everything here is double precision: the residual phase cancels O(N) terms
// (Sec. 1.3), and the warped points are reduced modulo 1 to 32-bit fractions
// before any lower-precision use.
#include <cuda_runtime.h>

#include <cstdint>

#include "fio_internal.h"
#include "phase_eval.cuh"

namespace fio {

using namespace pe;

namespace {

// ------------------------------------------------------------------ kernels --

__global__ void k_xdata(PhaseDev ph, const double *__restrict__ modes, int N, void *xd) {
  const long long NN = (long long)N * N;
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= NN) return;
  const double x1 = (double)(x / N) / N, x2 = (double)(x % N) / N;
  if (ph.kind == FIO_PHASE_ELLIPSE) {
    double2 c;
    if (ph.ell_form == 1) {  // product-form axes of Eq. nrphase's experiments
      c.x = ph.p[1] * (ph.p[0] + sinpi(4.0 * x1)) * (ph.p[0] + sinpi(4.0 * x2));
      c.y = ph.p[3] * (ph.p[2] + cospi(4.0 * x1)) * (ph.p[2] + cospi(4.0 * x2));
    } else {
      c.x = ph.p[0] + ph.p[1] * sinpi(2.0 * x1) * sinpi(2.0 * x2);
      c.y = ph.p[2] + ph.p[3] * cospi(2.0 * x1) * cospi(2.0 * x2);
    }
    ((double2 *)xd)[x] = c;
  } else if (ph.kind == FIO_PHASE_TAU_MODES) {
    double2 C[kNm];
    for (int m = 0; m < kNm; ++m) C[m] = make_double2(0.0, 0.0);
    for (int j = 0; j < ph.nmodes; ++j) {
      const double *p = modes + 5 * j;
      const int m = (int)llrint(p[3]);
      double s, c;
      sincos(kTwoPi * (p[1] * x1 + p[2] * x2) + p[4], &s, &c);
      C[m + kMmax].x += p[0] * c;
      C[m + kMmax].y += p[0] * s;
    }
    double2 *out = (double2 *)xd + x * kNm;
    for (int m = 0; m < kNm; ++m) out[m] = C[m];
  }
}

__global__ void k_warp(PhaseDev ph, const void *xd, int N, int L, const WedgeDev *__restrict__ W,
                       uint2 *__restrict__ warp) {
  const long long NN = (long long)N * N;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= NN * L) return;
  const int l = (int)(idx / NN);
  const long long x = idx % NN;
  const WedgeDev w = W[l];
  const XView xv = xview(ph, xd);
  double st, ct;
  sincospi(2.0 * l / L, &st, &ct);  // xihat_l = (cos 2 pi l / L, sin 2 pi l / L)
  double g1, g2;
  grad_psi_unit(ph, xv, x, ct, st, g1, g2);
  const double y1 = (double)(x / N) / N + g1, y2 = (double)(x % N) / N + g2;
  // y'.xi'' = y.xi with xi = Minv xi''  =>  y' = Minv^T y
  const double yp[2] = {w.Minv[0] * y1 + w.Minv[2] * y2, w.Minv[1] * y1 + w.Minv[3] * y2};
  uint32_t Y[2];
  for (int d = 0; d < 2; ++d) {
    const double f = yp[d] - floor(yp[d]);
    const double s = rint(f * 4294967296.0);
    Y[d] = s >= 4294967296.0 ? 0u : (uint32_t)s;
  }
  warp[idx] = make_uint2(Y[0], Y[1]);
}

__global__ void k_eval_cols(PhaseDev ph, const void *xd, int N, WedgeDev w,
                            const uint2 *__restrict__ warp_l, const int *__restrict__ ck1,
                            const int *__restrict__ ck2, int r, double2 *__restrict__ AC) {
  const long long NN = (long long)N * N;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= NN * r) return;
  const long long x = idx / r;
  const int c = (int)(idx % r);
  AC[idx] = entry(ph, xview(ph, xd), N, w, x, warp_l[x], ck1[c], ck2[c]);
}

// Householder QR of the row panels of a tall matrix `in` (rows x r, row-major),
// the first step of the tall-skinny QR (TSQR) of A_[C].  CTA p copies rows
// [p P, p P + h) into its own region of `work` and reduces them to upper
// triangular form with h' = min(h, r) reflectors H_k = I - u u^H (u^H u = 2, u
// zero above row k; u is kept in column k, R_kk in rdiag).  It writes its r x r
// factor R_p (zero below the diagonal and in rows >= h') to Rout[p].  Stacking
// the R_p and factoring the stack again gives the R of the whole matrix; the Q
// factors are never formed.
//
// Threads: lane -> column j (stride 32), warp -> row group i = k + warp (stride
// 8), so the reads of a row are coalesced and u_i is a broadcast.
constexpr int kQrThreads = 256;
constexpr int kQrGroups = kQrThreads / 32;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__global__ void __launch_bounds__(kQrThreads)
k_panel_qr(const double2 *__restrict__ in, long long rows, int r, int P, double2 *__restrict__ work,
           double2 *__restrict__ Rout) {
  extern __shared__ double2 qsm[];
  double2 *dots = qsm;                // [kQrGroups][r] partial u^H a_j, then the sums in row 0
  double2 *rdiag = dots + kQrGroups * r;
  __shared__ double red[kQrGroups];
  __shared__ double s_scale;
  const long long row0 = (long long)blockIdx.x * P;
  const int h = (int)min((long long)P, rows - row0);
  double2 *a = work + row0 * r;
  const double2 *src = in + row0 * r;
  const long long ne = (long long)h * r;
  for (long long e = threadIdx.x; e < ne; e += kQrThreads) a[e] = src[e];
  __syncthreads();
  const int lane = threadIdx.x & 31, rg = threadIdx.x >> 5;
  const int kmax = min(h, r);
  for (int k = 0; k < kmax; ++k) {
    double s2 = 0.0;
    for (int i = k + threadIdx.x; i < h; i += kQrThreads) {
      const double2 v = a[(long long)i * r + k];
      s2 += v.x * v.x + v.y * v.y;
    }
    s2 = warp_sum_d(s2);
    if (lane == 0) red[rg] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sig2 = 0.0;
      for (int w = 0; w < kQrGroups; ++w) sig2 += red[w];
      const double sigma = sqrt(sig2);
      const double2 x0 = a[(long long)k * r + k];
      const double ax0 = hypot(x0.x, x0.y);
      if (sigma == 0.0) {
        rdiag[k] = make_double2(0.0, 0.0);
        s_scale = 0.0;
      } else {
        // alpha = -phase(x0) sigma: no cancellation in x0 - alpha
        const double2 ph = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
        const double2 alpha = make_double2(-ph.x * sigma, -ph.y * sigma);
        const double sc = 1.0 / sqrt(sigma * (sigma + ax0));  // u = (x - alpha e1) sc, u^H u = 2
        rdiag[k] = alpha;
        a[(long long)k * r + k] = make_double2((x0.x - alpha.x) * sc, (x0.y - alpha.y) * sc);
        s_scale = sc;
      }
    }
    __syncthreads();
    const double sc = s_scale;
    if (sc == 0.0) continue;  // a zero column: H_k = I (uniform across the CTA)
    for (int i = k + 1 + threadIdx.x; i < h; i += kQrThreads) {
      double2 &v = a[(long long)i * r + k];
      v = make_double2(v.x * sc, v.y * sc);
    }
    __syncthreads();
    // w_j = u^H a_j for the trailing columns
    for (int j = k + 1 + lane; j < r; j += 32) {
      double2 acc = make_double2(0.0, 0.0);
      for (int i = k + rg; i < h; i += kQrGroups) {
        const double2 u = a[(long long)i * r + k], v = a[(long long)i * r + j];
        acc.x += u.x * v.x + u.y * v.y;
        acc.y += u.x * v.y - u.y * v.x;
      }
      dots[rg * r + j] = acc;
    }
    __syncthreads();
    for (int j = k + 1 + threadIdx.x; j < r; j += kQrThreads) {
      double2 sum = dots[j];
      for (int g = 1; g < kQrGroups; ++g) {
        const double2 v = dots[g * r + j];
        sum.x += v.x;
        sum.y += v.y;
      }
      dots[j] = sum;
    }
    __syncthreads();
    // a_j -= u w_j
    for (int j = k + 1 + lane; j < r; j += 32) {
      const double2 wj = dots[j];
      for (int i = k + rg; i < h; i += kQrGroups) {
        const double2 u = a[(long long)i * r + k];
        double2 &v = a[(long long)i * r + j];
        v.x -= u.x * wj.x - u.y * wj.y;
        v.y -= u.x * wj.y + u.y * wj.x;
      }
    }
    __syncthreads();
  }
  double2 *R = Rout + (long long)blockIdx.x * r * r;
  for (int e = threadIdx.x; e < r * r; e += kQrThreads) {
    const int i = e / r, j = e - (e / r) * r;
    double2 v = make_double2(0.0, 0.0);
    if (i < kmax && j >= i) v = j == i ? rdiag[i] : a[(long long)i * r + j];
    R[e] = v;
  }
}

template <typename C>
__device__ __forceinline__ void store_c(void *base, long long i, double2 v) {
  if constexpr (sizeof(C) == 8) ((float2 *)base)[i] = make_float2((float)v.x, (float)v.y);
  else ((double2 *)base)[i] = v;
}

template <typename C>
__global__ void k_form_alpha(const double2 *__restrict__ AC, int N, int r, int q,
                             const double2 *__restrict__ Wm, WedgeDev w,
                             const uint2 *__restrict__ warp_l, const uint32_t *__restrict__ perm_l,
                             void *alpha_l) {
  const long long NN = (long long)N * N;
  const long long pos = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= NN) return;
  const long long x = perm_l[pos];  // alpha is stored in the sorted point order [pos][t]
  // centre-frequency factor exp(2 pi i y'.xi_c) / N (Sec. 3.4), exact mod 1
  const uint2 Y = warp_l[x];
  const uint32_t yk = Y.x * (uint32_t)w.xc1 + Y.y * (uint32_t)w.xc2;
  double s, c;
  sincospi(2.0 * ((double)yk * 2.3283064365386962890625e-10), &s, &c);
  const double invN = 1.0 / N;
  const double2 ctr = make_double2(c * invN, s * invN);
  const double2 *row = AC + x * r;
  for (int t = 0; t < q; ++t) {
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < r; ++k) {
      const double2 a = row[k], b = Wm[k * q + t];
      acc.x += a.x * b.x - a.y * b.y;
      acc.y += a.x * b.y + a.y * b.x;
    }
    const double2 v = make_double2(acc.x * ctr.x - acc.y * ctr.y, acc.x * ctr.y + acc.y * ctr.x);
    store_c<C>(alpha_l, pos * w.qp + t, v);
  }
}

constexpr int kBetaChunk = 16;

template <typename C>
__global__ void k_form_beta(PhaseDev ph, const void *xd, int N, WedgeDev w,
                            const uint2 *__restrict__ warp_l, const int *__restrict__ rx, int r,
                            int q, const double2 *__restrict__ P, const int *__restrict__ pk1,
                            const int *__restrict__ pk2, const double *__restrict__ dec,
                            void *beta_l) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= w.npts) return;
  const XView xv = xview(ph, xd);
  const int k1 = pk1[p], k2 = pk2[p];
  const double d = dec ? dec[p] : 1.0;
  for (int t0 = 0; t0 < q; t0 += kBetaChunk) {
    double2 acc[kBetaChunk];
#pragma unroll
    for (int k = 0; k < kBetaChunk; ++k) acc[k] = make_double2(0.0, 0.0);
    for (int i = 0; i < r; ++i) {
      const long long x = rx[i];
      const double2 a = entry(ph, xv, N, w, x, warp_l[x], k1, k2);
#pragma unroll
      for (int k = 0; k < kBetaChunk; ++k) {
        if (t0 + k < q) {
          const double2 b = P[(long long)(t0 + k) * r + i];
          acc[k].x += b.x * a.x - b.y * a.y;
          acc[k].y += b.x * a.y + b.y * a.x;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kBetaChunk; ++k)
      if (t0 + k < q)
        store_c<C>(beta_l, (long long)(t0 + k) * w.npts + p,
                   make_double2(acc[k].x * d, acc[k].y * d));
  }
}

// Column-wise error of the separated factors on s sampled rows (the
// estimator of Sec. 4, Table 1, taken over every column of the wedge):
// err[p] = sum_i |A(x_i, xi_p) - sum_t U[i][t] T[t][p]|^2, nrm[p] = sum_i |A|^2.
__global__ void k_validate(PhaseDev ph, const void *xd, int N, WedgeDev w,
                           const uint2 *__restrict__ warp_l, const int *__restrict__ gx, int s,
                           const double2 *__restrict__ UG, const double2 *__restrict__ T, int q,
                           const int *__restrict__ pk1, const int *__restrict__ pk2,
                           double *__restrict__ err, double *__restrict__ nrm) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= w.npts) return;
  const XView xv = xview(ph, xd);
  const int k1 = pk1[p], k2 = pk2[p];
  double e = 0.0, n = 0.0;
  for (int i = 0; i < s; ++i) {
    const long long x = gx[i];
    const double2 a = entry(ph, xv, N, w, x, warp_l[x], k1, k2);
    double2 u = make_double2(0.0, 0.0);
    for (int t = 0; t < q; ++t) {
      const double2 b = UG[(long long)i * q + t], c = T[(long long)t * w.npts + p];
      u.x += b.x * c.x - b.y * c.y;
      u.y += b.x * c.y + b.y * c.x;
    }
    const double dx = a.x - u.x, dy = a.y - u.y;
    e += dx * dx + dy * dy;
    n += a.x * a.x + a.y * a.y;
  }
  err[p] = e;
  nrm[p] = n;
}

unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t plan_validate(const PhaseDev &ph, const void *d_xdata, int N, const WedgeDev &w,
                          const uint2 *d_warp_l, const int *d_gx, int s, const double2 *d_UG,
                          const double2 *d_T, int q, const int *d_pk1, const int *d_pk2,
                          double *d_err, double *d_nrm, cudaStream_t st) {
  k_validate<<<blocks(w.npts, 128), 128, 0, st>>>(ph, d_xdata, N, w, d_warp_l, d_gx, s, d_UG, d_T,
                                                  q, d_pk1, d_pk2, d_err, d_nrm);
  return cudaGetLastError();
}

size_t plan_xdata_bytes(const PhaseDev &ph, int N) {
  const size_t NN = (size_t)N * N;
  if (ph.kind == FIO_PHASE_ELLIPSE) return NN * sizeof(double2);
  if (ph.kind == FIO_PHASE_TAU_MODES) return NN * kNm * sizeof(double2);
  return 16;
}

cudaError_t plan_xdata(const PhaseDev &ph, const double *d_modes, int N, void *d_xdata,
                       cudaStream_t s) {
  const long long NN = (long long)N * N;
  k_xdata<<<blocks(NN, 256), 256, 0, s>>>(ph, d_modes, N, d_xdata);
  return cudaGetLastError();
}

cudaError_t plan_warp(const PhaseDev &ph, const void *d_xdata, int N, int L, const WedgeDev *d_w,
                      uint2 *d_warp, cudaStream_t s) {
  const long long n = (long long)N * N * L;
  k_warp<<<blocks(n, 256), 256, 0, s>>>(ph, d_xdata, N, L, d_w, d_warp);
  return cudaGetLastError();
}

cudaError_t plan_eval_cols(const PhaseDev &ph, const void *d_xdata, int N, const WedgeDev &w,
                           const uint2 *d_warp_l, const int *d_ck1, const int *d_ck2, int r,
                           double2 *d_AC, cudaStream_t s) {
  const long long n = (long long)N * N * r;
  k_eval_cols<<<blocks(n, 256), 256, 0, s>>>(ph, d_xdata, N, w, d_warp_l, d_ck1, d_ck2, r, d_AC);
  return cudaGetLastError();
}

int tsqr_panel_rows(int r) { return r * 4 > 128 ? r * 4 : 128; }

size_t tsqr_stack_elems(long long rows, int r) {
  const long long P = tsqr_panel_rows(r);
  return (size_t)((rows + P - 1) / P) * r * r;
}

cudaError_t plan_tsqr(const double2 *d_A, long long rows, int r, double2 *d_work, double2 *d_stk0,
                      double2 *d_stk1, double2 *h_R, cudaStream_t s) {
  const int P = tsqr_panel_rows(r);
  const size_t smem = (size_t)(kQrGroups + 1) * r * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(k_panel_qr, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  double2 *stk[2] = {d_stk0, d_stk1};
  const double2 *in = d_A;
  long long n = rows;
  int lvl = 0;
  for (;;) {
    const long long np = (n + P - 1) / P;
    k_panel_qr<<<(unsigned)np, kQrThreads, smem, s>>>(in, n, r, P, d_work, stk[lvl & 1]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (np == 1) break;
    in = stk[lvl & 1];
    n = np * r;
    ++lvl;
  }
  return cudaMemcpyAsync(h_R, stk[lvl & 1], sizeof(double2) * r * r, cudaMemcpyDeviceToHost, s);
}

cudaError_t plan_form_alpha(const double2 *d_AC, int N, int r, int q, const double2 *d_W,
                            const WedgeDev &w, const uint2 *d_warp_l, const uint32_t *d_perm_l,
                            void *d_alpha_l, int precision, cudaStream_t s) {
  const long long NN = (long long)N * N;
  if (precision == FIO_FP64)
    k_form_alpha<double2><<<blocks(NN, 256), 256, 0, s>>>(d_AC, N, r, q, d_W, w, d_warp_l,
                                                          d_perm_l, d_alpha_l);
  else
    k_form_alpha<float2><<<blocks(NN, 256), 256, 0, s>>>(d_AC, N, r, q, d_W, w, d_warp_l,
                                                         d_perm_l, d_alpha_l);
  return cudaGetLastError();
}

cudaError_t plan_form_beta(const PhaseDev &ph, const void *d_xdata, int N, const WedgeDev &w,
                           const uint2 *d_warp_l, const int *d_rx, int r, int q,
                           const double2 *d_P, const int *d_pk1, const int *d_pk2,
                           const double *d_dec, void *d_beta_l, int precision, cudaStream_t s) {
  if (precision == FIO_FP64)
    k_form_beta<double2><<<blocks(w.npts, 128), 128, 0, s>>>(ph, d_xdata, N, w, d_warp_l, d_rx,
                                                             r, q, d_P, d_pk1, d_pk2, d_dec,
                                                             d_beta_l);
  else
    k_form_beta<float2><<<blocks(w.npts, 128), 128, 0, s>>>(ph, d_xdata, N, w, d_warp_l, d_rx, r,
                                                            q, d_P, d_pk1, d_pk2, d_dec,
                                                            d_beta_l);
  return cudaGetLastError();
}

}  // namespace fio
