/*
 * fio_oracle.c -- plain FP64 CPU evaluation of the discrete Fourier integral
 * operator of Candes, Demanet and Ying, "Fast Computation of Fourier Integral
 * Operators" (Sec. 1.2, Eq. dfio and Eq. dft; adjoint from Sec. 3.5).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  It shares no code, header, table or constant with the
 * CUDA library; only tests/, __graft_entry__.smoke() and the cpu_baseline leg
 * of bench.py load it.  Nothing here is blocked, fused or reordered beyond the
 * definitions it cites: every output is the literal sum of the definition.
 *
 * Conventions (Sec. 1.2):
 *   X     = { x = (n1/N, n2/N) : 0 <= n1, n2 < N },   f stored f[n1*N + n2]
 *   Omega = { xi = (k1, k2) : -N/2 <= k1, k2 < N/2 },  fhat stored
 *           fhat[(k1 + N/2)*N + (k2 + N/2)]  ("centred" order)
 *   fhat(xi) = (1/N) sum_x exp(-2 pi i x.xi) f(x)                      (Eq. dft)
 *   (Lf)(x)  = (1/N) sum_xi a(x,xi) exp(2 pi i Phi(x,xi)) fhat(xi)     (Eq. dfio)
 *   (L*g)^(xi) = (1/N) sum_y conj(a(y,xi)) exp(-2 pi i Phi(y,xi)) g(y) (Sec. 3.5,
 *                 with the amplitude's conjugate added for general a)
 *   (L*g)(x) = (1/N) sum_xi exp(2 pi i x.xi) (L*g)^(xi)
 *
 * Every phase used here has the form Phi(x,xi) = x.xi + Psi(x,xi).  The x.xi
 * part is evaluated exactly as the integer (n1 k1 + n2 k2) mod N over N.
 *
 * Phase kinds (parameters are plain input data):
 *   0  shift+wave   Psi = -x0.xi + c|xi|            params {x01, x02, c}
 *                   (Phi = (x-x0).xi + c|xi|: the translation and the
 *                   constant-speed wave propagator of Sec. 1, Eq. wave_solution)
 *   1  ellipse      Psi = sqrt(c1(x)^2 xi1^2 + c2(x)^2 xi2^2),
 *                   c1 = A1 + B1 sin(2 pi x1) sin(2 pi x2),
 *                   c2 = A2 + B2 cos(2 pi x1) cos(2 pi x2)  params {A1,B1,A2,B2}
 *                   (the phase family of Eq. nrphase)
 *   3  ellipse with product-form axes (the paper's own experiments, Sec. 4):
 *                   Psi = sqrt(r1^2 xi1^2 + r2^2 xi2^2),
 *                   r1 = s1 (a1 + sin 4 pi x1)(a1 + sin 4 pi x2),
 *                   r2 = s2 (a2 + cos 4 pi x1)(a2 + cos 4 pi x2)  params {a1,s1,a2,s2}
 *   2  tau modes    Psi = |xi| tau(x, theta),
 *                   tau = sum_j a_j cos(2 pi (k1_j x1 + k2_j x2) + m_j theta + p_j)
 *                   params: nmodes rows of {a_j, k1_j, k2_j, m_j, p_j}
 * theta = arg(xi) = atan2(xi2, xi1); at xi = 0 the phase is 0 (homogeneity).
 *
 * Amplitude kinds: 0  a = 1;   1  a = (1 + a1 sin 2 pi x1)(1 + a2 cos theta),
 * with cos theta := 1 at xi = 0;   2  the Hankel amplitude of the integration
 * along ellipses (Appendix A, Eq. ellipses_amp): with s = a1 = +1 or -1 and
 * rho = s (Phi(x, xi) - x.xi),
 *     a = (J0(2 pi rho) + i s Y0(2 pi rho)) exp(-2 pi i s rho) / (4 pi),
 * and the Y0 term dropped where rho <= 0 (xi = 0, where Y0 is singular: the
 * regularisation Appendix A calls for).
 */
#define _DEFAULT_SOURCE 1 /* j0, y0 (POSIX Bessel functions) from math.h */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double TWO_PI = 6.283185307179586476925286766559;

typedef struct {
  int kind;
  int nmodes;
  const double *params;
} or_phase;

typedef struct {
  int kind;
  double a1, a2;
} or_amp;

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* exp(sign * 2 pi i j / N) for j = 0..N-1: twiddles indexed by exact integers. */
static cplx *twiddles(int N, int sign) {
  cplx *tw = (cplx *)malloc(sizeof(cplx) * (size_t)N);
  for (int j = 0; j < N; ++j) tw[j] = cexp(sign * TWO_PI * I * (double)j / (double)N);
  return tw;
}

static int imod(long long a, int n) {
  long long r = a % n;
  return (int)(r < 0 ? r + n : r);
}

/* ---------------------------------------------------------------- Eq. dft -- */

/* fhat(xi) = (1/N) sum_x exp(-2 pi i x.xi) f(x), separably: first over n2,
 * then over n1.  in: f[n1*N+n2]; out: centred fhat. */
void or_dft2(int N, const double *in_ri, double *out_ri) {
  const cplx *f = (const cplx *)in_ri;
  cplx *fh = (cplx *)out_ri;
  cplx *tw = twiddles(N, -1);
  cplx *h = (cplx *)malloc(sizeof(cplx) * (size_t)N * N); /* h[n1][k2 idx] */
#pragma omp parallel for schedule(static)
  for (int n1 = 0; n1 < N; ++n1)
    for (int ik2 = 0; ik2 < N; ++ik2) {
      int k2 = ik2 - N / 2;
      cplx s = 0;
      for (int n2 = 0; n2 < N; ++n2) s += tw[imod((long long)n2 * k2, N)] * f[(size_t)n1 * N + n2];
      h[(size_t)n1 * N + ik2] = s;
    }
#pragma omp parallel for schedule(static)
  for (int ik1 = 0; ik1 < N; ++ik1) {
    int k1 = ik1 - N / 2;
    for (int ik2 = 0; ik2 < N; ++ik2) {
      cplx s = 0;
      for (int n1 = 0; n1 < N; ++n1) s += tw[imod((long long)n1 * k1, N)] * h[(size_t)n1 * N + ik2];
      fh[(size_t)ik1 * N + ik2] = s / (double)N;
    }
  }
  free(h);
  free(tw);
}

/* Inverse of Eq. dft: f(x) = (1/N) sum_xi exp(+2 pi i x.xi) fhat(xi). */
void or_idft2(int N, const double *in_ri, double *out_ri) {
  const cplx *fh = (const cplx *)in_ri;
  cplx *f = (cplx *)out_ri;
  cplx *tw = twiddles(N, +1);
  cplx *h = (cplx *)malloc(sizeof(cplx) * (size_t)N * N); /* h[k1 idx][n2] */
#pragma omp parallel for schedule(static)
  for (int ik1 = 0; ik1 < N; ++ik1)
    for (int n2 = 0; n2 < N; ++n2) {
      cplx s = 0;
      for (int ik2 = 0; ik2 < N; ++ik2)
        s += tw[imod((long long)n2 * (ik2 - N / 2), N)] * fh[(size_t)ik1 * N + ik2];
      h[(size_t)ik1 * N + n2] = s;
    }
#pragma omp parallel for schedule(static)
  for (int n1 = 0; n1 < N; ++n1)
    for (int n2 = 0; n2 < N; ++n2) {
      cplx s = 0;
      for (int ik1 = 0; ik1 < N; ++ik1)
        s += tw[imod((long long)n1 * (ik1 - N / 2), N)] * h[(size_t)ik1 * N + n2];
      f[(size_t)n1 * N + n2] = s / (double)N;
    }
  free(h);
  free(tw);
}

/* ------------------------------------------------------ phase / amplitude -- */

/* Per-x data a phase needs (so that the loop over xi stays cheap). */
typedef struct {
  double c1, c2;   /* ellipse axes at x */
  cplx Cm[17];     /* tau modes grouped by m in [-8, 8] (index m+8) */
  int grouped;     /* Cm valid */
} xdata;

static void prepare_x(const or_phase *ph, double x1, double x2, int grouped, xdata *d) {
  memset(d, 0, sizeof(*d));
  if (ph->kind == 1) {
    const double *p = ph->params;
    d->c1 = p[0] + p[1] * sin(TWO_PI * x1) * sin(TWO_PI * x2);
    d->c2 = p[2] + p[3] * cos(TWO_PI * x1) * cos(TWO_PI * x2);
  } else if (ph->kind == 3) {
    const double *p = ph->params;
    d->c1 = p[1] * (p[0] + sin(2 * TWO_PI * x1)) * (p[0] + sin(2 * TWO_PI * x2));
    d->c2 = p[3] * (p[2] + cos(2 * TWO_PI * x1)) * (p[2] + cos(2 * TWO_PI * x2));
  } else if (ph->kind == 2 && grouped) {
    /* tau(x,theta) = Re sum_m C_m(x) exp(i m theta) with
     * C_m(x) = sum_{j : m_j = m} a_j exp(i (2 pi k_j.x + p_j)); an exact
     * regrouping of the sum over modes. */
    for (int j = 0; j < ph->nmodes; ++j) {
      const double *p = ph->params + 5 * j;
      int m = (int)lrint(p[3]);
      d->Cm[m + 8] += p[0] * cexp(I * (TWO_PI * (p[1] * x1 + p[2] * x2) + p[4]));
    }
    d->grouped = 1;
  }
}

/* tau(x, theta) as the literal sum over modes. */
static double tau_direct(const or_phase *ph, double x1, double x2, double theta) {
  double s = 0.0;
  for (int j = 0; j < ph->nmodes; ++j) {
    const double *p = ph->params + 5 * j;
    s += p[0] * cos(TWO_PI * (p[1] * x1 + p[2] * x2) + p[3] * theta + p[4]);
  }
  return s;
}

/* tau from the grouped coefficients; e^{i theta} = xi / |xi|. */
static double tau_grouped(const xdata *d, cplx eith) {
  cplx s = d->Cm[8];
  cplx pp = 1.0, pn = 1.0;
  for (int m = 1; m <= 8; ++m) {
    pp *= eith;
    pn *= conj(eith);
    s += d->Cm[8 + m] * pp + d->Cm[8 - m] * pn;
  }
  return creal(s);
}

/* Psi(x, xi) = Phi(x, xi) - x.xi */
static double psi(const or_phase *ph, const xdata *d, double x1, double x2, int k1, int k2) {
  const double *p = ph->params;
  double r = sqrt((double)k1 * k1 + (double)k2 * k2);
  if (k1 == 0 && k2 == 0) return 0.0;
  switch (ph->kind) {
    case 0:
      return -(p[0] * k1 + p[1] * k2) + p[2] * r;
    case 1:
    case 3:
      return sqrt(d->c1 * d->c1 * (double)k1 * k1 + d->c2 * d->c2 * (double)k2 * k2);
    case 2:
      if (d->grouped) return r * tau_grouped(d, (k1 + I * k2) / r);
      return r * tau_direct(ph, x1, x2, atan2((double)k2, (double)k1));
  }
  return NAN;
}

/* a(x, xi); psi = Phi(x, xi) - x.xi is needed by the Hankel kind only. */
static cplx amp(const or_amp *a, double x1, int k1, int k2, double psi_val) {
  if (a == NULL || a->kind == 0) return 1.0;
  if (a->kind == 2) {
    const double s = a->a1, rho = s * psi_val;
    const double y = rho > 0 ? y0(TWO_PI * rho) : 0.0;
    return (j0(TWO_PI * rho) + I * s * y) * cexp(-I * TWO_PI * s * rho) / (2.0 * TWO_PI);
  }
  double r = sqrt((double)k1 * k1 + (double)k2 * k2);
  double cth = (r > 0) ? (double)k1 / r : 1.0;
  return (1.0 + a->a1 * sin(TWO_PI * x1)) * (1.0 + a->a2 * cth);
}

/* Phi(x, xi) at arbitrary points (for pinning the phase formulas). */
void or_phase_eval(int kind, int nmodes, const double *params, int grouped, int npts,
                   const double *x1, const double *x2, const int *k1, const int *k2,
                   double *phi_out) {
  or_phase ph = {kind, nmodes, params};
  for (int i = 0; i < npts; ++i) {
    xdata d;
    prepare_x(&ph, x1[i], x2[i], grouped, &d);
    phi_out[i] = x1[i] * k1[i] + x2[i] * k2[i] + psi(&ph, &d, x1[i], x2[i], k1[i], k2[i]);
  }
}

/* a(x_i, xi_i) as interleaved complex; psi = Phi - x.xi at the same points (read
 * by the Hankel kind only, may be NULL otherwise). */
void or_amp_eval(int kind, double a1, double a2, int npts, const double *x1, const int *k1,
                 const int *k2, const double *psi_vals, double *out_ri) {
  or_amp a = {kind, a1, a2};
  for (int i = 0; i < npts; ++i) {
    const cplx v = amp(&a, x1[i], k1[i], k2[i], psi_vals ? psi_vals[i] : 0.0);
    out_ri[2 * i] = creal(v);
    out_ri[2 * i + 1] = cimag(v);
  }
}

/* tau(x, theta) of the tau-mode phase and its derivatives, by the literal sum
 * over modes: out[4 i + 0..3] = tau, d tau/d x1, d tau/d x2, d tau/d theta. */
void or_tau_eval(int nmodes, const double *params, int npts, const double *x1, const double *x2,
                 const double *theta, double *out) {
  for (int i = 0; i < npts; ++i) {
    double t = 0, d1 = 0, d2 = 0, dt = 0;
    for (int j = 0; j < nmodes; ++j) {
      const double *p = params + 5 * j;
      const double arg = TWO_PI * (p[1] * x1[i] + p[2] * x2[i]) + p[3] * theta[i] + p[4];
      const double s = sin(arg);
      t += p[0] * cos(arg);
      d1 -= p[0] * s * TWO_PI * p[1];
      d2 -= p[0] * s * TWO_PI * p[2];
      dt -= p[0] * s * p[3];
    }
    out[4 * i] = t;
    out[4 * i + 1] = d1;
    out[4 * i + 2] = d2;
    out[4 * i + 3] = dt;
  }
}

/* ---------------------------------------------------------------- Eq. dfio -- */

/* (Lf)(x_i) at grid points x_i = (n1_i/N, n2_i/N), from the centred fhat. */
void or_apply_points(int N, int kind, int nmodes, const double *params, int grouped,
                     int amp_kind, double a1, double a2, const double *fhat_ri, int npts,
                     const int *n1, const int *n2, double *out_ri) {
  or_phase ph = {kind, nmodes, params};
  or_amp am = {amp_kind, a1, a2};
  const cplx *fh = (const cplx *)fhat_ri;
  cplx *out = (cplx *)out_ri;
  cplx *tw = twiddles(N, +1);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < npts; ++i) {
    double x1 = (double)n1[i] / N, x2 = (double)n2[i] / N;
    xdata d;
    prepare_x(&ph, x1, x2, grouped, &d);
    cplx s = 0;
    for (int ik1 = 0; ik1 < N; ++ik1) {
      int k1 = ik1 - N / 2;
      for (int ik2 = 0; ik2 < N; ++ik2) {
        int k2 = ik2 - N / 2;
        const double ps = psi(&ph, &d, x1, x2, k1, k2);
        cplx e = tw[imod((long long)n1[i] * k1 + (long long)n2[i] * k2, N)] *
                 cexp(TWO_PI * I * ps);
        s += amp(&am, x1, k1, k2, ps) * e * fh[(size_t)ik1 * N + ik2];
      }
    }
    out[i] = s / (double)N;
  }
  free(tw);
}

/* Dense O(N^4) apply on the whole grid: Eq. dft then Eq. dfio at every x. */
void or_apply_dense(int N, int kind, int nmodes, const double *params, int grouped, int amp_kind,
                    double a1, double a2, const double *f_ri, double *out_ri) {
  size_t n = (size_t)N * N;
  double *fh = (double *)malloc(sizeof(double) * 2 * n);
  int *n1 = (int *)malloc(sizeof(int) * n), *n2 = (int *)malloc(sizeof(int) * n);
  for (size_t i = 0; i < n; ++i) {
    n1[i] = (int)(i / N);
    n2[i] = (int)(i % N);
  }
  or_dft2(N, f_ri, fh);
  or_apply_points(N, kind, nmodes, params, grouped, amp_kind, a1, a2, fh, (int)n, n1, n2, out_ri);
  free(fh);
  free(n1);
  free(n2);
}

/* ------------------------------------------------------------- Sec. 3.5 -- */

/* (L*g)^(xi_j) = (1/N) sum_y conj(a(y, xi_j)) exp(-2 pi i Phi(y, xi_j)) g(y). */
void or_adjoint_hat_points(int N, int kind, int nmodes, const double *params, int grouped,
                           int amp_kind, double a1, double a2, const double *g_ri, int nxi,
                           const int *k1, const int *k2, double *out_ri) {
  or_phase ph = {kind, nmodes, params};
  or_amp am = {amp_kind, a1, a2};
  const cplx *g = (const cplx *)g_ri;
  cplx *out = (cplx *)out_ri;
  size_t n = (size_t)N * N;
  cplx *tw = twiddles(N, -1);
  /* per-y data is reused for every xi */
  xdata *xd = (xdata *)malloc(sizeof(xdata) * n);
#pragma omp parallel for schedule(static)
  for (size_t i = 0; i < n; ++i)
    prepare_x(&ph, (double)(i / N) / N, (double)(i % N) / N, grouped, &xd[i]);
#pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j < nxi; ++j) {
    cplx s = 0;
    for (size_t i = 0; i < n; ++i) {
      int m1 = (int)(i / N), m2 = (int)(i % N);
      double y1 = (double)m1 / N, y2 = (double)m2 / N;
      const double ps = psi(&ph, &xd[i], y1, y2, k1[j], k2[j]);
      cplx e = tw[imod((long long)m1 * k1[j] + (long long)m2 * k2[j], N)] * cexp(-TWO_PI * I * ps);
      s += conj(amp(&am, y1, k1[j], k2[j], ps)) * e * g[i];
    }
    out[j] = s / (double)N;
  }
  free(xd);
  free(tw);
}

/* Dense adjoint: (L*g)^ at every xi, then the inverse of Eq. dft. */
void or_adjoint_dense(int N, int kind, int nmodes, const double *params, int grouped,
                      int amp_kind, double a1, double a2, const double *g_ri, double *out_ri) {
  size_t n = (size_t)N * N;
  double *gh = (double *)malloc(sizeof(double) * 2 * n);
  int *k1 = (int *)malloc(sizeof(int) * n), *k2 = (int *)malloc(sizeof(int) * n);
  for (size_t i = 0; i < n; ++i) {
    k1[i] = (int)(i / N) - N / 2;
    k2[i] = (int)(i % N) - N / 2;
  }
  or_adjoint_hat_points(N, kind, nmodes, params, grouped, amp_kind, a1, a2, g_ri, (int)n, k1, k2,
                        gh);
  or_idft2(N, gh, out_ri);
  free(gh);
  free(k1);
  free(k2);
}

/* The dense matrix of L at small N: K[x][y] = (Lf)(x) for f = delta_y.
 * Built column by column from the definition (for the adjoint identity). */
void or_matrix(int N, int kind, int nmodes, const double *params, int grouped, int amp_kind,
               double a1, double a2, double *mat_ri) {
  size_t n = (size_t)N * N;
  double *e = (double *)calloc(2 * n, sizeof(double));
  double *col = (double *)malloc(sizeof(double) * 2 * n);
  cplx *m = (cplx *)mat_ri;
  for (size_t j = 0; j < n; ++j) {
    memset(e, 0, sizeof(double) * 2 * n);
    e[2 * j] = 1.0;
    or_apply_dense(N, kind, nmodes, params, grouped, amp_kind, a1, a2, e, col);
    const cplx *c = (const cplx *)col;
    for (size_t i = 0; i < n; ++i) m[i * n + j] = c[i];
  }
  free(e);
  free(col);
}
