// api.cpp -- the C ABI of include/fio.h: argument checks, status codes and
// thread-local error text around the plan builder (plan.cpp) and the apply
// launchers (apply.cu).  No exception crosses this boundary.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fio_internal.h"
#include "plan_host.h"

static thread_local std::string g_last_error;

namespace fio {
void set_error(const std::string &msg) { g_last_error = msg; }
}  // namespace fio

using namespace fio;

namespace {

fio_status cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FIO_ENOMEM : FIO_ECUDA;
}

bool plan_ok(fio_plan p) {
  if (!p || !p->d_alpha) {
    set_error("invalid plan handle");
    return false;
  }
  return true;
}

}  // namespace

extern "C" {

int fio_version(void) { return 100; }

const char *fio_status_string(fio_status s) {
  switch (s) {
    case FIO_OK: return "FIO_OK";
    case FIO_EINVAL: return "FIO_EINVAL: invalid argument";
    case FIO_ENOMEM: return "FIO_ENOMEM: out of memory";
    case FIO_ECUDA: return "FIO_ECUDA: CUDA error";
    case FIO_ERANK: return "FIO_ERANK: separation rank exceeds rank_cap";
    case FIO_ETIMEOUT: return "FIO_ETIMEOUT: bounded device wait gave up";
    case FIO_EUNSUPPORTED: return "FIO_EUNSUPPORTED: not supported";
  }
  return "unknown status";
}

const char *fio_last_error(void) { return g_last_error.c_str(); }

fio_status fio_options_default(fio_options *opt) {
  if (!opt) return FIO_EINVAL;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = FIO_MIXED;
  opt->seed = 0x5EED5EEDULL;
  opt->max_batch = 1;
  return FIO_OK;
}

fio_status fio_plan_create(int N, const fio_phase *phase, const fio_amplitude *amp, double eps,
                           const fio_options *opt, fio_plan *out_plan) {
  if (!out_plan) {
    set_error("out_plan is NULL");
    return FIO_EINVAL;
  }
  *out_plan = nullptr;
  fio_plan_s *p = new (std::nothrow) fio_plan_s();
  if (!p) {
    set_error("host allocation failed");
    return FIO_ENOMEM;
  }
  fio_status s;
  try {
    s = build_plan(p, N, phase, amp, eps, opt);
  } catch (const std::bad_alloc &) {
    set_error("host allocation failed");
    s = FIO_ENOMEM;
  } catch (...) {
    set_error("unexpected host exception");
    s = FIO_EINVAL;
  }
  if (s != FIO_OK) {
    free_plan_device(p);
    delete p;
    return s;
  }
  *out_plan = p;
  return FIO_OK;
}

void fio_plan_destroy(fio_plan p) {
  if (!p) return;
  release_timing_events(p);
  free_plan_device(p);
  delete p;
}

fio_status fio_plan_save(fio_plan p, const char *path) {
  if (!plan_ok(p) || !path) {
    set_error("fio_plan_save: invalid plan or path");
    return FIO_EINVAL;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    set_error("fio_plan_save: pending CUDA error");
    return FIO_ECUDA;
  }
  return save_plan(p, path);
}

fio_status fio_plan_load(const char *path, int max_batch, fio_plan *out_plan) {
  if (!out_plan || !path || max_batch < 0 || max_batch > 4096) {
    set_error("fio_plan_load: bad arguments");
    return FIO_EINVAL;
  }
  *out_plan = nullptr;
  fio_plan_s *p = new (std::nothrow) fio_plan_s();
  if (!p) {
    set_error("host allocation failed");
    return FIO_ENOMEM;
  }
  fio_status s;
  try {
    s = load_plan(p, path, max_batch);
  } catch (const std::bad_alloc &) {
    set_error("host allocation failed");
    s = FIO_ENOMEM;
  }
  if (s != FIO_OK) {
    free_plan_device(p);
    delete p;
    return s;
  }
  *out_plan = p;
  return FIO_OK;
}

fio_status fio_apply(fio_plan p, const void *f, void *out, int batch, void *stream) {
  if (!plan_ok(p)) return FIO_EINVAL;
  if (!f || !out || f == out || batch < 1 || batch > p->max_batch) {
    set_error("fio_apply: null/aliased pointers or batch outside [1, max_batch]");
    return FIO_EINVAL;
  }
  cudaError_t e = launch_apply(p, f, out, batch, (cudaStream_t)stream);
  return e == cudaSuccess ? FIO_OK : cuda_fail(e, "fio_apply");
}

fio_status fio_apply_real(fio_plan p, const void *f, void *out, int batch, void *stream) {
  if (!plan_ok(p)) return FIO_EINVAL;
  if (!f || !out || batch < 1 || batch > p->max_batch) {
    set_error("fio_apply_real: null pointers or batch outside [1, max_batch]");
    return FIO_EINVAL;
  }
  // the real input spans half the bytes of the complex output: no overlap at all
  const size_t rs = p->precision == FIO_FP64 ? 8 : 4;
  const size_t n = (size_t)batch * p->N * p->N;
  const char *fa = static_cast<const char *>(f), *oa = static_cast<const char *>(out);
  if (fa < oa + 2 * rs * n && oa < fa + rs * n) {
    set_error("fio_apply_real: out overlaps f");
    return FIO_EINVAL;
  }
  cudaError_t e = launch_apply(p, f, out, batch, (cudaStream_t)stream, true);
  return e == cudaSuccess ? FIO_OK : cuda_fail(e, "fio_apply_real");
}

fio_status fio_apply_adjoint(fio_plan p, const void *g, void *out, int batch, void *stream) {
  if (!plan_ok(p)) return FIO_EINVAL;
  if (!g || !out || g == out || batch < 1 || batch > p->max_batch) {
    set_error("fio_apply_adjoint: null/aliased pointers or batch outside [1, max_batch]");
    return FIO_EINVAL;
  }
  cudaError_t e = launch_adjoint(p, g, out, batch, (cudaStream_t)stream);
  return e == cudaSuccess ? FIO_OK : cuda_fail(e, "fio_apply_adjoint");
}

fio_status fio_apply_normal(fio_plan p, const void *f, void *out, int batch, void *stream) {
  if (!plan_ok(p)) return FIO_EINVAL;
  if (!f || !out || f == out || batch < 1 || batch > p->max_batch) {
    set_error("fio_apply_normal: null/aliased pointers or batch outside [1, max_batch]");
    return FIO_EINVAL;
  }
  cudaError_t e = launch_apply(p, f, out, batch, (cudaStream_t)stream);
  // the adjoint's first stage (the spread) consumes its whole input before any
  // later stage writes the output, so L f may be read from out in place
  if (e == cudaSuccess) e = launch_adjoint(p, out, out, batch, (cudaStream_t)stream);
  return e == cudaSuccess ? FIO_OK : cuda_fail(e, "fio_apply_normal");
}

fio_status fio_plan_sync(fio_plan p, void *stream) {
  if (!plan_ok(p)) return FIO_EINVAL;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "fio_plan_sync");
  int word = 0;
  e = cudaMemcpy(&word, p->d_errword, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "fio_plan_sync");
  if (word != 0) {
    set_error("fio_plan_sync: an in-kernel consistency check failed (a point's window start "
              "left the bin it was sorted into); the affected terms were skipped");
    return FIO_ECUDA;
  }
  return FIO_OK;
}

fio_status fio_plan_get_info(fio_plan p, fio_plan_info *info) {
  if (!plan_ok(p) || !info) return FIO_EINVAL;
  std::memset(info, 0, sizeof(*info));
  const size_t cs = p->precision == FIO_FP64 ? 16 : 8;
  info->N = p->N;
  info->L = p->L;
  info->precision = p->precision;
  info->kb_width = p->kb.w;
  info->max_batch = p->max_batch;
  info->sigma = p->sigma;
  info->kb_beta = p->kb.beta;
  info->eps = p->eps;
  info->q_max = p->q_max;
  info->q_min = p->q_min;
  info->r_max = p->r_max;
  info->q_mean = p->q_mean;
  info->bytes_alpha = (unsigned long long)p->alpha_elems * cs;
  info->bytes_beta = (unsigned long long)p->beta_elems * cs;
  info->bytes_warp = (unsigned long long)p->N * p->N * p->L * 8ULL;
  info->bytes_grid = (unsigned long long)p->grid_units * p->max_batch * cs;
  info->bytes_total = p->bytes_total;
  info->grid_points = (unsigned long long)p->grid_units;
  info->alg_bytes_apply = p->alg_bytes;
  info->plan_seconds = p->plan_seconds;
  info->sep_error = p->sep_err;
  info->kernel_launches = p->launches;
  info->surrogate_warp = p->sur_warp;
  info->surrogate_warp_cycles = p->sur_warp_cycles;
  info->surrogate_residual_cycles = p->sur_residual_cycles;
  info->max_bin_points = p->max_bin_pts;
  info->mean_bin_points = p->mean_bin_pts;
  info->max_spread_candidates = p->max_cand;
  info->alpha_mode = p->alpha_mode;
  info->alpha_groups = p->alpha_mode == FIO_ALPHA_RECOMPUTE ? (int)p->grp_first.size() - 1 : 0;
  info->bytes_recompute = (unsigned long long)rc_bytes(p);
  return FIO_OK;
}

fio_status fio_plan_set_timing(fio_plan p, int on) {
  if (!plan_ok(p)) return FIO_EINVAL;
  p->timing = on != 0;
  return FIO_OK;
}

fio_status fio_plan_stage_times(fio_plan p, double *ms, long long *count) {
  if (!plan_ok(p)) return FIO_EINVAL;
  if (ms)
    for (int i = 0; i < FIO_NUM_STAGES; ++i) ms[i] = 0.0;
  if (count)
    for (int i = 0; i < FIO_NUM_STAGES; ++i) count[i] = 0;
  for (size_t k = 0; k < p->ev_used; ++k) {
    cudaError_t e = cudaEventSynchronize(p->ev_pool[2 * k + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "fio_plan_stage_times");
    float t = 0.f;
    e = cudaEventElapsedTime(&t, p->ev_pool[2 * k], p->ev_pool[2 * k + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "fio_plan_stage_times");
    const int st = p->ev_stage[k];
    if (ms) ms[st] += t;
    if (count) count[st] += 1;
  }
  p->ev_used = 0;
  return FIO_OK;
}

fio_status fio_plan_get_wedge(fio_plan p, int l, fio_wedge_info *info) {
  if (!plan_ok(p) || !info || l < 0 || l >= p->L) {
    set_error("fio_plan_get_wedge: bad arguments");
    return FIO_EINVAL;
  }
  const WedgeDev &w = p->wedges[l];
  std::memcpy(info->M, w.M, sizeof(info->M));
  info->xc1 = w.xc1;
  info->xc2 = w.xc2;
  info->b1 = w.b1;
  info->n1 = w.n1;
  info->b2 = w.b2;
  info->n2 = w.n2;
  info->m1 = w.m1;
  info->m2 = w.m2;
  info->q = w.q;
  info->r = p->wedge_r[l];
  info->npts = w.npts;
  return FIO_OK;
}

fio_status fio_plan_export_wedge(fio_plan p, int l, double *alpha, double *beta, int *k1,
                                 int *k2) {
  if (!plan_ok(p) || l < 0 || l >= p->L) {
    set_error("fio_plan_export_wedge: bad arguments");
    return FIO_EINVAL;
  }
  const WedgeDev &w = p->wedges[l];
  const long long NN = (long long)p->N * p->N;
  const bool f64 = p->precision == FIO_FP64;
  const size_t cs = f64 ? 16 : 8;
  using cd = std::complex<double>;
  auto fetch = [&](const void *base, long long off, long long n, std::vector<cd> &dst) {
    std::vector<unsigned char> raw((size_t)n * cs);
    cudaError_t e = cudaMemcpy(raw.data(), (const char *)base + (size_t)off * cs, raw.size(),
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    dst.resize((size_t)n);
    for (long long i = 0; i < n; ++i) {
      if (f64) {
        const double *d = (const double *)raw.data() + 2 * i;
        dst[i] = cd(d[0], d[1]);
      } else {
        const float *d = (const float *)raw.data() + 2 * i;
        dst[i] = cd(d[0], d[1]);
      }
    }
    return cudaSuccess;
  };
  if (alpha) {
    // stored in sorted point order [pos][t]: gamma^x * exp(2 pi i y'.xi_c) / N --
    // undo the centre factor and 1/N
    std::vector<cd> a;
    cudaError_t e = fetch(p->d_alpha, w.alpha_off, (long long)w.qp * NN, a);
    if (e != cudaSuccess) return cuda_fail(e, "export alpha");
    std::vector<uint2> Y((size_t)NN);
    e = cudaMemcpy(Y.data(), p->d_warp + (size_t)l * NN, sizeof(uint2) * NN, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "export warp");
    std::vector<uint32_t> perm((size_t)NN);
    e = cudaMemcpy(perm.data(), p->d_perm + (size_t)l * NN, sizeof(uint32_t) * NN,
                   cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "export point order");
    for (long long pos = 0; pos < NN; ++pos) {
      const long long x = perm[pos];
      const uint32_t yk = Y[x].x * (uint32_t)w.xc1 + Y[x].y * (uint32_t)w.xc2;
      const double ang = 2.0 * M_PI * ((double)yk * 2.3283064365386962890625e-10);
      const cd undo = std::polar((double)p->N, -ang);
      for (int t = 0; t < w.q; ++t) {
        const cd v = a[(size_t)(pos * w.qp + t)] * undo;
        alpha[2 * ((size_t)t * NN + x)] = v.real();
        alpha[2 * ((size_t)t * NN + x) + 1] = v.imag();
      }
    }
  }
  if (beta) {
    // stored: gamma^xi / (phihat(xi'_1/m1) phihat(xi'_2/m2))
    std::vector<cd> b;
    cudaError_t e = fetch(p->d_beta, w.beta_off, (long long)w.q * w.npts, b);
    if (e != cudaSuccess) return cuda_fail(e, "export beta");
    for (int i = 0; i < w.npts; ++i) {
      const int kk1 = p->pt_k1[w.pt_off + i], kk2 = p->pt_k2[w.pt_off + i];
      const int x1 = w.M[0] * kk1 + w.M[1] * kk2 - w.xc1, x2 = w.M[2] * kk1 + w.M[3] * kk2 - w.xc2;
      const double ph = kb_phihat_host((double)x1 / w.m1, p->kb.w, p->kb.beta) *
                        kb_phihat_host((double)x2 / w.m2, p->kb.w, p->kb.beta);
      for (int t = 0; t < w.q; ++t) {
        const cd v = b[(size_t)t * w.npts + i] * ph;
        beta[2 * ((size_t)t * w.npts + i)] = v.real();
        beta[2 * ((size_t)t * w.npts + i) + 1] = v.imag();
      }
    }
  }
  for (int i = 0; i < w.npts; ++i) {
    if (k1) k1[i] = p->pt_k1[w.pt_off + i];
    if (k2) k2[i] = p->pt_k2[w.pt_off + i];
  }
  return FIO_OK;
}

fio_status fio_plan_export_warp(fio_plan p, int l, double *y) {
  if (!plan_ok(p) || l < 0 || l >= p->L || !y) {
    set_error("fio_plan_export_warp: bad arguments");
    return FIO_EINVAL;
  }
  const long long NN = (long long)p->N * p->N;
  std::vector<uint2> Y((size_t)NN);
  cudaError_t e =
      cudaMemcpy(Y.data(), p->d_warp + (size_t)l * NN, sizeof(uint2) * NN, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "export warp");
  for (long long x = 0; x < NN; ++x) {
    y[2 * x] = (double)Y[x].x * 2.3283064365386962890625e-10;
    y[2 * x + 1] = (double)Y[x].y * 2.3283064365386962890625e-10;
  }
  return FIO_OK;
}

fio_status fio_dft2(int N, int precision, const void *in, void *out, int batch, int inverse,
                    void *stream) {
  if (N < 8 || N > kMaxFftLen || (N & 1) || fft_factor(N).empty()) {
    set_error("fio_dft2: N must be 2^a 3^b 5^c, even, 8 <= N <= 4096");
    return FIO_EINVAL;
  }
  if (!in || !out || batch < 1 || (precision != FIO_MIXED && precision != FIO_FP64)) {
    set_error("fio_dft2: bad arguments");
    return FIO_EINVAL;
  }
  FftPlanDev pl{};
  pl.n = N;
  const auto rad = fft_factor(N);
  pl.nstages = (int)rad.size();
  for (size_t i = 0; i < rad.size(); ++i) pl.radix[i] = rad[i];
  cudaError_t e = launch_dft2(N, precision, in, out, batch, inverse ? 1 : 0, &pl, nullptr,
                              (cudaStream_t)stream);
  return e == cudaSuccess ? FIO_OK : cuda_fail(e, "fio_dft2");
}

// ------------------------------------------------------------ host utilities

int fio_default_wedges(int N) { return default_L(N); }

int fio_kb_width_for(double eps) { return kb_width_for(eps); }

fio_status fio_wedge_map(int N, int L, int *wedge_of_out) {
  if (N < 2 || (N & 1) || L < 1 || !wedge_of_out) {
    set_error("fio_wedge_map: bad arguments");
    return FIO_EINVAL;
  }
  for (int i1 = 0; i1 < N; ++i1)
    for (int i2 = 0; i2 < N; ++i2)
      wedge_of_out[(size_t)i1 * N + i2] = wedge_of(i1 - N / 2, i2 - N / 2, L);
  return FIO_OK;
}

fio_status fio_wedge_geometry(int N, int L, double sigma, int kb_width, int l,
                              fio_wedge_info *info) {
  if (N < 2 || (N & 1) || L < 1 || l < 0 || l >= L || !info || kb_width < 2 || sigma < 1.0) {
    set_error("fio_wedge_geometry: bad arguments");
    return FIO_EINVAL;
  }
  std::vector<std::pair<int, int>> pts;
  for (int k1 = -N / 2; k1 < N / 2; ++k1)
    for (int k2 = -N / 2; k2 < N / 2; ++k2)
      if (wedge_of(k1, k2, L) == l) pts.push_back({k1, k2});
  if (pts.empty()) {
    set_error("empty wedge");
    return FIO_EINVAL;
  }
  WedgeDev wd;
  std::vector<RowDev> rows;
  std::vector<int> a, b, c, d;
  std::string err;
  if (!wedge_geometry(pts, sigma, kb_width, wd, rows, a, b, c, d, err)) {
    set_error(err);
    return FIO_EINVAL;
  }
  std::memset(info, 0, sizeof(*info));
  std::memcpy(info->M, wd.M, sizeof(info->M));
  info->xc1 = wd.xc1;
  info->xc2 = wd.xc2;
  info->b1 = wd.b1;
  info->n1 = wd.n1;
  info->b2 = wd.b2;
  info->n2 = wd.n2;
  info->m1 = wd.m1;
  info->m2 = wd.m2;
  info->npts = wd.npts;
  return FIO_OK;
}

fio_status fio_kb_eval(int w, double beta, int n, const double *s, double *phi, const double *nu,
                       double *phihat) {
  if (w < 2 || w > kMaxKbWidth || n < 0) {
    set_error("fio_kb_eval: bad arguments");
    return FIO_EINVAL;
  }
  if (beta <= 0) beta = kb_beta_for(w, 2.0);
  for (int i = 0; i < n; ++i) {
    if (phi && s) phi[i] = kb_phi_host(s[i], w, beta);
    if (phihat && nu) phihat[i] = kb_phihat_host(nu[i], w, beta);
  }
  return FIO_OK;
}

fio_status fio_host_eigh(int n, const double *A, double *evals, double *V) {
  if (n < 1 || n > 1024 || !A || !evals || !V) {
    set_error("fio_host_eigh: bad arguments");
    return FIO_EINVAL;
  }
  using cd = std::complex<double>;
  std::vector<cd> M((size_t)n * n);
  for (size_t i = 0; i < M.size(); ++i) M[i] = cd(A[2 * i], A[2 * i + 1]);
  std::vector<double> ev;
  std::vector<cd> Vm;
  herm_eig(n, M, ev, Vm);
  for (int i = 0; i < n; ++i) evals[i] = ev[i];
  for (size_t i = 0; i < Vm.size(); ++i) {
    V[2 * i] = Vm[i].real();
    V[2 * i + 1] = Vm[i].imag();
  }
  return FIO_OK;
}

fio_status fio_host_svd(int m, int n, const double *A, double *s, double *AV, double *V) {
  if (m < 1 || m > (1 << 20) || n < 1 || n > 1024 || !A) {
    set_error("fio_host_svd: bad arguments");
    return FIO_EINVAL;
  }
  using cd = std::complex<double>;
  std::vector<cd> M((size_t)m * n);
  for (size_t i = 0; i < M.size(); ++i) M[i] = cd(A[2 * i], A[2 * i + 1]);
  std::vector<double> sig;
  std::vector<cd> Vm;
  svd_jacobi(m, n, M, sig, Vm);
  for (int i = 0; s && i < n; ++i) s[i] = sig[i];
  for (size_t i = 0; AV && i < M.size(); ++i) {
    AV[2 * i] = M[i].real();
    AV[2 * i + 1] = M[i].imag();
  }
  for (size_t i = 0; V && i < Vm.size(); ++i) {
    V[2 * i] = Vm[i].real();
    V[2 * i + 1] = Vm[i].imag();
  }
  return FIO_OK;
}

fio_status fio_host_svd_right(int n, const double *R, double *s, double *V) {
  if (n < 1 || n > 2048 || !R || !s || !V) {
    set_error("fio_host_svd_right: bad arguments");
    return FIO_EINVAL;
  }
  using cd = std::complex<double>;
  std::vector<cd> M((size_t)n * n);
  for (size_t i = 0; i < M.size(); ++i) M[i] = cd(R[2 * i], R[2 * i + 1]);
  std::vector<double> sig;
  std::vector<cd> Vm;
  svd_right_pivoted(n, M, sig, Vm);
  for (int i = 0; i < n; ++i) s[i] = sig[i];
  for (size_t i = 0; i < Vm.size(); ++i) {
    V[2 * i] = Vm[i].real();
    V[2 * i + 1] = Vm[i].imag();
  }
  return FIO_OK;
}

}  // extern "C"
