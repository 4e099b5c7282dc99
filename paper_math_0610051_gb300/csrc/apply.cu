// apply.cu -- the evaluation step of the wedge-factorised FIO (Sec. 3.4) and
// its adjoint (Sec. 3.5), as sm_103a kernels templated on the real type
// (float: the mixed path, double: the FP64 path).
//
// Forward, for each input b:
//   S0  fhat = unitary 2D DFT of f                                   (Eq. dft)
//   S1  for every wedge l, rank term t and box row xi'_1: place
//       beta'_t(xi) fhat(xi) at xi'_2 mod m2 (beta' = gamma^xi / phihat) and
//       FFT the row (exp(+2 pi i)) -- the "form fhat_{l t}" step
//   S2  FFT every grid column over the box rows (exp(+2 pi i))
//   S3  for every x: KB-interpolate each grid G_{l t} at the warped point
//       u = y'_l(x) m, multiply by alpha'_t(x) (gamma^x with the centre-frequency
//       factor exp(2 pi i y'.xi_c) and 1/N folded in), sum over t and l.
// Adjoint: S4a spread conj(alpha') g onto the grids (type-1), S4b forward
// FFTs (exp(-2 pi i)) with pruned output, S4c sum_t conj(beta') G into the
// owner wedge's frequencies, S4d inverse unitary DFT.
//
// Grid layout: wedge l's grid is [g1 < m1][g2 < m2][ch < B qp_l], ch = b qp_l + t
// (qp_l = q_l rounded up to even; the padded term has zero factors).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "apply_common.cuh"
#include "fft_engine.cuh"
#include "fio_internal.h"

namespace fio {

// Lines per CTA of an in-place line FFT of length n (S1, S2, S4b): the CTA's
// buffer holds 8192 complex64 or 4096 complex128 values (64 KB), and a line
// transfer is at most 32 elements wide.
__host__ __device__ inline int fft_lines(int n, int prec) {
  const int elems = prec == FIO_FP64 ? 4096 : 8192;
  const int nl = elems / n;
  return nl < 1 ? 1 : (nl > 32 ? 32 : nl);
}
constexpr int kFftThreads = 512;  // threads of the in-place line-FFT kernels
// CTAs per SM of the column FFT: two for complex64 (64 registers a thread), so
// that one CTA's loads and stores overlap the other's butterfly stages.
template <typename T> constexpr int kFftCtas = sizeof(T) == 4 ? 2 : 1;
template <typename T> __host__ __device__ constexpr int prec_of() {
  return sizeof(T) == 4 ? FIO_MIXED : FIO_FP64;
}

// --------------------------------------------------------------- S0 / S4d --
// Unitary 2D DFT passes.  Rows: lines are rows of N contiguous elements.
// load index (e + load_shift) mod N, store index (e + store_shift) mod N.
// REAL: the input holds real values (T), read as x + 0i; the first pass of a
// real f, which reads half the bytes of its complex form.
template <typename T, bool REAL = false>
__global__ void __launch_bounds__(kThreads)
k_dft_rows(const void *in_v, Cx<T> *out, int N, int nrows, int nl, int sign, int load_shift,
           int store_shift, FftPlanDev pl, const Cx<T> *tw_g) {
  using C = Cx<T>;
  extern __shared__ unsigned char smem_raw[];
  C *a = reinterpret_cast<C *>(smem_raw);
  C *b = a + N * nl;
  C *tw = b + N * nl;
  const int r0 = blockIdx.x * nl;
  const int nlc = min(nl, nrows - r0);
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    if (tw_g) {
      tw[k] = tw_g[k];
    } else {
      T s, c;
      if constexpr (sizeof(T) == 4) sincospif(-2.0f * (float)k / (float)N, &s, &c);
      else sincospi(-2.0 * (double)k / (double)N, &s, &c);
      tw[k] = C{c, s};
    }
  }
  if constexpr (REAL) {
    const T *in = static_cast<const T *>(in_v);
    for (int it = threadIdx.x; it < N * nlc; it += blockDim.x) {
      const int e = it % N, l = it / N;
      a[e * nlc + l] = C{in[(size_t)(r0 + l) * N + (e + load_shift) % N], T(0)};
    }
  } else {
    const C *in = static_cast<const C *>(in_v);
    for (int it = threadIdx.x; it < N * nlc; it += blockDim.x) {
      const int e = it % N, l = it / N;
      cp_async_elem(&a[e * nlc + l], &in[(size_t)(r0 + l) * N + (e + load_shift) % N]);
    }
    cp_async_wait();
  }
  __syncthreads();
  C *res = fft_exec(a, b, N, nlc, pl, sign, tw);
  for (int it = threadIdx.x; it < N * nlc; it += blockDim.x) {
    const int e = it % N, l = it / N;
    out[(size_t)(r0 + l) * N + (e + store_shift) % N] = res[e * nlc + l];
  }
}

// Columns: lines are nl consecutive columns of one N x N array.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_dft_cols(const Cx<T> *in, Cx<T> *out, int N, int nl, int sign, int load_shift, int store_shift,
           T scale, FftPlanDev pl, const Cx<T> *tw_g) {
  using C = Cx<T>;
  extern __shared__ unsigned char smem_raw[];
  C *a = reinterpret_cast<C *>(smem_raw);
  C *b = a + N * nl;
  C *tw = b + N * nl;
  const int chunks = (N + nl - 1) / nl;
  const int bb = blockIdx.x / chunks;
  const int c0 = (blockIdx.x % chunks) * nl;
  const int nlc = min(nl, N - c0);
  const size_t base = (size_t)bb * N * N + c0;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    if (tw_g) {
      tw[k] = tw_g[k];
    } else {
      T s, c;
      if constexpr (sizeof(T) == 4) sincospif(-2.0f * (float)k / (float)N, &s, &c);
      else sincospi(-2.0 * (double)k / (double)N, &s, &c);
      tw[k] = C{c, s};
    }
  }
  for (int it = threadIdx.x; it < N * nlc; it += blockDim.x) {
    const int l = it % nlc, e = it / nlc;
    cp_async_elem(&a[e * nlc + l], &in[base + (size_t)((e + load_shift) % N) * N + l]);
  }
  cp_async_wait();
  __syncthreads();
  C *res = fft_exec(a, b, N, nlc, pl, sign, tw);
  for (int it = threadIdx.x; it < N * nlc; it += blockDim.x) {
    const int l = it % nlc, e = it / nlc;
    out[base + (size_t)((e + store_shift) % N) * N + l] = cscale(res[e * nlc + l], scale);
  }
}

// ----------------------------------------------------------------- S1 ------
// One CTA per (box row, chunk of fft_lines(m2) channels): scatter beta' fhat into
// the zero-padded row and FFT it along g2 with exp(+2 pi i), in place.
template <typename T>
__global__ void __launch_bounds__(kFftThreads)
k_scatter_rowfft(const Cx<T> *__restrict__ fhat, const WedgeDev *__restrict__ W,
                 const RowDev *__restrict__ rows, const FftPlanDev *__restrict__ ffts,
                 const Cx<T> *__restrict__ tw_all, const Cx<T> *__restrict__ beta,
                 Cx<T> *__restrict__ grid, int N, int B) {
  using C = Cx<T>;
  extern __shared__ unsigned char smem_raw[];
  const RowDev rw = rows[blockIdx.x];
  const WedgeDev w = W[rw.wedge];
  const int nch = B * w.qp;
  const int n = w.m2;
  const int nl = fft_lines(n, prec_of<T>());
  const int c0 = blockIdx.y * nl;
  if (c0 >= nch) return;
  const int nlc = min(nl, nch - c0);
  C *a = reinterpret_cast<C *>(smem_raw);
  C *tw = a + n * nl;
  short *pos = reinterpret_cast<short *>(tw + n);
  const FftPlanDev pl = ffts[w.fft2];
  for (int k = threadIdx.x; k < n; k += blockDim.x) tw[k] = tw_all[w.tw2_off + k];
  for (int k = threadIdx.x; k < n * nlc; k += blockDim.x) a[k] = C{0, 0};
  fft_dif_table(pos, pl);
  __syncthreads();
  const int k1pp = rw.xi1 + w.xc1;
  const LineMap lm = line_map(nlc);
  if ((int)threadIdx.x < lm.lanes) {
    const int ch = c0 + lm.l, bb = ch / w.qp, t = ch - bb * w.qp;
    const C *bt = beta + w.beta_off + (long long)t * w.npts + rw.pt;
    const C *fb = fhat + (size_t)bb * N * N;
    for (int j = lm.i0; j < rw.len; j += lm.step) {
      const int x2p = rw.a + j;
      const int k2pp = x2p + w.xc2;
      const int k1 = w.Minv[0] * k1pp + w.Minv[1] * k2pp;
      const int k2 = w.Minv[2] * k1pp + w.Minv[3] * k2pp;
      // k1, k2 in [-N/2, N/2) and x2p in (-n, n): one conditional add each
      const size_t idx = (size_t)(k1 < 0 ? k1 + N : k1) * N + (k2 < 0 ? k2 + N : k2);
      a[(x2p < 0 ? x2p + n : x2p) * nlc + lm.l] = cmul(bt[j], fb[idx]);
    }
  }
  __syncthreads();
  fft_exec_dif<+1>(a, n, nlc, pl, tw);
  C *out = grid + w.grid_unit * B + (long long)(rw.xi1 < 0 ? rw.xi1 + w.m1 : rw.xi1) * n * nch + c0;
  if ((int)threadIdx.x < lm.lanes)
    for (int e = lm.i0; e < n; e += lm.step) out[(long long)e * nch + lm.l] = a[pos[e] * nlc + lm.l];
}

// ------------------------------------------------------------ S2 / S4b -----
// Column FFTs along g1, in place.  A CTA owns fft_lines(m1) consecutive entries
// of the flattened [g2][ch] dimension of one wedge.  adjoint = 0: input rows
// outside the box are zero (not read), all m1 outputs written, exp(+2 pi i).
// adjoint = 1: all rows read, only box rows written, exp(-2 pi i).
// First column block of every wedge (a prefix sum over the wedges, made on the
// host for the launch's batch): the CTA finds its wedge by binary search.
struct ColBlocks {
  int L;
  int start[kMaxWedges + 1];
};

template <typename T>
__global__ void __launch_bounds__(kFftThreads, kFftCtas<T>)
k_colfft(Cx<T> *__restrict__ grid, const WedgeDev *__restrict__ W,
         const FftPlanDev *__restrict__ ffts, const Cx<T> *__restrict__ tw_all,
         const ColBlocks cb, int B, int adjoint) {
  using C = Cx<T>;
  extern __shared__ unsigned char smem_raw[];
  int lo = 0, hi = cb.L - 1;  // the wedge with start[l] <= blockIdx.x < start[l + 1]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cb.start[mid] <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const int l = lo, blk = blockIdx.x - cb.start[l];
  const WedgeDev w = W[l];
  const int nl = fft_lines(w.m1, prec_of<T>());
  const int nch = B * w.qp;
  const long long rs = (long long)w.m2 * nch;  // row stride
  const long long cc0 = (long long)blk * nl;
  const int nlc = (int)min((long long)nl, rs - cc0);
  const int n = w.m1;
  C *a = reinterpret_cast<C *>(smem_raw);
  C *tw = a + n * nl;
  short *pos = reinterpret_cast<short *>(tw + n);
  const FftPlanDev pl = ffts[w.fft1];
  C *g = grid + w.grid_unit * B + cc0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) tw[k] = tw_all[w.tw1_off + k];
  fft_dif_table(pos, pl);
  const LineMap lm = line_map(nlc);
  const bool on = (int)threadIdx.x < lm.lanes;
  const int c = lm.l;
  if (!adjoint) {
    for (int k = threadIdx.x; k < n * nlc; k += blockDim.x) a[k] = C{0, 0};
    __syncthreads();
    if (on)
      for (int e = lm.i0; e < w.n1; e += lm.step) {
        int g1 = w.b1 + e;  // box row, -n < g1 < n
        if (g1 < 0) g1 += n;
        cp_async_elem(&a[g1 * nlc + c], &g[g1 * rs + c]);
      }
  } else if (on) {
    for (int e = lm.i0; e < n; e += lm.step) cp_async_elem(&a[e * nlc + c], &g[e * rs + c]);
  }
  cp_async_wait();
  __syncthreads();
  if (adjoint) fft_exec_dif<-1>(a, n, nlc, pl, tw);
  else fft_exec_dif<+1>(a, n, nlc, pl, tw);
  if (!on) return;
  if (!adjoint) {
    for (int e = lm.i0; e < n; e += lm.step) g[e * rs + c] = a[pos[e] * nlc + c];
  } else {
    for (int e = lm.i0; e < w.n1; e += lm.step) {
      int g1 = w.b1 + e;
      if (g1 < 0) g1 += n;
      g[g1 * rs + c] = a[pos[g1] * nlc + c];
    }
  }
}

// ---------------------------------------------------------------- S4b rows --
// Row FFT along g2 with exp(-2 pi i) for each box row, in place; only the
// run's columns are written back.
template <typename T>
__global__ void __launch_bounds__(kFftThreads)
k_rowfft_adj(Cx<T> *__restrict__ grid, const WedgeDev *__restrict__ W,
             const RowDev *__restrict__ rows, const FftPlanDev *__restrict__ ffts,
             const Cx<T> *__restrict__ tw_all, int B) {
  using C = Cx<T>;
  extern __shared__ unsigned char smem_raw[];
  const RowDev rw = rows[blockIdx.x];
  const WedgeDev w = W[rw.wedge];
  const int nch = B * w.qp;
  const int n = w.m2;
  const int nl = fft_lines(n, prec_of<T>());
  const int c0 = blockIdx.y * nl;
  if (c0 >= nch || rw.len == 0) return;
  const int nlc = min(nl, nch - c0);
  C *a = reinterpret_cast<C *>(smem_raw);
  C *tw = a + n * nl;
  short *pos = reinterpret_cast<short *>(tw + n);
  const FftPlanDev pl = ffts[w.fft2];
  C *row = grid + w.grid_unit * B + (long long)imodp(rw.xi1, w.m1) * n * nch + c0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) tw[k] = tw_all[w.tw2_off + k];
  fft_dif_table(pos, pl);
  const LineMap lm = line_map(nlc);
  const bool on = (int)threadIdx.x < lm.lanes;
  if (on)
    for (int e = lm.i0; e < n; e += lm.step)
      cp_async_elem(&a[e * nlc + lm.l], &row[(long long)e * nch + lm.l]);
  cp_async_wait();
  __syncthreads();
  fft_exec_dif<-1>(a, n, nlc, pl, tw);
  if (on)
    for (int j = lm.i0; j < rw.len; j += lm.step) {
      const int g2 = imodp(rw.a + j, n);
      row[(long long)g2 * nch + lm.l] = a[pos[g2] * nlc + lm.l];
    }
}

// ---------------------------------------------------------------- S4c ------
// fhat_adj(xi) = sum_t conj(beta'_t(xi)) Ghat_{l t}(xi') for the owner wedge.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_gather_adj(const Cx<T> *__restrict__ grid, const WedgeDev *__restrict__ W,
             const RowDev *__restrict__ rows, const Cx<T> *__restrict__ beta,
             Cx<T> *__restrict__ fhat, int N, int B) {
  using C = Cx<T>;
  const RowDev rw = rows[blockIdx.x];
  const WedgeDev w = W[rw.wedge];
  const int nch = B * w.qp;
  const C *row = grid + w.grid_unit * B + (long long)imodp(rw.xi1, w.m1) * w.m2 * nch;
  const int k1pp = rw.xi1 + w.xc1;
  for (int it = threadIdx.x; it < rw.len * B; it += blockDim.x) {
    const int j = it % rw.len, bb = it / rw.len;
    const int x2p = rw.a + j;
    const C *cell = row + (long long)imodp(x2p, w.m2) * nch + bb * w.qp;
    C acc{0, 0};
    for (int t = 0; t < w.qp; ++t)
      acc = cadd(acc, cmulc(cell[t], beta[w.beta_off + (long long)t * w.npts + rw.pt + j]));
    const int k2pp = x2p + w.xc2;
    const int k1 = w.Minv[0] * k1pp + w.Minv[1] * k2pp;
    const int k2 = w.Minv[2] * k1pp + w.Minv[3] * k2pp;
    fhat[(size_t)bb * N * N + (size_t)imodp(k1, N) * N + imodp(k2, N)] = acc;
  }
}

// ============================================================= launchers ===

size_t apply_smem_bytes(int n, int nl, int precision) {
  const size_t cs = precision == FIO_FP64 ? 16 : 8;
  return (2 * (size_t)n * nl + n) * cs;
}

static int pick_nl(int n, int precision, int want) {
  const size_t budget = 96 * 1024;
  int nl = want;
  while (nl > 1 && apply_smem_bytes(n, nl, precision) > budget) nl >>= 1;
  return nl;
}

// Dynamic shared memory above the 48 KB default.  max_shared: also ask for the
// largest shared-memory carveout, so that two CTAs of the column FFT fit on an
// SM (the row kernels gather through L1 and keep the default split).
template <typename K> static cudaError_t set_smem(K kernel, size_t bytes, bool max_shared = false) {
  cudaError_t e = cudaSuccess;
  if (max_shared)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess || bytes <= 48 * 1024) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T>
static cudaError_t dft2_impl(int N, const void *in, void *out, int batch, int inverse,
                             const FftPlanDev &pl, const void *d_tw, bool centred,
                             cudaStream_t s, bool real_in = false) {
  using C = Cx<T>;
  const int prec = sizeof(T) == 8 ? FIO_FP64 : FIO_MIXED;
  const int nl = pick_nl(N, prec, 16);
  const size_t smem = apply_smem_bytes(N, nl, prec);
  cudaError_t e;
  if ((e = set_smem(k_dft_rows<T>, smem)) != cudaSuccess) return e;
  if ((e = set_smem(k_dft_rows<T, true>, smem)) != cudaSuccess) return e;
  if ((e = set_smem(k_dft_cols<T>, smem)) != cudaSuccess) return e;
  const int sign = inverse ? +1 : -1;
  const int sh = centred ? N / 2 : 0;
  const int nrows = batch * N;
  // rows: forward stores shifted, inverse loads shifted
  if (real_in)
    k_dft_rows<T, true><<<(nrows + nl - 1) / nl, kThreads, smem, s>>>(
        in, (C *)out, N, nrows, nl, sign, inverse ? sh : 0, inverse ? 0 : sh, pl, (const C *)d_tw);
  else
    k_dft_rows<T><<<(nrows + nl - 1) / nl, kThreads, smem, s>>>(
        in, (C *)out, N, nrows, nl, sign, inverse ? sh : 0, inverse ? 0 : sh, pl, (const C *)d_tw);
  const int chunks = (N + nl - 1) / nl;
  k_dft_cols<T><<<batch * chunks, kThreads, smem, s>>>((const C *)out, (C *)out, N, nl, sign,
                                                      inverse ? sh : 0, inverse ? 0 : sh,
                                                      T(1.0) / T(N), pl, (const C *)d_tw);
  return cudaGetLastError();
}

cudaError_t launch_dft2(int N, int precision, const void *in, void *out, int batch, int inverse,
                        const FftPlanDev *plan, const void *d_tw, cudaStream_t s) {
  if (precision == FIO_FP64) return dft2_impl<double>(N, in, out, batch, inverse, *plan, d_tw, true, s);
  return dft2_impl<float>(N, in, out, batch, inverse, *plan, d_tw, true, s);
}


struct LaunchGeom {
  int max_m1 = 0, max_m2 = 0, max_q = 0, col_blocks = 0, row_chunks = 0;
  size_t smem_col = 0, smem_row = 0;
  ColBlocks cb{};
};

// Launch shapes of the in-place line FFTs: column blocks, row-chunk count and
// the largest shared buffers (n * fft_lines(n) values, n twiddles, n slots).
static LaunchGeom geom(const fio_plan_s *p, int B) {
  LaunchGeom g;
  const int prec = p->precision;
  const size_t cs = prec == FIO_FP64 ? 16 : 8;
  for (const auto &w : p->wedges) {
    g.max_m1 = std::max(g.max_m1, w.m1);
    g.max_m2 = std::max(g.max_m2, w.m2);
    g.max_q = std::max(g.max_q, w.qp);
    const int nl1 = fft_lines(w.m1, prec), nl2 = fft_lines(w.m2, prec);
    g.cb.start[g.cb.L++] = g.col_blocks;
    g.col_blocks += (w.m2 * B * w.qp + nl1 - 1) / nl1;
    g.row_chunks = std::max(g.row_chunks, (B * w.qp + nl2 - 1) / nl2);
    g.smem_col = std::max(g.smem_col, ((size_t)w.m1 * nl1 + w.m1) * cs + ((size_t)w.m1 * 2 + 15) / 16 * 16);
    g.smem_row = std::max(g.smem_row, ((size_t)w.m2 * nl2 + w.m2) * cs + ((size_t)w.m2 * 2 + 15) / 16 * 16);
  }
  return g;
}

// Per-stage timing: a (start, stop) event pair recorded around a stage on the
// launch stream when the plan's timing flag is set.
struct StageTimer {
  const fio_plan_s *p;
  cudaStream_t s;
  size_t pair = (size_t)-1;
  StageTimer(const fio_plan_s *plan, cudaStream_t st, int stage, bool allowed = true)
      : p(plan), s(st) {
    if (!allowed || !p->timing) return;
    if (2 * (p->ev_used + 1) > p->ev_pool.size()) {
      cudaEvent_t a, b;
      if (cudaEventCreate(&a) != cudaSuccess) return;
      if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
      p->ev_pool.push_back(a);
      p->ev_pool.push_back(b);
    }
    pair = p->ev_used++;
    if (p->ev_stage.size() < p->ev_used) p->ev_stage.resize(p->ev_used);
    p->ev_stage[pair] = stage;
    cudaEventRecord(p->ev_pool[2 * pair], s);
  }
  ~StageTimer() {
    if (pair != (size_t)-1) cudaEventRecord(p->ev_pool[2 * pair + 1], s);
  }
};

void release_timing_events(fio_plan_s *p) {
  for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
  p->ev_pool.clear();
  p->ev_stage.clear();
  p->ev_used = 0;
}

static FftPlanDev plan_for_N(const fio_plan_s *p, const void **tw) {
  for (const auto &f : p->ffts)
    if (f.n == p->N) {
      *tw = (const char *)p->d_twiddle + (size_t)f.tw_off * (p->precision == FIO_FP64 ? 16 : 8);
      return f;
    }
  *tw = nullptr;
  return FftPlanDev{};
}

template <typename T>
static cudaError_t apply_impl(const fio_plan_s *p, const void *f, void *out, int B,
                              cudaStream_t s, void *grid_ws, void *fhat_ws, bool timing,
                              bool real_in) {
  using C = Cx<T>;
  const int N = p->N, L = p->L;
  const void *twN;
  const FftPlanDev plN = plan_for_N(p, &twN);
  cudaError_t e;
  // S0: fhat in natural order (no centring shift)
  {
    StageTimer st(p, s, FIO_STAGE_S0_DFT, timing);
    e = dft2_impl<T>(N, f, fhat_ws, B, 0, plN, twN, false, s, real_in);
    p->launches += 2;
  }
  if (e != cudaSuccess) return e;
  const LaunchGeom g0 = geom(p, B);
  // S1
  if ((e = set_smem(k_scatter_rowfft<T>, g0.smem_row)) != cudaSuccess) return e;
  {
    StageTimer st(p, s, FIO_STAGE_S1_SCATTER, timing);
    k_scatter_rowfft<T><<<dim3((unsigned)p->rows.size(), (unsigned)g0.row_chunks), kFftThreads,
                          g0.smem_row, s>>>((const C *)fhat_ws, p->d_wedges, p->d_rows, p->d_ffts,
                                            (const C *)p->d_twiddle, (const C *)p->d_beta,
                                            (C *)grid_ws, N, B);
    p->launches += 1;
  }
  // S2
  if ((e = set_smem(k_colfft<T>, g0.smem_col, true)) != cudaSuccess) return e;
  {
    StageTimer st(p, s, FIO_STAGE_S2_COLFFT, timing);
    k_colfft<T><<<g0.col_blocks, kFftThreads, g0.smem_col, s>>>((C *)grid_ws, p->d_wedges, p->d_ffts,
                                                            (const C *)p->d_twiddle, g0.cb, B, 0);
    p->launches += 1;
  }
  // S3 (recompute mode: gamma^x of a group of wedges is formed, then their
  // points are interpolated, group after group; the stage time includes both)
  {
    StageTimer st(p, s, FIO_STAGE_S3_INTERP, timing);
    if (p->alpha_mode == FIO_ALPHA_RECOMPUTE) {
      for (int g = 0; g + 1 < (int)p->grp_first.size(); ++g) {
        if ((e = regen_alpha(p, g, s)) != cudaSuccess) return e;
        if ((e = launch_interp(p, grid_ws, out, B, s, group_range(p, g, g == 0))) != cudaSuccess)
          return e;
        p->launches += 2;
      }
    } else {
      e = launch_interp(p, grid_ws, out, B, s, full_range(p));
      if (e != cudaSuccess) return e;
      p->launches += 1;
    }
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t adjoint_impl(const fio_plan_s *p, const void *gin, void *out, int B,
                                cudaStream_t s) {
  using C = Cx<T>;
  const int N = p->N, L = p->L;
  cudaError_t e;
  // S4a (writes every grid cell)
  {
    StageTimer st(p, s, FIO_STAGE_S4A_SPREAD);
    if (p->alpha_mode == FIO_ALPHA_RECOMPUTE) {
      for (int g = 0; g + 1 < (int)p->grp_first.size(); ++g) {
        if ((e = regen_alpha(p, g, s)) != cudaSuccess) return e;
        if ((e = launch_spread(p, gin, p->d_grid, B, s, group_range(p, g, false))) != cudaSuccess)
          return e;
        p->launches += 2;
      }
    } else {
      e = launch_spread(p, gin, p->d_grid, B, s, full_range(p));
      if (e != cudaSuccess) return e;
      p->launches += 1;
    }
  }
  // S4b columns
  const LaunchGeom g0 = geom(p, B);
  if ((e = set_smem(k_colfft<T>, g0.smem_col, true)) != cudaSuccess) return e;
  {
    StageTimer st(p, s, FIO_STAGE_S4B_COLFFT);
    k_colfft<T><<<g0.col_blocks, kFftThreads, g0.smem_col, s>>>((C *)p->d_grid, p->d_wedges,
                                                            p->d_ffts, (const C *)p->d_twiddle,
                                                            g0.cb, B, 1);
    p->launches += 1;
  }
  // S4b rows
  if ((e = set_smem(k_rowfft_adj<T>, g0.smem_row)) != cudaSuccess) return e;
  {
    StageTimer st(p, s, FIO_STAGE_S4B_ROWFFT);
    k_rowfft_adj<T><<<dim3((unsigned)p->rows.size(), (unsigned)g0.row_chunks), kFftThreads,
                      g0.smem_row, s>>>((C *)p->d_grid, p->d_wedges, p->d_rows, p->d_ffts,
                                        (const C *)p->d_twiddle, B);
    p->launches += 1;
  }
  // S4c
  {
    StageTimer st(p, s, FIO_STAGE_S4C_GATHER);
    k_gather_adj<T><<<(unsigned)p->rows.size(), kThreads, 0, s>>>(
        (const C *)p->d_grid, p->d_wedges, p->d_rows, (const C *)p->d_beta, (C *)p->d_fhat, N, B);
    p->launches += 1;
  }
  // S4d: inverse unitary DFT from natural order
  const void *twN;
  const FftPlanDev plN = plan_for_N(p, &twN);
  StageTimer st(p, s, FIO_STAGE_S4D_IDFT);
  p->launches += 2;
  return dft2_impl<T>(N, p->d_fhat, out, B, 1, plN, twN, false, s);
}

cudaError_t launch_apply(const fio_plan_s *p, const void *f, void *out, int batch,
                         cudaStream_t s, bool real_in) {
  return launch_apply_ws(p, f, out, batch, s, p->d_grid, p->d_fhat, true, real_in);
}

cudaError_t launch_apply_ws(const fio_plan_s *p, const void *f, void *out, int batch,
                            cudaStream_t s, void *grid_ws, void *fhat_ws, bool timing,
                            bool real_in) {
  if (p->precision == FIO_FP64)
    return apply_impl<double>(p, f, out, batch, s, grid_ws, fhat_ws, timing, real_in);
  return apply_impl<float>(p, f, out, batch, s, grid_ws, fhat_ws, timing, real_in);
}

cudaError_t launch_adjoint(const fio_plan_s *p, const void *g, void *out, int batch,
                           cudaStream_t s) {
  if (p->precision == FIO_FP64) return adjoint_impl<double>(p, g, out, batch, s);
  return adjoint_impl<float>(p, g, out, batch, s);
}

}  // namespace fio
