// fio_internal.h -- plan layout shared by the host code and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fio.h"

namespace fio {

constexpr int kMaxRadixStages = 16;
constexpr int kMaxWedges = 256;  // largest L a plan accepts
constexpr int kMaxFftLen = 4096;
constexpr int kMaxKbWidth = 12;
constexpr int kMaxHornerDeg = 15;
constexpr int kTauMmax = 8;  // tau-mode phases: angular orders m in [-8, 8]

// One FFT length: its radix factorisation (Stockham stages) and where its
// twiddle table exp(-2 pi i k / n), k < n, starts in the plan's table.
struct FftPlanDev {
  int n;
  int nstages;
  int radix[kMaxRadixStages];
  int tw_off;  // complex offset into the twiddle table
};

// One wedge W_l after the shear/translation of Sec. 3.4: xi' = M xi - xi_c.
struct WedgeDev {
  int M[4];       // xi'' = M xi (row-major), det M = 1
  int Minv[4];    // xi = Minv xi''
  int xc1, xc2;   // translation xi_c
  int b1, n1;     // rows    xi'_1 in [b1, b1 + n1)
  int b2, n2;     // columns xi'_2 in [b2, b2 + n2)
  int m1, m2;     // oversampled grid dims
  int q;          // separation rank
  int qp;         // q rounded up to even: rank terms stored per input (the padded term is zero)
  int npts;       // |W_l|
  int fft1, fft2;         // FftPlanDev index for lengths m1, m2
  int row_off;            // first RowDev of this wedge
  long long grid_unit;    // grid offset in units of complex * batch: sum_{l'<l} m1 m2 qp
  long long alpha_off;    // complex offset of alpha[l][0][0] (layout [pos][t])
  long long beta_off;     // complex offset of beta[l][0][0]  (layout [t][p])
  int pt_off;             // first point of this wedge in the global point order
  int tw1_off, tw2_off;   // twiddle offsets for m1 / m2 (copies of the FftPlanDev fields)
  int nb1, nb2;           // bins of kBin x kBin window-start cells per grid axis
  long long key_off;      // first entry of this wedge's bucket table (nb1 nb2 kBin^2 + 1 ints)
  int rc_r;               // recompute mode: sampled columns of this wedge
  long long rc_col_off;   // recompute mode: first RcCol of this wedge
  long long rc_w_off;     // recompute mode: first entry of V S^-1 ([k][qp], complex)
};

// One sampled column xi_c of a wedge in the recompute storage mode: the values
// the regeneration of gamma^x needs that do not depend on x, made in FP64 on
// the host (rounded to float for complex64 plans).
struct alignas(16) RcCol {
  int k1, k2;      // the frequency xi_c
  float ctk1;      // cos(theta_l) k1 (theta_l: the wedge's centre direction)
  float stk2;      // sin(theta_l) k2
  float cross2;    // (cos(theta_l) k2 - sin(theta_l) k1)^2
  float fk1, fk2;  // k1, k2 as floats
  float rsw;       // shift/wave phase: its residual, which does not depend on x
  float ampc;      // the amplitude's column factor (1 + a2 cos theta), or 1
  float pad[3];
};

// Phase and amplitude parameters on the device.
struct PhaseDev {
  int kind;          // FIO_PHASE_ELLIPSE_PRODUCT is carried as FIO_PHASE_ELLIPSE, ell_form = 1
  int nmodes;
  int ell_form;      // ellipse axes: 0 A + B sin sin / cos cos, 1 product form
  double p[8];       // scalar parameters (shift/wave, ellipse)
  int amp_kind;
  double a1, a2;
};

// Points of a wedge are sorted by the grid cell where their KB window starts,
// bin by bin (kBin x kBin start cells, row-major inside a bin), so that the
// points of one bin touch only a (kBin + w - 1)^2 cell footprint.
constexpr int kBin = 16;

// The bucket-table key of window-start cell (s1, s2) of a wedge with nb2 bins per row.
__host__ __device__ inline long long bin_key(int s1, int s2, int nb2) {
  return ((long long)(s1 / kBin) * nb2 + s2 / kBin) * (kBin * kBin) + (s1 % kBin) * kBin + s2 % kBin;
}

// Piecewise-polynomial KB weights for the FP32 path: with z = u - j0 - (w/2 - 1)
// in [0, 1) and t = 2z - 1, phi(u - j0 - a) = sum_k c[k][a] t^k.
struct HornerDev {
  int deg;
  float c[kMaxHornerDeg + 1][kMaxKbWidth];
};

// One box row xi'_1 = b1 + r: the wedge's frequencies on it are the contiguous
// run xi'_2 in [a, a + len) (a convex cone meets a lattice line in a run).
struct RowDev {
  int wedge;
  int xi1;     // xi'_1
  int a, len;  // run of xi'_2
  int pt;      // index of the run's first point within the wedge's point list
};

// KB kernel phi(s) = I0(beta sqrt(1 - (2s/w)^2)), |s| <= w/2.
struct KbParams {
  int w;
  double beta;
};

struct PlanHost;  // host-side mirror, defined in plan.cpp

}  // namespace fio

// The plan object behind the opaque fio_plan handle.
struct fio_plan_s {
  int N = 0, L = 0, precision = FIO_MIXED, max_batch = 1;
  double eps = 0, sigma = 2.0, plan_seconds = 0;
  fio::KbParams kb{};
  int q_max = 0, q_min = 0, r_max = 0;
  double sep_err = 0;
  int sur_warp = 0;
  double sur_warp_cycles = 0, sur_residual_cycles = 0;
  double q_mean = 0;
  int device = 0;

  // host copies of the tables
  std::vector<fio::WedgeDev> wedges;
  std::vector<fio::RowDev> rows;
  std::vector<fio::FftPlanDev> ffts;
  std::vector<int> wedge_r;
  std::vector<double> wedge_err;   // separation error estimate per wedge
  std::vector<int> pt_k1, pt_k2;   // every frequency, wedge by wedge, row-major in each box
  long long grid_units = 0;        // sum_l m1 m2 q
  long long alpha_elems = 0, beta_elems = 0;
  long long cstart_elems = 0;      // entries of all bucket tables
  long long twiddle_elems = 0;     // complex entries of the twiddle tables
  int max_row_len = 0;

  // device arrays
  fio::WedgeDev *d_wedges = nullptr;
  fio::RowDev *d_rows = nullptr;
  fio::FftPlanDev *d_ffts = nullptr;
  void *d_twiddle = nullptr;      // complex (float2 / double2) exp(-2 pi i k/n) tables
  void *d_alpha = nullptr;        // gamma^x * centre phase / N, [l][pos][t] (sorted point order);
                                  // recompute mode: the buffer of one group of wedges
  void *d_beta = nullptr;         // gamma^xi / phihat, [l][t][p]
  uint2 *d_warp = nullptr;        // warped points y' mod 1 as 32-bit fractions, [l][x]
  uint2 *d_warps = nullptr;       // the same in sorted point order, [l][pos]
  uint32_t *d_perm = nullptr;     // sorted position -> x = n1 N + n2, [l][pos]
  int *d_cstart = nullptr;        // per wedge: first sorted position of every bucket key (+ end)
  int4 *d_items = nullptr;        // interpolation work: (l, bin, first pos, end pos)
  int2 *d_bins = nullptr;         // FP64 spread work: (l, first bin of a pair of adjacent bins)
  int2 *d_bins1 = nullptr;        // mixed-precision spread work: (l, bin), every bin of every wedge
  int n_items = 0, n_bins = 0, n_bins1 = 0;
  fio::HornerDev horner{};
  void *d_grid = nullptr;         // NUFFT grids [l][g1][g2][b*q + t]
  void *d_fhat = nullptr;         // spectrum workspace, batch * N * N complex
  int *d_errword = nullptr;       // set by a kernel whose in-kernel bounds check fails
  int max_bin_pts = 0;            // most points in one bin
  double mean_bin_pts = 0;        // mean points per non-empty bin
  int max_cand = 0;               // most points whose windows reach one bin's cells
  size_t bytes_total = 0;
  unsigned long long alg_bytes = 0;

  // work lists per wedge: first item / bin pair / bin of wedge l (and the ends)
  std::vector<int> item_off, bin_off, bin1_off;

  // recompute storage mode (FIO_ALPHA_RECOMPUTE): d_alpha is the buffer of one
  // group of wedges, d_wedges_rc the wedge table whose alpha_off is relative to
  // the wedge's group
  int alpha_mode = FIO_ALPHA_STORED;
  std::vector<int> grp_first;           // first wedge of every group, then L
  std::vector<int> rc_r;                // sampled columns per wedge
  std::vector<long long> rc_col_off;    // first RcCol of wedge l
  std::vector<long long> rc_w_off;      // first entry of wedge l's V S^-1 ([k][qp], complex)
  long long rc_cols = 0, rc_w_elems = 0;
  long long rc_x_elems = 0;             // bytes of d_rc_x
  fio::WedgeDev *d_wedges_rc = nullptr;
  fio::RcCol *d_rc_col = nullptr;
  void *d_rc_w = nullptr;               // V S^-1 of every wedge, complex (plan precision)
  void *d_rc_g = nullptr;               // tau phases, complex64 plans: G_{m,c} per column [c][kNm]
  void *d_rc_x = nullptr;               // per-x phase data (complex64: floats; FP64: the plan's own)
  fio::PhaseDev phase{};

  // diagnostics: launch counter and optional per-stage CUDA-event timing
  mutable unsigned long long launches = 0;
  bool timing = false;
  mutable std::vector<cudaEvent_t> ev_pool;   // pairs (start, stop)
  mutable std::vector<int> ev_stage;          // stage of each used pair
  mutable size_t ev_used = 0;

};

namespace fio {

// Device bytes of the recompute mode's tables (columns, V S^-1, tau column
// factors, per-x phase data, the second wedge table); 0 in the stored mode.
inline size_t rc_bytes(const fio_plan_s *p) {
  if (p->alpha_mode != FIO_ALPHA_RECOMPUTE) return 0;
  const size_t cs = p->precision == FIO_FP64 ? 16 : 8;
  return (size_t)p->rc_cols * sizeof(RcCol) + (size_t)p->rc_w_elems * cs +
         (p->d_rc_g ? (size_t)p->rc_cols * (2 * kTauMmax + 1) * 8 : 0) + (size_t)p->rc_x_elems +
         p->wedges.size() * sizeof(WedgeDev);
}

// Thread-local error text (api.cpp).
void set_error(const std::string &msg);

// plan_io.cpp: the plan file of fio_plan_save / fio_plan_load
fio_status save_plan(const fio_plan_s *p, const char *path);
fio_status load_plan(fio_plan_s *p, const char *path, int max_batch);

// plan.cpp
fio_status build_plan(fio_plan_s *p, int N, const fio_phase *phase, const fio_amplitude *amp,
                      double eps, const fio_options *opt);
void free_plan_device(fio_plan_s *p);
// Recompute mode: the wedge table whose alpha_off places each wedge's gamma^x
// relative to its group (groups: wedges grp_first[g] .. grp_first[g + 1] - 1),
// and the buffer size the largest group needs.
std::vector<WedgeDev> rc_wedge_table(const std::vector<WedgeDev> &wedges,
                                     const std::vector<int> &grp_first, long long NN,
                                     long long *buf_elems);

// Host helpers shared by plan.cpp and the launchers.
std::vector<int> fft_factor(int n);   // radices (16, 8, 4, 2, 9, 3, 5), empty if n is not 2^a 3^b 5^c
int fft_good_size(int n);             // smallest even 2^a 3^b 5^c >= n

// apply.cu launchers (return cudaGetLastError()).
// real_in: f holds B x N x N real values (float or double as the plan's
// precision), read as x + 0i by the first DFT pass.
cudaError_t launch_apply(const fio_plan_s *p, const void *f, void *out, int batch,
                         cudaStream_t s, bool real_in = false);
cudaError_t launch_adjoint(const fio_plan_s *p, const void *g, void *out, int batch,
                           cudaStream_t s);
// The forward apply on caller-chosen workspace: grid_ws holds grid_units * batch
// complex values and fhat_ws N * N * batch; timing = false records no events.
cudaError_t launch_apply_ws(const fio_plan_s *p, const void *f, void *out, int batch,
                            cudaStream_t s, void *grid_ws, void *fhat_ws, bool timing,
                            bool real_in = false);
cudaError_t launch_dft2(int N, int precision, const void *in, void *out, int batch, int inverse,
                        const FftPlanDev *d_plan, const void *d_tw, cudaStream_t s);
size_t apply_smem_bytes(int n, int nl, int precision);
// interp.cu
constexpr int kItemPts = 1024;  // most points of one interpolation work item (w <= 6)
// Most points of one work item for KB width w: the mixed-precision S3 keeps the
// weights of a whole item in shared memory, so wider windows take smaller items.
inline int item_points(int w) { return w <= 6 ? kItemPts : kItemPts / 2; }
// Sort wedge l's points by window-start cell: fills d_perm[l], d_warps[l], the
// bucket table at d_cstart + key_off (synchronises; host counting sort, stable in x).
cudaError_t sort_wedge_points(fio_plan_s *p, int l, std::vector<int> &cstart_host);
// Work lists and bin statistics from every wedge's bucket table.
cudaError_t build_work_lists(fio_plan_s *p, const std::vector<std::vector<int>> &cstart);
void fit_horner(fio_plan_s *p);           // host: piecewise-polynomial KB weights
// The S3 / S4a work of one launch: the wedge table and the gamma^x array the
// kernels read (a wedge's factors at alpha + alpha_off), and the sub-lists of
// interpolation items, FP64 spread bin pairs and mixed-precision spread bins.
// The stored mode runs every wedge in one launch; the recompute mode one group
// of wedges per launch, right after their gamma^x is formed.
struct WorkRange {
  const WedgeDev *wedges;
  const void *alpha;
  const int4 *items;
  int n_items;
  const int2 *bins;
  int n_bins;
  const int2 *bins1;
  int n_bins1;
  bool clear;  // S3: zero the output before accumulating
};
WorkRange full_range(const fio_plan_s *p);
WorkRange group_range(const fio_plan_s *p, int g, bool clear);
cudaError_t launch_interp(const fio_plan_s *p, const void *grid, void *out, int B, cudaStream_t s,
                          const WorkRange &wr);
cudaError_t launch_spread(const fio_plan_s *p, const void *g, void *grid, int B, cudaStream_t s,
                          const WorkRange &wr);
// interp_tasks.cu: the mixed-precision S3 (zeroes out if wr.clear, then accumulates).
cudaError_t launch_interp_tasks(const fio_plan_s *p, const void *grid, void *out, int B,
                                cudaStream_t s, const WorkRange &wr);
// spread.cu: the mixed-precision S4a, all inputs of a launch in one sweep.
cudaError_t launch_spread_sweep(const fio_plan_s *p, const void *g, void *grid, int B,
                                cudaStream_t s, const WorkRange &wr);
// alpha_regen.cu (recompute mode): gamma^x of group g's wedges into p->d_alpha,
// in the layout of the stored mode with offsets from d_wedges_rc.
cudaError_t regen_alpha(const fio_plan_s *p, int g, cudaStream_t s);
// Per-x phase data of the complex64 regeneration from the plan's FP64 data:
// ellipse (c1^2, c2^2) as float2 [x]; tau modes C_m(x) as float2 [x][2 kMmax + 1].
cudaError_t rc_xdata_f32(const PhaseDev &ph, const void *d_xdata64, int N, void *d_out,
                         cudaStream_t s);
void release_timing_events(fio_plan_s *p);

// plan_kernels.cu (FP64 plan construction on the device)

cudaError_t plan_xdata(const PhaseDev &ph, const double *d_modes, int N, void *d_xdata,
                       cudaStream_t s);
size_t plan_xdata_bytes(const PhaseDev &ph, int N);
cudaError_t plan_warp(const PhaseDev &ph, const void *d_xdata, int N, int L, const WedgeDev *d_w,
                      uint2 *d_warp, cudaStream_t s);
// A_C[x][c] = a(x, xi_c) exp(2 pi i Phi_l(x, xi_c)) for the sampled columns of wedge l.
cudaError_t plan_eval_cols(const PhaseDev &ph, const void *d_xdata, int N, const WedgeDev &w,
                           const uint2 *d_warp_l, const int *d_ck1, const int *d_ck2, int r,
                           double2 *d_AC, cudaStream_t s);
// R of A = Q R (A: rows x r, row-major) by tall-skinny Householder QR: panels of
// tsqr_panel_rows(r) rows are factored in parallel, their R factors stacked and
// factored again until one remains; h_R (HOST, r x r row-major, zero below the
// diagonal) receives it after the stream synchronises.  d_work holds rows * r
// values, d_stk0 and d_stk1 tsqr_stack_elems(rows, r) each.
int tsqr_panel_rows(int r);
size_t tsqr_stack_elems(long long rows, int r);
cudaError_t plan_tsqr(const double2 *d_A, long long rows, int r, double2 *d_work, double2 *d_stk0,
                      double2 *d_stk1, double2 *h_R, cudaStream_t s);
// alpha[pos][t] = (sum_c A_C[x][c] W[c][t]) * exp(2 pi i y'.xi_c) / N with x = perm[pos]
// (W = V S^-1, r x q)
cudaError_t plan_form_alpha(const double2 *d_AC, int N, int r, int q, const double2 *d_W,
                            const WedgeDev &w, const uint2 *d_warp_l, const uint32_t *d_perm_l,
                            void *d_alpha_l, int precision, cudaStream_t s);
// beta[t][p] = (sum_i P[t][i] A(x_i, xi_p)) * dec[p], P = U_R^+ (q x r),
// dec[p] = 1 / (phihat(xi'_1/m1) phihat(xi'_2/m2)) (NUFFT deconvolution)
cudaError_t plan_form_beta(const PhaseDev &ph, const void *d_xdata, int N, const WedgeDev &w,
                           const uint2 *d_warp_l, const int *d_rx, int r, int q,
                           const double2 *d_P, const int *d_pk1, const int *d_pk2,
                           const double *d_dec, void *d_beta_l, int precision, cudaStream_t s);

// surrogate.cu: warped points from a trained surrogate, and its judged errors.
cudaError_t surrogate_warp(const fio_surrogate_s *s, int N, int L, const WedgeDev *d_w,
                           uint2 *d_warp);
const fio_surrogate_info *surrogate_info(const fio_surrogate_s *s);

// Per-column squared error of U T against A on s sampled rows (validation).
cudaError_t plan_validate(const PhaseDev &ph, const void *d_xdata, int N, const WedgeDev &w,
                          const uint2 *d_warp_l, const int *d_gx, int s, const double2 *d_UG,
                          const double2 *d_T, int q, const int *d_pk1, const int *d_pk2,
                          double *d_err, double *d_nrm, cudaStream_t st);


}  // namespace fio
