// plan_io.cpp -- the plan file of fio_plan_save / fio_plan_load: everything a
// plan's apply paths read (the preprocessing of Sec. 3.2 and its layout), so
// that a plan built once can be applied in another process without repeating
// the randomized separation.
//
// Layout (little-endian, as both supported hosts are): a header of 8 magic
// bytes "FIOPLAN1", a format version and a byte-order word, the scalar
// fields, then length-prefixed sections in a fixed order: the host tables
// (wedges, row runs, FFT plans, per-wedge sample counts and errors, the
// wedge frequencies, the KB polynomials) and the device arrays, copied as they
// are (twiddles, factors alpha' and beta', warped points in plan and sorted
// order, point order, bucket tables, work lists).  The NUFFT grid and spectrum
// workspace is not stored: load allocates it for the requested batch.  A plan
// in the recompute storage mode stores, in place of gamma^x, its phase
// parameters, the sampled columns, V S^-1 and the per-x phase data; its
// regeneration buffer is allocated on load.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fio_internal.h"

namespace fio {

namespace {

constexpr char kMagic[8] = {'F', 'I', 'O', 'P', 'L', 'A', 'N', '1'};
constexpr uint32_t kVersion = 2;
constexpr uint32_t kByteOrder = 0x01020304u;

// The scalar fields of a plan, as stored.
struct PlanScalars {
  int32_t N, L, precision, max_batch, kb_w, q_max, q_min, r_max, sur_warp, max_bin_pts,
      max_cand, n_items, n_bins, n_bins1, max_row_len, pad;
  double eps, sigma, kb_beta, sep_err, q_mean, plan_seconds, sur_warp_cycles,
      sur_residual_cycles, mean_bin_pts;
  int64_t grid_units, alpha_elems, beta_elems, cstart_elems, twiddle_elems, alg_bytes;
  int32_t alpha_mode, has_rc_g;
  int64_t rc_cols, rc_w_elems, rc_x_elems;
};

struct File {
  std::FILE *f = nullptr;
  ~File() {
    if (f) std::fclose(f);
  }
};

bool put(std::FILE *f, const void *p, size_t n) { return n == 0 || std::fwrite(p, 1, n, f) == n; }
bool get(std::FILE *f, void *p, size_t n) { return n == 0 || std::fread(p, 1, n, f) == n; }

template <typename T> bool put_vec(std::FILE *f, const std::vector<T> &v) {
  const uint64_t n = v.size();
  return put(f, &n, 8) && put(f, v.data(), n * sizeof(T));
}
template <typename T> bool get_vec(std::FILE *f, std::vector<T> &v, uint64_t max_n) {
  uint64_t n = 0;
  if (!get(f, &n, 8) || n > max_n) return false;
  v.resize(n);
  return get(f, v.data(), n * sizeof(T));
}

// A device array: its byte count, then its bytes (streamed through a host buffer).
bool put_dev(std::FILE *f, const void *d, uint64_t bytes) {
  if (!put(f, &bytes, 8)) return false;
  std::vector<unsigned char> buf(std::min<uint64_t>(bytes, 64ull << 20));
  for (uint64_t o = 0; o < bytes; o += buf.size()) {
    const size_t n = (size_t)std::min<uint64_t>(buf.size(), bytes - o);
    if (cudaMemcpy(buf.data(), (const char *)d + o, n, cudaMemcpyDeviceToHost) != cudaSuccess)
      return false;
    if (!put(f, buf.data(), n)) return false;
  }
  return true;
}
fio_status get_dev(std::FILE *f, void **d, uint64_t want) {
  uint64_t bytes = 0;
  if (!get(f, &bytes, 8) || bytes != want) {
    set_error("plan file: a device array has the wrong size");
    return FIO_EINVAL;
  }
  if (cudaMalloc(d, std::max<uint64_t>(bytes, 16)) != cudaSuccess) {
    *d = nullptr;
    set_error("plan file: device allocation failed");
    return FIO_ENOMEM;
  }
  std::vector<unsigned char> buf(std::min<uint64_t>(bytes, 64ull << 20));
  for (uint64_t o = 0; o < bytes; o += buf.size()) {
    const size_t n = (size_t)std::min<uint64_t>(buf.size(), bytes - o);
    if (!get(f, buf.data(), n)) {
      set_error("plan file: truncated");
      return FIO_EINVAL;
    }
    if (cudaMemcpy((char *)*d + o, buf.data(), n, cudaMemcpyHostToDevice) != cudaSuccess) {
      set_error("plan file: upload failed");
      return FIO_ECUDA;
    }
  }
  return FIO_OK;
}

}  // namespace

fio_status save_plan(const fio_plan_s *p, const char *path) {
  File fl;
  fl.f = std::fopen(path, "wb");
  if (!fl.f) {
    set_error(std::string("fio_plan_save: cannot open ") + path);
    return FIO_EINVAL;
  }
  const size_t cs = p->precision == FIO_FP64 ? 16 : 8;
  const uint64_t NN = (uint64_t)p->N * p->N, LNN = NN * p->L;
  PlanScalars sc{};
  sc.N = p->N; sc.L = p->L; sc.precision = p->precision; sc.max_batch = p->max_batch;
  sc.kb_w = p->kb.w; sc.q_max = p->q_max; sc.q_min = p->q_min; sc.r_max = p->r_max;
  sc.sur_warp = p->sur_warp; sc.max_bin_pts = p->max_bin_pts; sc.max_cand = p->max_cand;
  sc.n_items = p->n_items; sc.n_bins = p->n_bins; sc.n_bins1 = p->n_bins1;
  sc.max_row_len = p->max_row_len;
  sc.eps = p->eps; sc.sigma = p->sigma; sc.kb_beta = p->kb.beta; sc.sep_err = p->sep_err;
  sc.q_mean = p->q_mean; sc.plan_seconds = p->plan_seconds; sc.sur_warp_cycles = p->sur_warp_cycles;
  sc.sur_residual_cycles = p->sur_residual_cycles; sc.mean_bin_pts = p->mean_bin_pts;
  sc.grid_units = p->grid_units; sc.alpha_elems = p->alpha_elems; sc.beta_elems = p->beta_elems;
  sc.cstart_elems = p->cstart_elems; sc.twiddle_elems = p->twiddle_elems;
  sc.alg_bytes = (int64_t)p->alg_bytes;
  sc.alpha_mode = p->alpha_mode;
  sc.has_rc_g = p->d_rc_g != nullptr;
  sc.rc_cols = p->rc_cols; sc.rc_w_elems = p->rc_w_elems; sc.rc_x_elems = p->rc_x_elems;
  const bool rc = p->alpha_mode == FIO_ALPHA_RECOMPUTE;
  const bool ok =
      put(fl.f, kMagic, 8) && put(fl.f, &kVersion, 4) && put(fl.f, &kByteOrder, 4) &&
      put(fl.f, &sc, sizeof(sc)) && put_vec(fl.f, p->wedges) && put_vec(fl.f, p->rows) &&
      put_vec(fl.f, p->ffts) && put_vec(fl.f, p->wedge_r) && put_vec(fl.f, p->wedge_err) &&
      put_vec(fl.f, p->pt_k1) && put_vec(fl.f, p->pt_k2) && put(fl.f, &p->horner, sizeof(p->horner)) &&
      put_vec(fl.f, p->item_off) && put_vec(fl.f, p->bin_off) && put_vec(fl.f, p->bin1_off) &&
      put_vec(fl.f, p->grp_first) && put(fl.f, &p->phase, sizeof(p->phase)) &&
      put_dev(fl.f, p->d_twiddle, (uint64_t)p->twiddle_elems * cs) &&
      (rc || put_dev(fl.f, p->d_alpha, (uint64_t)p->alpha_elems * cs)) &&
      (!rc || (put_dev(fl.f, p->d_rc_col, (uint64_t)p->rc_cols * sizeof(RcCol)) &&
               put_dev(fl.f, p->d_rc_w, (uint64_t)p->rc_w_elems * cs) &&
               (!p->d_rc_g || put_dev(fl.f, p->d_rc_g, (uint64_t)p->rc_cols * (2 * kTauMmax + 1) * 8)) &&
               (!p->d_rc_x || put_dev(fl.f, p->d_rc_x, (uint64_t)p->rc_x_elems)))) &&
      put_dev(fl.f, p->d_beta, (uint64_t)p->beta_elems * cs) &&
      put_dev(fl.f, p->d_warp, LNN * sizeof(uint2)) && put_dev(fl.f, p->d_warps, LNN * sizeof(uint2)) &&
      put_dev(fl.f, p->d_perm, LNN * sizeof(uint32_t)) &&
      put_dev(fl.f, p->d_cstart, (uint64_t)p->cstart_elems * sizeof(int)) &&
      put_dev(fl.f, p->d_items, (uint64_t)p->n_items * sizeof(int4)) &&
      put_dev(fl.f, p->d_bins, (uint64_t)p->n_bins * sizeof(int2)) &&
      put_dev(fl.f, p->d_bins1, (uint64_t)p->n_bins1 * sizeof(int2));
  if (!ok || std::fflush(fl.f) != 0) {
    set_error(std::string("fio_plan_save: write to ") + path + " failed");
    return FIO_ECUDA;
  }
  return FIO_OK;
}

fio_status load_plan(fio_plan_s *p, const char *path, int max_batch) {
  File fl;
  fl.f = std::fopen(path, "rb");
  if (!fl.f) {
    set_error(std::string("fio_plan_load: cannot open ") + path);
    return FIO_EINVAL;
  }
  char magic[8];
  uint32_t ver = 0, bo = 0;
  PlanScalars sc{};
  if (!get(fl.f, magic, 8) || std::memcmp(magic, kMagic, 8) != 0 || !get(fl.f, &ver, 4) ||
      ver != kVersion || !get(fl.f, &bo, 4) || bo != kByteOrder || !get(fl.f, &sc, sizeof(sc))) {
    set_error(std::string("fio_plan_load: ") + path + " is not a plan file of this version");
    return FIO_EINVAL;
  }
  if (sc.N < 8 || sc.N > 2048 || sc.L < 1 || sc.L > 256 || (sc.precision != FIO_MIXED && sc.precision != FIO_FP64) ||
      sc.kb_w < 3 || sc.kb_w > kMaxKbWidth || sc.grid_units < 0 || sc.alpha_elems < 0 ||
      sc.beta_elems < 0 || sc.cstart_elems < 0 || sc.twiddle_elems < 0 || sc.n_items < 0 ||
      sc.n_bins < 0 || sc.n_bins1 < 0 ||
      (sc.alpha_mode != FIO_ALPHA_STORED && sc.alpha_mode != FIO_ALPHA_RECOMPUTE) ||
      sc.rc_cols < 0 || sc.rc_w_elems < 0 || sc.rc_x_elems < 0) {
    set_error("fio_plan_load: corrupt plan header");
    return FIO_EINVAL;
  }
  const uint64_t NN = (uint64_t)sc.N * sc.N, LNN = NN * sc.L;
  const bool tables = get_vec(fl.f, p->wedges, (uint64_t)sc.L) && p->wedges.size() == (size_t)sc.L &&
                      get_vec(fl.f, p->rows, 1ull << 24) && get_vec(fl.f, p->ffts, 1ull << 16) &&
                      get_vec(fl.f, p->wedge_r, (uint64_t)sc.L) && get_vec(fl.f, p->wedge_err, (uint64_t)sc.L) &&
                      get_vec(fl.f, p->pt_k1, NN) && get_vec(fl.f, p->pt_k2, NN) &&
                      get(fl.f, &p->horner, sizeof(p->horner)) &&
                      get_vec(fl.f, p->item_off, (uint64_t)sc.L + 1) &&
                      get_vec(fl.f, p->bin_off, (uint64_t)sc.L + 1) &&
                      get_vec(fl.f, p->bin1_off, (uint64_t)sc.L + 1) &&
                      get_vec(fl.f, p->grp_first, (uint64_t)sc.L + 1) &&
                      get(fl.f, &p->phase, sizeof(p->phase));
  bool offsets = tables && p->item_off.size() == (size_t)sc.L + 1 &&
                 p->bin_off.size() == (size_t)sc.L + 1 && p->bin1_off.size() == (size_t)sc.L + 1 &&
                 p->item_off.back() == sc.n_items && p->bin_off.back() == sc.n_bins &&
                 p->bin1_off.back() == sc.n_bins1;
  for (int l = 0; offsets && l < sc.L; ++l)
    offsets = p->item_off[l] <= p->item_off[l + 1] && p->bin_off[l] <= p->bin_off[l + 1] &&
              p->bin1_off[l] <= p->bin1_off[l + 1] && p->item_off[l] >= 0 && p->bin_off[l] >= 0 &&
              p->bin1_off[l] >= 0;
  if (sc.alpha_mode == FIO_ALPHA_RECOMPUTE) {
    offsets = offsets && p->grp_first.size() >= 2 && p->grp_first.front() == 0 &&
              p->grp_first.back() == sc.L;
    for (size_t g = 0; offsets && g + 1 < p->grp_first.size(); ++g)
      offsets = p->grp_first[g] < p->grp_first[g + 1];
    // every wedge's columns and V S^-1 lie inside the stored arrays
    for (int l = 0; offsets && l < sc.L; ++l) {
      const WedgeDev &w = p->wedges[l];
      offsets = w.rc_r >= 0 && w.qp >= 0 && w.rc_col_off >= 0 && w.rc_w_off >= 0 &&
                w.rc_col_off + w.rc_r <= sc.rc_cols &&
                w.rc_w_off + (int64_t)w.rc_r * w.qp <= sc.rc_w_elems;
    }
    // the phase and the per-x data the regeneration reads agree with each other:
    // complex64 plans keep float2 per x (ellipse) or per (x, m) (tau modes) and
    // the tau column factors; FP64 plans keep the plan's own FP64 phase data
    const PhaseDev &ph = p->phase;
    const bool kind_ok = ph.kind == FIO_PHASE_SHIFT_WAVE || ph.kind == FIO_PHASE_ELLIPSE ||
                         ph.kind == FIO_PHASE_TAU_MODES;
    const bool amp_ok = ph.amp_kind == FIO_AMP_ONE || ph.amp_kind == FIO_AMP_SEPARABLE ||
                        (ph.amp_kind == FIO_AMP_HANKEL && sc.precision == FIO_FP64);
    const int64_t per_x = ph.kind == FIO_PHASE_ELLIPSE ? 1
                          : ph.kind == FIO_PHASE_TAU_MODES ? 2 * kTauMmax + 1 : 0;
    const int64_t want_x = sc.precision == FIO_FP64 ? (per_x ? (int64_t)NN * per_x * 16 : 16)
                                                    : (int64_t)NN * per_x * 8;
    const bool want_g = sc.precision == FIO_MIXED && ph.kind == FIO_PHASE_TAU_MODES;
    offsets = offsets && kind_ok && amp_ok && sc.rc_x_elems == want_x &&
              (sc.has_rc_g != 0) == want_g;
  }
  if (!tables || !offsets) {
    set_error("fio_plan_load: corrupt or truncated host tables");
    return FIO_EINVAL;
  }
  p->N = sc.N; p->L = sc.L; p->precision = sc.precision;
  p->max_batch = max_batch > 0 ? max_batch : sc.max_batch;
  p->eps = sc.eps; p->sigma = sc.sigma; p->kb.w = sc.kb_w; p->kb.beta = sc.kb_beta;
  p->q_max = sc.q_max; p->q_min = sc.q_min; p->r_max = sc.r_max; p->sep_err = sc.sep_err;
  p->q_mean = sc.q_mean; p->plan_seconds = sc.plan_seconds; p->sur_warp = sc.sur_warp;
  p->sur_warp_cycles = sc.sur_warp_cycles; p->sur_residual_cycles = sc.sur_residual_cycles;
  p->max_bin_pts = sc.max_bin_pts; p->mean_bin_pts = sc.mean_bin_pts; p->max_cand = sc.max_cand;
  p->n_items = sc.n_items; p->n_bins = sc.n_bins; p->n_bins1 = sc.n_bins1;
  p->max_row_len = sc.max_row_len;
  p->grid_units = sc.grid_units; p->alpha_elems = sc.alpha_elems; p->beta_elems = sc.beta_elems;
  p->cstart_elems = sc.cstart_elems; p->twiddle_elems = sc.twiddle_elems;
  p->alg_bytes = (unsigned long long)sc.alg_bytes;
  p->alpha_mode = sc.alpha_mode;
  p->rc_cols = sc.rc_cols; p->rc_w_elems = sc.rc_w_elems; p->rc_x_elems = sc.rc_x_elems;
  const bool rc = p->alpha_mode == FIO_ALPHA_RECOMPUTE;
  cudaGetDevice(&p->device);
  const size_t cs = p->precision == FIO_FP64 ? 16 : 8;
  fio_status s;
  if ((s = get_dev(fl.f, &p->d_twiddle, (uint64_t)p->twiddle_elems * cs)) != FIO_OK) return s;
  if (rc) {  // the regeneration buffer: allocated, not stored
    if (cudaMalloc(&p->d_alpha, std::max<size_t>((size_t)p->alpha_elems * cs, 16)) != cudaSuccess) {
      p->d_alpha = nullptr;
      set_error("fio_plan_load: device allocation failed");
      return FIO_ENOMEM;
    }
    if ((s = get_dev(fl.f, (void **)&p->d_rc_col, (uint64_t)p->rc_cols * sizeof(RcCol))) != FIO_OK) return s;
    if ((s = get_dev(fl.f, &p->d_rc_w, (uint64_t)p->rc_w_elems * cs)) != FIO_OK) return s;
    if (sc.has_rc_g &&
        (s = get_dev(fl.f, &p->d_rc_g, (uint64_t)p->rc_cols * (2 * kTauMmax + 1) * 8)) != FIO_OK)
      return s;
    if (p->rc_x_elems > 0 && (s = get_dev(fl.f, &p->d_rc_x, (uint64_t)p->rc_x_elems)) != FIO_OK) return s;
  } else if ((s = get_dev(fl.f, &p->d_alpha, (uint64_t)p->alpha_elems * cs)) != FIO_OK) {
    return s;
  }
  if ((s = get_dev(fl.f, &p->d_beta, (uint64_t)p->beta_elems * cs)) != FIO_OK) return s;
  if ((s = get_dev(fl.f, (void **)&p->d_warp, LNN * sizeof(uint2))) != FIO_OK) return s;
  if ((s = get_dev(fl.f, (void **)&p->d_warps, LNN * sizeof(uint2))) != FIO_OK) return s;
  if ((s = get_dev(fl.f, (void **)&p->d_perm, LNN * sizeof(uint32_t))) != FIO_OK) return s;
  if ((s = get_dev(fl.f, (void **)&p->d_cstart, (uint64_t)p->cstart_elems * sizeof(int))) != FIO_OK) return s;
  if ((s = get_dev(fl.f, (void **)&p->d_items, (uint64_t)p->n_items * sizeof(int4))) != FIO_OK) return s;
  if ((s = get_dev(fl.f, (void **)&p->d_bins, (uint64_t)p->n_bins * sizeof(int2))) != FIO_OK) return s;
  if ((s = get_dev(fl.f, (void **)&p->d_bins1, (uint64_t)p->n_bins1 * sizeof(int2))) != FIO_OK) return s;
  // the small device tables come from the host copies; the workspace is new
  auto upload = [&](void **d, const void *h, size_t bytes) -> fio_status {
    if (cudaMalloc(d, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      *d = nullptr;
      set_error("fio_plan_load: device allocation failed");
      return FIO_ENOMEM;
    }
    if (bytes && cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
      set_error("fio_plan_load: upload failed");
      return FIO_ECUDA;
    }
    return FIO_OK;
  };
  if ((s = upload((void **)&p->d_wedges, p->wedges.data(), p->wedges.size() * sizeof(WedgeDev))) != FIO_OK) return s;
  if (rc) {
    long long abuf = 0;
    const std::vector<WedgeDev> wrc = rc_wedge_table(p->wedges, p->grp_first, (long long)NN, &abuf);
    if (abuf != p->alpha_elems) {
      set_error("fio_plan_load: corrupt plan header");
      return FIO_EINVAL;
    }
    if ((s = upload((void **)&p->d_wedges_rc, wrc.data(), wrc.size() * sizeof(WedgeDev))) != FIO_OK) return s;
  }
  if ((s = upload((void **)&p->d_rows, p->rows.data(), p->rows.size() * sizeof(RowDev))) != FIO_OK) return s;
  if ((s = upload((void **)&p->d_ffts, p->ffts.data(), p->ffts.size() * sizeof(FftPlanDev))) != FIO_OK) return s;
  const int zero = 0;
  if ((s = upload((void **)&p->d_errword, &zero, sizeof(int))) != FIO_OK) return s;
  const size_t gbytes = (size_t)p->grid_units * p->max_batch * cs, fbytes = (size_t)NN * p->max_batch * cs;
  if (cudaMalloc(&p->d_grid, std::max<size_t>(gbytes, 16)) != cudaSuccess ||
      cudaMalloc(&p->d_fhat, std::max<size_t>(fbytes, 16)) != cudaSuccess) {
    set_error("fio_plan_load: workspace allocation failed");
    return FIO_ENOMEM;
  }
  p->bytes_total = (size_t)(p->twiddle_elems + p->alpha_elems + p->beta_elems) * cs +
                   LNN * (2 * sizeof(uint2) + sizeof(uint32_t)) + p->cstart_elems * sizeof(int) +
                   p->n_items * sizeof(int4) + (p->n_bins + p->n_bins1) * sizeof(int2) +
                   p->wedges.size() * sizeof(WedgeDev) + p->rows.size() * sizeof(RowDev) +
                   p->ffts.size() * sizeof(FftPlanDev) + gbytes + fbytes + rc_bytes(p);
  return FIO_OK;
}

}  // namespace fio
