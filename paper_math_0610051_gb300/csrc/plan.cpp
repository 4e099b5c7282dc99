// plan.cpp -- host side of fio_plan_create: polar wedges (Sec. 1.3), the
// shear/translate boxes and NUFFT grids (Sec. 3.4), the Kaiser-Bessel kernel,
// and the randomized separation of Sec. 3.2 (sample columns, SVD of A_[C]
// through its QR factorization, threshold eps, double r until q <= r/3, sample
// rows, T = U_[R]^+ A_[R]).  Large FP64 work (A_[C], its tall-skinny QR, the
// factors) runs in plan_kernels.cu; the SVDs of the r x r triangular factor and
// of U_[R] run here by one-sided Jacobi.
#include <cuda_runtime.h>

#include <algorithm>
#include <limits>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <set>
#include <string>
#include <unordered_set>
#include <vector>

#include "fio_internal.h"
#include "plan_host.h"

namespace fio {

using cd = std::complex<double>;

// Separation rule (Sec. 3.2 with a stricter acceptance test): singular values
// of A_[C] above sep_cut * eps * s_1 are kept; a sample is accepted when
// q <= r/3 and the relative Frobenius error of U T, measured on
// kValidationRows fresh random rows against every column of the wedge, is at
// most sep_target * eps.  Otherwise the worst-fitted columns join the next
// sample and r doubles.  The defaults below apply when fio_options leaves
// them 0.
constexpr double kSvdFraction = 0.25;
constexpr double kValidationTarget = 0.5;
constexpr int kValidationRows = 200;

// ------------------------------------------------------------- FFT sizes --

std::vector<int> fft_factor(int n) {
  std::vector<int> r;
  if (n < 2) return r;
  while (n % 16 == 0) { r.push_back(16); n /= 16; }
  while (n % 8 == 0) { r.push_back(8); n /= 8; }
  while (n % 4 == 0) { r.push_back(4); n /= 4; }
  while (n % 2 == 0) { r.push_back(2); n /= 2; }
  while (n % 9 == 0) { r.push_back(9); n /= 9; }
  while (n % 3 == 0) { r.push_back(3); n /= 3; }
  while (n % 5 == 0) { r.push_back(5); n /= 5; }
  if (n != 1) r.clear();
  return r;
}

int fft_good_size(int n) {
  for (int m = std::max(n, 2);; ++m)
    if (m % 2 == 0 && !fft_factor(m).empty()) return m;
}

// ---------------------------------------------------------- KB kernel ------

int kb_width_for(double eps) {
  // 1D relative NUFFT error of the sigma = 2 KB kernel is about 4.5 * 10^-w
  // (measured against direct sums); ask for eps / 10.
  int w = (int)std::ceil(std::log10(45.0 / eps));
  return std::min(std::max(w, 3), kMaxKbWidth);
}

double kb_beta_for(int w, double sigma) {
  // Beatty, Nishimura, Pauly (2005): beta = pi sqrt((w/sigma)^2 (sigma - 1/2)^2 - 0.8)
  const double a = (w / sigma) * (w / sigma) * (sigma - 0.5) * (sigma - 0.5) - 0.8;
  return M_PI * std::sqrt(std::max(a, 0.1));
}

double kb_phi_host(double s, int w, double beta) {
  const double z = 2.0 * s / w, a = 1.0 - z * z;
  return a > 0 ? std::cyl_bessel_i(0.0, beta * std::sqrt(a)) / std::cyl_bessel_i(0.0, beta) : 0.0;
}

// phihat(nu) = int phi(s) exp(-2 pi i nu s) ds = w sinh(sqrt(b^2 - a^2)) / sqrt(b^2 - a^2) / I0(b),
// a = pi w nu (the sin form when a > b).
double kb_phihat_host(double nu, int w, double beta) {
  const double a = M_PI * w * nu;
  const double d = beta * beta - a * a;
  double v;
  if (d > 1e-12) v = w * std::sinh(std::sqrt(d)) / std::sqrt(d);
  else if (d < -1e-12) v = w * std::sin(std::sqrt(-d)) / std::sqrt(-d);
  else v = w;
  return v / std::cyl_bessel_i(0.0, beta);
}

// -------------------------------------------------------------- wedges -----

int default_L(int N) {
  int L = (int)std::ceil(std::sqrt((double)N) - 1e-12);
  L = (L + 7) / 8 * 8;
  return std::max(L, 8);
}

// W_l = {(2l - 1) pi / L <= arg xi < (2l + 1) pi / L}; xi = 0 belongs to wedge 0.
int wedge_of(int k1, int k2, int L) {
  if (k1 == 0 && k2 == 0) return 0;
  const double th = std::atan2((double)k2, (double)k1);
  int l = (int)std::floor((th + M_PI / L) / (2.0 * M_PI / L));
  l %= L;
  if (l < 0) l += L;
  return l;
}

static const int kShears[5][4] = {
    {1, 0, 0, 1}, {1, 0, -1, 1}, {1, 0, 1, 1}, {1, -1, 0, 1}, {1, 1, 0, 1}};
static const int kShearInv[5][4] = {
    {1, 0, 0, 1}, {1, 0, 1, 1}, {1, 0, -1, 1}, {1, 1, 0, 1}, {1, -1, 0, 1}};

static int grid_len(int n, double sigma, int w) {
  const int want = std::max({(int)std::ceil(sigma * n - 1e-9), n + 2, 2 * w, 16});
  return fft_good_size(want);
}

// Box, grid and row runs for one wedge, choosing among identity and the four
// 45-degree shears the one with the smallest oversampled grid (Sec. 3.4).
bool wedge_geometry(const std::vector<std::pair<int, int>> &pts, double sigma, int w,
                    WedgeDev &wd, std::vector<RowDev> &rows, std::vector<int> &k1s,
                    std::vector<int> &k2s, std::vector<int> &x1p, std::vector<int> &x2p,
                    std::string &err) {
  long long best = -1;
  int bi = 0;
  for (int s = 0; s < 5; ++s) {
    const int *M = kShears[s];
    int lo1 = 1 << 30, hi1 = -(1 << 30), lo2 = 1 << 30, hi2 = -(1 << 30);
    for (auto &p : pts) {
      const int a = M[0] * p.first + M[1] * p.second, b = M[2] * p.first + M[3] * p.second;
      lo1 = std::min(lo1, a); hi1 = std::max(hi1, a);
      lo2 = std::min(lo2, b); hi2 = std::max(hi2, b);
    }
    const long long cost = (long long)grid_len(hi1 - lo1 + 1, sigma, w) *
                           grid_len(hi2 - lo2 + 1, sigma, w);
    if (best < 0 || cost < best) { best = cost; bi = s; }
  }
  std::memset(&wd, 0, sizeof(wd));
  std::memcpy(wd.M, kShears[bi], sizeof(wd.M));
  std::memcpy(wd.Minv, kShearInv[bi], sizeof(wd.Minv));
  const int *M = wd.M;
  std::vector<std::pair<int, int>> pp;  // (xi''_1, xi''_2)
  pp.reserve(pts.size());
  int lo1 = 1 << 30, hi1 = -(1 << 30), lo2 = 1 << 30, hi2 = -(1 << 30);
  for (auto &p : pts) {
    const int a = M[0] * p.first + M[1] * p.second, b = M[2] * p.first + M[3] * p.second;
    pp.push_back({a, b});
    lo1 = std::min(lo1, a); hi1 = std::max(hi1, a);
    lo2 = std::min(lo2, b); hi2 = std::max(hi2, b);
  }
  const int n1 = hi1 - lo1 + 1, n2 = hi2 - lo2 + 1;
  wd.xc1 = lo1 + n1 / 2;
  wd.xc2 = lo2 + n2 / 2;
  wd.b1 = lo1 - wd.xc1;
  wd.n1 = n1;
  wd.b2 = lo2 - wd.xc2;
  wd.n2 = n2;
  wd.m1 = grid_len(n1, sigma, w);
  wd.m2 = grid_len(n2, sigma, w);
  wd.npts = (int)pts.size();
  std::sort(pp.begin(), pp.end());
  rows.clear();
  k1s.clear(); k2s.clear(); x1p.clear(); x2p.clear();
  size_t i = 0;
  for (int a = lo1; a <= hi1; ++a) {
    RowDev rw{};
    rw.xi1 = a - wd.xc1;
    rw.pt = (int)k1s.size();
    rw.len = 0;
    rw.a = 0;
    int prev = 0;
    while (i < pp.size() && pp[i].first == a) {
      const int b = pp[i].second;
      if (rw.len == 0) rw.a = b - wd.xc2;
      else if (b != prev + 1) {
        err = "wedge row is not a contiguous run";
        return false;
      }
      prev = b;
      const int kk1 = wd.Minv[0] * a + wd.Minv[1] * b, kk2 = wd.Minv[2] * a + wd.Minv[3] * b;
      k1s.push_back(kk1);
      k2s.push_back(kk2);
      x1p.push_back(a - wd.xc1);
      x2p.push_back(b - wd.xc2);
      ++rw.len;
      ++i;
    }
    rows.push_back(rw);
  }
  return true;
}

// -------------------------------------------------------------- sampling ---

struct SplitMix64 {  // Steele, Lea and Flood (2014)
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  }
  uint64_t below(uint64_t n) { return (uint64_t)(((unsigned __int128)next() * n) >> 64); }
};

// k distinct integers of [0, n), uniformly (Floyd's algorithm), sorted.
static std::vector<int> sample_distinct(int n, int k, SplitMix64 &rng) {
  std::unordered_set<int> S;
  S.reserve(2 * k);
  for (int j = n - k; j < n; ++j) {
    const int t = (int)rng.below((uint64_t)j + 1);
    if (!S.insert(t).second) S.insert(j);
  }
  std::vector<int> v(S.begin(), S.end());
  std::sort(v.begin(), v.end());
  return v;
}

static uint64_t mix_seed(uint64_t seed, uint64_t a, uint64_t b) {
  SplitMix64 m{seed ^ (a * 0xD1B54A32D192ED03ULL) ^ (b * 0x8CB92BA72F3D8DD7ULL)};
  return m.next();
}

// ---------------------------------------------------------- eigensolver ----

// Eigen-decomposition of a Hermitian n x n matrix A (row-major): eigenvalues in
// descending order, eigenvectors as the columns of V (row-major).
//  1. Householder reduction A = Q T Q^H, T Hermitian tridiagonal: reflector k
//     H = I - u u^H maps column k below the diagonal onto alpha e1, with
//     alpha = -phase(x0) |x| (no cancellation in x0 - alpha).
//  2. T' = D^H T D with a unitary diagonal D makes the off-diagonal real and
//     non-negative: T' is real symmetric tridiagonal.
//  3. T' = W diag(lambda) W^T by implicit symmetric QR steps with Wilkinson
//     shifts (Golub and Van Loan, Algorithm 8.3.2): a Givens rotation chases the
//     bulge down the unreduced block; converged off-diagonals are deflated.
//  4. The eigenvectors of A are the columns of Q D W.
void herm_eig(int n, std::vector<cd> A, std::vector<double> &ev, std::vector<cd> &V) {
  auto at = [&](int i, int j) -> cd & { return A[(size_t)i * n + j]; };
  std::vector<cd> U((size_t)n * n, cd(0));  // reflector k in row k, entries k+1 .. n-1
  std::vector<char> has(n, 0);
  std::vector<cd> pv(n), wv(n);
  for (int k = 0; k + 2 < n; ++k) {
    double sig2 = 0;
    for (int i = k + 1; i < n; ++i) sig2 += std::norm(at(i, k));
    const double sigma = std::sqrt(sig2);
    if (sigma == 0.0) continue;
    const cd x0 = at(k + 1, k);
    const double ax0 = std::abs(x0);
    const cd phase = ax0 > 0 ? x0 / ax0 : cd(1.0);
    const cd alpha = -phase * sigma;
    // u = v sqrt(2 / v^H v), v = x - alpha e1, v^H v = 2 sigma (sigma + |x0|)
    const double scale = 1.0 / std::sqrt(sigma * (sigma + ax0));
    cd *u = &U[(size_t)k * n];
    u[k + 1] = (x0 - alpha) * scale;
    for (int i = k + 2; i < n; ++i) u[i] = at(i, k) * scale;
    has[k] = 1;
    // B = A[k+1.., k+1..] <- H B H = B - u w^H - w u^H, p = B u, w = p - (u^H p / 2) u
    double K = 0;
    for (int i = k + 1; i < n; ++i) {
      cd acc = 0;
      const cd *row = &A[(size_t)i * n];
      for (int j = k + 1; j < n; ++j) acc += row[j] * u[j];
      pv[i] = acc;
      K += (std::conj(u[i]) * acc).real();
    }
    for (int i = k + 1; i < n; ++i) wv[i] = pv[i] - 0.5 * K * u[i];
    for (int i = k + 1; i < n; ++i) {
      cd *row = &A[(size_t)i * n];
      const cd ui = u[i], wi = wv[i];
      for (int j = k + 1; j < n; ++j) row[j] -= ui * std::conj(wv[j]) + wi * std::conj(u[j]);
    }
    at(k + 1, k) = alpha;
    at(k, k + 1) = std::conj(alpha);
    for (int i = k + 2; i < n; ++i) at(i, k) = at(k, i) = 0;
  }
  // Q = H_0 H_1 ... H_{n-3}, accumulated from the last reflector
  std::vector<cd> Q((size_t)n * n, cd(0));
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  std::vector<cd> yv(n);
  for (int k = n - 3; k >= 0; --k) {
    if (!has[k]) continue;
    const cd *u = &U[(size_t)k * n];
    std::fill(yv.begin(), yv.end(), cd(0));
    for (int i = k + 1; i < n; ++i) {
      const cd cu = std::conj(u[i]);
      const cd *row = &Q[(size_t)i * n];
      for (int j = k + 1; j < n; ++j) yv[j] += cu * row[j];
    }
    for (int i = k + 1; i < n; ++i) {
      cd *row = &Q[(size_t)i * n];
      const cd ui = u[i];
      for (int j = k + 1; j < n; ++j) row[j] -= ui * yv[j];
    }
  }
  // real symmetric tridiagonal d, e (e[k] couples k and k+1) and the phases D
  std::vector<double> d(n), e(std::max(n - 1, 0));
  std::vector<cd> D(n, cd(1.0));
  for (int k = 0; k < n; ++k) d[k] = at(k, k).real();
  for (int k = 0; k + 1 < n; ++k) {
    const cd b = at(k + 1, k);
    const double ab = std::abs(b);
    e[k] = ab;
    D[k + 1] = ab > 0 ? D[k] * (b / ab) : D[k];
  }
  // implicit symmetric QR on d, e; W accumulates the rotations (real, row-major)
  std::vector<double> W((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) W[(size_t)i * n + i] = 1.0;
  const double tol = 4.0 * std::numeric_limits<double>::epsilon();
  int hi = n - 1;
  long long steps = 0;
  while (hi > 0 && steps < 60LL * n) {
    if (std::abs(e[hi - 1]) <= tol * (std::abs(d[hi - 1]) + std::abs(d[hi]))) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && std::abs(e[lo - 1]) > tol * (std::abs(d[lo - 1]) + std::abs(d[lo]))) --lo;
    ++steps;
    // Wilkinson shift from the trailing 2 x 2 of the block
    const double t = 0.5 * (d[hi - 1] - d[hi]), b2 = e[hi - 1] * e[hi - 1];
    const double mu = d[hi] - b2 / (t + (t >= 0 ? 1.0 : -1.0) * std::sqrt(t * t + b2));
    double x = d[lo] - mu, z = e[lo];
    for (int k = lo; k < hi; ++k) {
      // P = [[c, s], [-s, c]] on (k, k+1): P^T [x; z] = [r; 0]
      const double r = std::hypot(x, z);
      const double c = r > 0 ? x / r : 1.0, s = r > 0 ? -z / r : 0.0;
      if (k > lo) e[k - 1] = r;  // the bulge at (k+1, k-1) is gone
      const double a = d[k], bb = e[k], cc = d[k + 1];
      d[k] = a * c * c - 2.0 * bb * c * s + cc * s * s;
      d[k + 1] = a * s * s + 2.0 * bb * c * s + cc * c * c;
      e[k] = (a - cc) * c * s + bb * (c * c - s * s);
      if (k + 1 < hi) {
        const double f = e[k + 1];
        z = -s * f;  // new bulge at (k+2, k)
        e[k + 1] = c * f;
        x = e[k];
      }
      for (int i = 0; i < n; ++i) {
        double *wr = &W[(size_t)i * n];
        const double wk = wr[k], wk1 = wr[k + 1];
        wr[k] = c * wk - s * wk1;
        wr[k + 1] = s * wk + c * wk1;
      }
    }
  }
  // V = Q D W, columns sorted by descending eigenvalue
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return d[a] > d[b]; });
  std::vector<cd> QD((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) QD[(size_t)i * n + k] = Q[(size_t)i * n + k] * D[k];
  std::vector<double> Ws((size_t)n * n);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j) Ws[(size_t)k * n + j] = W[(size_t)k * n + idx[j]];
  V.assign((size_t)n * n, cd(0));
  for (int i = 0; i < n; ++i) {
    cd *vr = &V[(size_t)i * n];
    for (int k = 0; k < n; ++k) {
      const cd q = QD[(size_t)i * n + k];
      const double *wr = &Ws[(size_t)k * n];
      for (int j = 0; j < n; ++j) vr[j] += q * wr[j];
    }
  }
  ev.resize(n);
  for (int j = 0; j < n; ++j) ev[j] = d[idx[j]];
}

// Singular value decomposition of an m x n complex matrix A (row-major) by
// one-sided Jacobi rotations (Hestenes): unitary plane rotations J applied on
// the right until every pair of columns of A V is orthogonal to working
// precision.  Then A V = U diag(sig): the column norms are the singular
// values, and V (n x n, row-major) collects the rotations.  A^H A is never
// formed, so small singular values keep their absolute accuracy eps ||A||
// (Demmel and Veselic, 1992).  On return A holds A V with its columns in the
// order of sig, which is descending.
//
// A pair (p, q) with gamma = a_p^H a_q = |gamma| e^{i phi} is rotated by
//   a_p <- c a_p - s e^{-i phi} a_q,   a_q <- s a_p + c e^{-i phi} a_q,
// t = s / c the smaller root of t^2 + 2 zeta t - 1 = 0,
// zeta = (|a_q|^2 - |a_p|^2) / (2 |gamma|), which makes the new pair orthogonal.
void svd_jacobi(int m, int n, std::vector<cd> &A, std::vector<double> &sig, std::vector<cd> &V) {
  std::vector<cd> Ac((size_t)m * n), Vc((size_t)n * n, cd(0));  // column-major work copies
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) Ac[(size_t)j * m + i] = A[(size_t)i * n + j];
  for (int j = 0; j < n; ++j) Vc[(size_t)j * n + j] = 1.0;
  const double tol = std::max(1e-15, std::sqrt((double)m) * std::numeric_limits<double>::epsilon());
  // squared column norms, refreshed by every rotation that changes a column
  std::vector<double> nrm2(n, 0.0);
  double fro2 = 0;
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < m; ++i) nrm2[j] += std::norm(Ac[(size_t)j * m + i]);
    fro2 += nrm2[j];
  }
  // columns below 1e-18 ||A||_F are numerically zero: rotating them changes A by
  // less than its rounding, and their tiny (even denormal) inner products would
  // give inexact rotation phases
  const double tiny2 = 1e-36 * fro2;
  // round-robin ordering: each round pairs every column once, the pairs of a
  // round are disjoint and are rotated in parallel
  const int nn = n + (n & 1);
  std::vector<int> perm(nn);
  std::iota(perm.begin(), perm.end(), 0);
  const bool par = (long long)m * n >= 4096;
  for (int sweep = 0; sweep < 60; ++sweep) {
    long long rotated = 0;
    for (int round = 0; round + 1 < nn; ++round) {
#pragma omp parallel for reduction(+ : rotated) schedule(static) if (par)
      for (int k = 0; k < nn / 2; ++k) {
        int p = perm[k], q = perm[nn - 1 - k];
        if (p >= n || q >= n) continue;
        if (p > q) std::swap(p, q);
        cd *ap = &Ac[(size_t)p * m], *aq = &Ac[(size_t)q * m];
        const double al = nrm2[p], be = nrm2[q];
        if (al <= tiny2 || be <= tiny2) continue;
        cd ga = 0;
        for (int i = 0; i < m; ++i) ga += std::conj(ap[i]) * aq[i];
        const double ag = std::abs(ga);
        if (ag <= tol * std::sqrt(al) * std::sqrt(be)) continue;
        ++rotated;
        const cd eph = std::conj(ga / ag);  // e^{-i phi}
        const double zeta = (be - al) / (2.0 * ag);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::abs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
        double np = 0, nq = 0;
        for (int i = 0; i < m; ++i) {
          const cd x = ap[i], y = eph * aq[i];
          ap[i] = c * x - sn * y;
          aq[i] = sn * x + c * y;
          np += std::norm(ap[i]);
          nq += std::norm(aq[i]);
        }
        nrm2[p] = np;
        nrm2[q] = nq;
        cd *vp = &Vc[(size_t)p * n], *vq = &Vc[(size_t)q * n];
        for (int i = 0; i < n; ++i) {
          const cd x = vp[i], y = eph * vq[i];
          vp[i] = c * x - sn * y;
          vq[i] = sn * x + c * y;
        }
      }
      const int last = perm[nn - 1];  // keep perm[0], rotate the others one place
      for (int i = nn - 1; i > 1; --i) perm[i] = perm[i - 1];
      if (nn > 1) perm[1] = last;
    }
    if (!rotated) break;
  }
  std::vector<double> nrm(n);
  for (int j = 0; j < n; ++j) {
    double acc = 0;
    for (int i = 0; i < m; ++i) acc += std::norm(Ac[(size_t)j * m + i]);
    nrm[j] = std::sqrt(acc);
  }
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return nrm[a] > nrm[b]; });
  sig.resize(n);
  V.assign((size_t)n * n, cd(0));
  for (int k = 0; k < n; ++k) {
    const int j = idx[k];
    sig[k] = nrm[j];
    for (int i = 0; i < m; ++i) A[(size_t)i * n + k] = Ac[(size_t)j * m + i];
    for (int i = 0; i < n; ++i) V[(size_t)i * n + k] = Vc[(size_t)j * n + i];
  }
}

// Right singular vectors and singular values of a square matrix R (n x n,
// row-major), for the triangular factor of A_[C].  One-sided Jacobi converges
// in a few sweeps when it is applied to the conjugate transpose of the
// triangular factor of a column-pivoted QR (Drmac and Veselic, 2008):
//   R P = Q1 R1 (Householder with column pivoting),  X = R1^H,
//   X V_X = U_X S (svd_jacobi),  so R = (Q1 V_X) S (P U_X)^H
// and the right singular vectors of R are V = P U_X, U_X = X V_X S^-1.  V's
// columns follow sig (descending); a column with sig = 0 is left zero.
void svd_right_pivoted(int n, const std::vector<cd> &R, std::vector<double> &sig,
                       std::vector<cd> &V) {
  std::vector<cd> A(R);
  std::vector<int> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::vector<double> nrm(n, 0.0);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) nrm[j] += std::norm(A[(size_t)i * n + j]);
  std::vector<cd> u(n), w(n);
  for (int k = 0; k < n; ++k) {
    int piv = k;  // the column of largest remaining norm (rows k .. n-1)
    for (int j = k + 1; j < n; ++j)
      if (nrm[j] > nrm[piv]) piv = j;
    if (piv != k) {
      for (int i = 0; i < n; ++i) std::swap(A[(size_t)i * n + k], A[(size_t)i * n + piv]);
      std::swap(nrm[k], nrm[piv]);
      std::swap(perm[k], perm[piv]);
    }
    double sig2 = 0;
    for (int i = k; i < n; ++i) sig2 += std::norm(A[(size_t)i * n + k]);
    const double sigma = std::sqrt(sig2);
    if (sigma > 0) {
      // reflector H = I - u u^H (u^H u = 2) maps column k onto alpha e_k
      const cd x0 = A[(size_t)k * n + k];
      const double ax0 = std::abs(x0);
      const cd alpha = -(ax0 > 0 ? x0 / ax0 : cd(1.0)) * sigma;
      const double sc = 1.0 / std::sqrt(sigma * (sigma + ax0));
      u[k] = (x0 - alpha) * sc;
      for (int i = k + 1; i < n; ++i) u[i] = A[(size_t)i * n + k] * sc;
#pragma omp parallel for schedule(static) if (n >= 128)
      for (int j = k + 1; j < n; ++j) {
        cd d = 0;
        for (int i = k; i < n; ++i) d += std::conj(u[i]) * A[(size_t)i * n + j];
        for (int i = k; i < n; ++i) A[(size_t)i * n + j] -= u[i] * d;
      }
      A[(size_t)k * n + k] = alpha;
      for (int i = k + 1; i < n; ++i) A[(size_t)i * n + k] = 0;
    }
    for (int j = k + 1; j < n; ++j) {  // remaining norms (rows k+1 ..), recomputed: no drift
      double t = 0;
      for (int i = k + 1; i < n; ++i) t += std::norm(A[(size_t)i * n + j]);
      nrm[j] = t;
    }
  }
  std::vector<cd> X((size_t)n * n, cd(0));  // X = R1^H
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) X[(size_t)j * n + i] = std::conj(A[(size_t)i * n + j]);
  std::vector<cd> VX;
  svd_jacobi(n, n, X, sig, VX);  // X now holds U_X S
  V.assign((size_t)n * n, cd(0));
  for (int kk = 0; kk < n; ++kk) {
    if (!(sig[kk] > 0)) continue;
    const double inv = 1.0 / sig[kk];
    for (int i = 0; i < n; ++i) V[(size_t)perm[i] * n + kk] = X[(size_t)i * n + kk] * inv;
  }
}

// ------------------------------------------------------ device bookkeeping --

namespace {

struct DevAllocs {
  std::vector<void *> ptrs;
  ~DevAllocs() {
    for (void *p : ptrs) cudaFree(p);
  }
};

int g_fault_countdown = -1;  // FIO_FAULT_ALLOC=k: the k-th device allocation fails

cudaError_t dev_alloc(void **p, size_t bytes) {
  if (g_fault_countdown > 0 && --g_fault_countdown == 0) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, std::max<size_t>(bytes, 16));
}

fio_status cuda_status(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return FIO_OK;
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FIO_ENOMEM : FIO_ECUDA;
}

}  // namespace

#define FIO_CK(expr, what)                                  \
  do {                                                      \
    fio_status st_ = cuda_status((expr), (what));           \
    if (st_ != FIO_OK) return st_;                          \
  } while (0)

std::vector<WedgeDev> rc_wedge_table(const std::vector<WedgeDev> &wedges,
                                     const std::vector<int> &grp_first, long long NN,
                                     long long *buf_elems) {
  std::vector<WedgeDev> wrc = wedges;
  long long most = 0;
  for (size_t g = 0; g + 1 < grp_first.size(); ++g) {
    long long rel = 0;
    for (int l = grp_first[g]; l < grp_first[g + 1]; ++l) {
      wrc[l].alpha_off = rel;
      rel += (long long)wrc[l].qp * NN;
    }
    most = std::max(most, rel);
  }
  *buf_elems = most;
  return wrc;
}

void free_plan_device(fio_plan_s *p) {
  void *ptrs[] = {p->d_wedges, p->d_rows,  p->d_ffts,    p->d_twiddle, p->d_alpha,
                  p->d_beta,   p->d_warp,  p->d_grid,    p->d_fhat,    p->d_errword,
                  p->d_warps,  p->d_perm,  p->d_cstart,  p->d_items,   p->d_bins,
                  p->d_bins1,  p->d_wedges_rc, p->d_rc_col, p->d_rc_w, p->d_rc_g, p->d_rc_x};
  for (void *q : ptrs)
    if (q) cudaFree(q);
  p->d_wedges = nullptr; p->d_rows = nullptr; p->d_ffts = nullptr; p->d_twiddle = nullptr;
  p->d_alpha = nullptr; p->d_beta = nullptr; p->d_warp = nullptr; p->d_grid = nullptr;
  p->d_fhat = nullptr; p->d_errword = nullptr;
  p->d_warps = nullptr; p->d_perm = nullptr; p->d_cstart = nullptr; p->d_items = nullptr;
  p->d_bins = nullptr;
  p->d_bins1 = nullptr;
  p->d_wedges_rc = nullptr; p->d_rc_col = nullptr; p->d_rc_w = nullptr; p->d_rc_g = nullptr;
  p->d_rc_x = nullptr;
}

// Piecewise polynomials of the KB kernel on the w unit intervals of a window:
// Chebyshev interpolation in t = 2z - 1 (degree max(8, w + 1)), then monomial
// coefficients by solving the interpolation system in FP64.
void fit_horner(fio_plan_s *p) {
  const int w = p->kb.w;
  const int D = std::min(std::max(8, w + 1), kMaxHornerDeg);
  HornerDev h{};
  h.deg = D;
  const int n = D + 1;
  std::vector<double> tk(n);
  for (int k = 0; k < n; ++k) tk[k] = std::cos(M_PI * (k + 0.5) / n);
  for (int a = 0; a < w; ++a) {
    std::vector<double> A((size_t)n * n), y(n);
    for (int k = 0; k < n; ++k) {
      double pw = 1.0;
      for (int c = 0; c < n; ++c) {
        A[(size_t)k * n + c] = pw;
        pw *= tk[k];
      }
      y[k] = kb_phi_host((tk[k] + 1.0) / 2.0 + w / 2.0 - 1.0 - a, w, p->kb.beta);
    }
    // Gaussian elimination with partial pivoting
    for (int c = 0; c < n; ++c) {
      int piv = c;
      for (int r = c + 1; r < n; ++r)
        if (std::abs(A[(size_t)r * n + c]) > std::abs(A[(size_t)piv * n + c])) piv = r;
      for (int k = 0; k < n; ++k) std::swap(A[(size_t)c * n + k], A[(size_t)piv * n + k]);
      std::swap(y[c], y[piv]);
      for (int r = c + 1; r < n; ++r) {
        const double f = A[(size_t)r * n + c] / A[(size_t)c * n + c];
        for (int k = c; k < n; ++k) A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
        y[r] -= f * y[c];
      }
    }
    for (int c = n - 1; c >= 0; --c) {
      double v = y[c];
      for (int k = c + 1; k < n; ++k) v -= A[(size_t)c * n + k] * y[k];
      y[c] = v / A[(size_t)c * n + c];
    }
    for (int k = 0; k < n; ++k) h.c[k][a] = (float)y[k];
  }
  p->horner = h;
}

template <typename T> static fio_status upload(void **dst, const std::vector<T> &v, const char *w) {
  FIO_CK(dev_alloc(dst, v.size() * sizeof(T)), w);
  if (!v.empty()) FIO_CK(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), w);
  return FIO_OK;
}

template <typename T>
static fio_status upload_tmp(DevAllocs &tmp, T **dst, const std::vector<T> &v, const char *w) {
  void *p = nullptr;
  fio_status s = upload(&p, v, w);
  if (p) tmp.ptrs.push_back(p);
  *dst = (T *)p;
  return s;
}

static bool finite_all(const double *p, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// ------------------------------------------------------------ build_plan --

fio_status build_plan(fio_plan_s *p, int N, const fio_phase *phase, const fio_amplitude *amp,
                      double eps, const fio_options *opt_in) {
  const auto t_start = std::chrono::steady_clock::now();
  fio_options opt;
  fio_options_default(&opt);
  if (opt_in) opt = *opt_in;
  // FIO_PLAN_TRACE=1: one line per separation attempt on stderr (wedge, r, q,
  // validated error, relative tail of the dropped singular values, seconds)
  const char *tr = std::getenv("FIO_PLAN_TRACE");
  const bool trace = tr && *tr && *tr != '0';
  const char *fa = std::getenv("FIO_FAULT_ALLOC");
  g_fault_countdown = fa ? std::atoi(fa) : -1;

  // ---- validation
  if (N < 8 || N > 2048 || (N & 1)) { set_error("N must be even, 8 <= N <= 2048"); return FIO_EINVAL; }
  if (!(eps >= 1e-12 && eps <= 0.1)) { set_error("eps must lie in [1e-12, 0.1]"); return FIO_EINVAL; }
  if (!phase || phase->kind < 0 || phase->kind > 3 || !phase->params) {
    set_error("invalid phase descriptor");
    return FIO_EINVAL;
  }
  const int nscal = phase->kind == FIO_PHASE_SHIFT_WAVE ? 3
                    : (phase->kind == FIO_PHASE_ELLIPSE || phase->kind == FIO_PHASE_ELLIPSE_PRODUCT) ? 4
                                                                                                      : 0;
  if (phase->kind == FIO_PHASE_TAU_MODES) {
    if (phase->nmodes < 1 || phase->nmodes > 65536) { set_error("nmodes out of range"); return FIO_EINVAL; }
    if (!finite_all(phase->params, 5 * phase->nmodes)) { set_error("non-finite phase parameter"); return FIO_EINVAL; }
    for (int j = 0; j < phase->nmodes; ++j) {
      const double m = phase->params[5 * j + 3];
      if (m != std::floor(m) || std::abs(m) > 8) { set_error("tau mode m must be an integer in [-8, 8]"); return FIO_EINVAL; }
    }
  } else if (!finite_all(phase->params, nscal)) {
    set_error("non-finite phase parameter");
    return FIO_EINVAL;
  }
  const fio_amplitude amp1 = amp ? *amp : fio_amplitude{FIO_AMP_ONE, 0, 0};
  if (amp1.kind < 0 || amp1.kind > 2 || !std::isfinite(amp1.a1) || !std::isfinite(amp1.a2) ||
      (amp1.kind == FIO_AMP_HANKEL && amp1.a1 != 1.0 && amp1.a1 != -1.0)) {
    set_error("invalid amplitude");
    return FIO_EINVAL;
  }
  if (opt.precision != FIO_MIXED && opt.precision != FIO_FP64) { set_error("invalid precision"); return FIO_EINVAL; }
  const int L = opt.L > 0 ? opt.L : default_L(N);
  const double sigma = opt.sigma > 0 ? opt.sigma : 2.0;
  if (L < 1 || L > kMaxWedges || sigma < 1.25 || sigma > 4.0) { set_error("L or sigma out of range"); return FIO_EINVAL; }
  const int w = opt.kb_width > 0 ? opt.kb_width : kb_width_for(eps);
  if (w < 3 || w > kMaxKbWidth) { set_error("kb_width must lie in [3, 12]"); return FIO_EINVAL; }
  const int r0 = opt.r0 > 0 ? opt.r0 : 8;
  const int rank_cap = opt.rank_cap > 0 ? opt.rank_cap : 1024;
  const int max_batch = opt.max_batch > 0 ? opt.max_batch : 1;
  if (max_batch > 4096) { set_error("max_batch too large"); return FIO_EINVAL; }
  if (!(opt.sep_cut >= 0 && opt.sep_cut <= 1) || !(opt.sep_target >= 0 && opt.sep_target <= 1)) {
    set_error("sep_cut and sep_target must lie in [0, 1] (0 = default)");
    return FIO_EINVAL;
  }
  if ((opt.alpha_mode != FIO_ALPHA_STORED && opt.alpha_mode != FIO_ALPHA_RECOMPUTE) ||
      opt.alpha_group < 0) {
    set_error("alpha_mode must be FIO_ALPHA_STORED or FIO_ALPHA_RECOMPUTE, alpha_group >= 0");
    return FIO_EINVAL;
  }
  const bool recompute = opt.alpha_mode == FIO_ALPHA_RECOMPUTE;
  if (recompute && opt.precision == FIO_MIXED && amp1.kind == FIO_AMP_HANKEL) {
    set_error("FIO_ALPHA_RECOMPUTE with the Hankel amplitude needs an FP64 plan");
    return FIO_EUNSUPPORTED;
  }

  p->N = N; p->L = L; p->eps = eps; p->sigma = sigma; p->precision = opt.precision;
  p->max_batch = max_batch;
  p->alpha_mode = opt.alpha_mode;
  p->kb.w = w;
  p->kb.beta = kb_beta_for(w, sigma);
  cudaGetDevice(&p->device);
  const long long NN = (long long)N * N;
  const size_t cs = p->precision == FIO_FP64 ? 16 : 8;

  // ---- wedge geometry (host)
  std::vector<std::vector<std::pair<int, int>>> wp(L);
  for (int k1 = -N / 2; k1 < N / 2; ++k1)
    for (int k2 = -N / 2; k2 < N / 2; ++k2) wp[wedge_of(k1, k2, L)].push_back({k1, k2});
  p->wedges.resize(L);
  p->rows.clear();
  p->pt_k1.clear(); p->pt_k2.clear();
  std::vector<std::vector<int>> x1p(L), x2p(L);
  for (int l = 0; l < L; ++l) {
    if (wp[l].empty()) { set_error("empty wedge: L too large for N"); return FIO_EINVAL; }
    std::vector<RowDev> rows;
    std::vector<int> k1s, k2s;
    std::string err;
    if (!wedge_geometry(wp[l], sigma, w, p->wedges[l], rows, k1s, k2s, x1p[l], x2p[l], err)) {
      set_error(err);
      return FIO_EINVAL;
    }
    p->wedges[l].row_off = (int)p->rows.size();
    p->wedges[l].pt_off = (int)p->pt_k1.size();
    for (auto &rw : rows) {
      rw.wedge = l;
      p->max_row_len = std::max(p->max_row_len, rw.len);
      p->rows.push_back(rw);
    }
    p->pt_k1.insert(p->pt_k1.end(), k1s.begin(), k1s.end());
    p->pt_k2.insert(p->pt_k2.end(), k2s.begin(), k2s.end());
  }

  // ---- FFT plans and twiddles for every length used
  std::vector<int> lens = {N};
  for (auto &wd : p->wedges) { lens.push_back(wd.m1); lens.push_back(wd.m2); }
  std::sort(lens.begin(), lens.end());
  lens.erase(std::unique(lens.begin(), lens.end()), lens.end());
  std::vector<double> tw;
  p->ffts.clear();
  for (int n : lens) {
    FftPlanDev f{};
    f.n = n;
    const auto rad = fft_factor(n);
    if (rad.empty() || (int)rad.size() > kMaxRadixStages || n > kMaxFftLen) {
      set_error("unsupported FFT length " + std::to_string(n));
      return FIO_EUNSUPPORTED;
    }
    f.nstages = (int)rad.size();
    for (size_t i = 0; i < rad.size(); ++i) f.radix[i] = rad[i];
    f.tw_off = (int)(tw.size() / 2);
    for (int k = 0; k < n; ++k) {
      tw.push_back(std::cos(2.0 * M_PI * k / n));
      tw.push_back(-std::sin(2.0 * M_PI * k / n));
    }
    p->ffts.push_back(f);
  }
  auto fft_index = [&](int n) {
    for (size_t i = 0; i < p->ffts.size(); ++i)
      if (p->ffts[i].n == n) return (int)i;
    return -1;
  };
  for (auto &wd : p->wedges) {
    wd.fft1 = fft_index(wd.m1);
    wd.fft2 = fft_index(wd.m2);
    wd.tw1_off = p->ffts[wd.fft1].tw_off;
    wd.tw2_off = p->ffts[wd.fft2].tw_off;
  }
  fit_horner(p);

  // ---- phase data on the device
  DevAllocs tmp;
  PhaseDev ph{};
  ph.kind = phase->kind == FIO_PHASE_ELLIPSE_PRODUCT ? FIO_PHASE_ELLIPSE : phase->kind;
  ph.ell_form = phase->kind == FIO_PHASE_ELLIPSE_PRODUCT ? 1 : 0;
  ph.nmodes = phase->kind == FIO_PHASE_TAU_MODES ? phase->nmodes : 0;
  for (int i = 0; i < nscal; ++i) ph.p[i] = phase->params[i];
  ph.amp_kind = amp1.kind;
  ph.a1 = amp1.a1;
  ph.a2 = amp1.a2;
  p->phase = ph;
  double *d_modes = nullptr;
  {
    const int nprm = ph.nmodes ? 5 * ph.nmodes : nscal;
    std::vector<double> modes(phase->params, phase->params + nprm);
    fio_status s = upload_tmp(tmp, &d_modes, modes, "upload phase");
    if (s != FIO_OK) return s;
  }
  void *d_xdata = nullptr;
  FIO_CK(dev_alloc(&d_xdata, plan_xdata_bytes(ph, N)), "alloc phase data");
  tmp.ptrs.push_back(d_xdata);
  FIO_CK(plan_xdata(ph, d_modes, N, d_xdata, 0), "phase data kernel");

  // warped points need only the geometry
  {
    void *q = nullptr;
    fio_status s = upload(&q, p->wedges, "upload wedges");
    p->d_wedges = (WedgeDev *)q;
    if (s != FIO_OK) return s;
  }
  FIO_CK(dev_alloc((void **)&p->d_warp, (size_t)NN * L * sizeof(uint2)), "alloc warp");
  FIO_CK(plan_warp(ph, d_xdata, N, L, p->d_wedges, p->d_warp, 0), "warp kernel");
  if (opt.surrogate && phase->kind == FIO_PHASE_TAU_MODES) {
    // the surrogate's warped points, if its judged error is within budget: the
    // residual below always uses the plain phase, so the factorisation of
    // a exp(2 pi i Phi) stays exact and only the rank can change
    const fio_surrogate_info *si = surrogate_info(opt.surrogate);
    const double xi_max = N / std::sqrt(2.0);
    p->sur_warp_cycles = xi_max * (si->heldout_tau_maxerr + si->heldout_dtheta_maxerr);
    p->sur_residual_cycles = xi_max * si->heldout_tau_maxerr;
    const double budget = opt.surrogate_warp_budget > 0 ? opt.surrogate_warp_budget : 0.5;
    // the single-precision regeneration of the recompute mode writes the residual
    // phase with the exact gradient as the warp, so it keeps the plain warp
    const bool rc32 = recompute && p->precision == FIO_MIXED;
    if (p->sur_warp_cycles <= budget && !rc32) {
      FIO_CK(surrogate_warp(opt.surrogate, N, L, p->d_wedges, p->d_warp), "surrogate warp");
      p->sur_warp = 1;
    }
  }

  // ---- pass 1: randomized separation rank per wedge (Sec. 3.2)
  p->wedge_r.assign(L, 0);
  double2 *d_AC = nullptr, *d_qrw = nullptr, *d_stk0 = nullptr, *d_stk1 = nullptr;
  long long ac_cap = 0, qrw_cap = 0, stk0_cap = 0, stk1_cap = 0;
  auto regrow = [&](double2 **q, long long &cap, long long need, const char *what) -> fio_status {
    if (need <= cap) return FIO_OK;
    if (*q) {
      tmp.ptrs.erase(std::find(tmp.ptrs.begin(), tmp.ptrs.end(), (void *)*q));
      cudaFree(*q);
      *q = nullptr;
      cap = 0;
    }
    FIO_CK(dev_alloc((void **)q, (size_t)need * sizeof(double2)), what);
    tmp.ptrs.push_back(*q);
    cap = need;
    return FIO_OK;
  };
  auto ensure_ac = [&](int r) -> fio_status {
    return regrow(&d_AC, ac_cap, (long long)r * NN, "alloc A_C");
  };
  // workspace of the tall-skinny QR of A_C (pass 1 only)
  auto ensure_qr = [&](int r) -> fio_status {
    const long long st = (long long)tsqr_stack_elems(NN, r);
    fio_status s = regrow(&d_qrw, qrw_cap, (long long)r * NN, "alloc QR workspace");
    if (s == FIO_OK) s = regrow(&d_stk0, stk0_cap, st, "alloc QR stack");
    if (s == FIO_OK) s = regrow(&d_stk1, stk1_cap, st, "alloc QR stack");
    return s;
  };
  int *d_ck1 = nullptr, *d_ck2 = nullptr;
  // the largest sample: rank_cap columns, or a whole wedge of up to 2 rank_cap
  // columns (the exact projection); T is fitted on up to 4 rmax rows
  const int rmax = 2 * rank_cap, nrmax = std::max(4 * rmax, 256);
  FIO_CK(dev_alloc((void **)&d_ck1, sizeof(int) * rmax * 2 + 64), "alloc samples");
  tmp.ptrs.push_back(d_ck1);
  d_ck2 = d_ck1 + rmax + 16;
  const int *pk1 = p->pt_k1.data(), *pk2 = p->pt_k2.data();

  auto eval_cols = [&](int l, const std::vector<int> &C) -> fio_status {
    const WedgeDev &wd = p->wedges[l];
    const int r = (int)C.size();
    std::vector<int> c1(r), c2(r);
    for (int i = 0; i < r; ++i) { c1[i] = pk1[wd.pt_off + C[i]]; c2[i] = pk2[wd.pt_off + C[i]]; }
    FIO_CK(cudaMemcpy(d_ck1, c1.data(), sizeof(int) * r, cudaMemcpyHostToDevice), "upload C");
    FIO_CK(cudaMemcpy(d_ck2, c2.data(), sizeof(int) * r, cudaMemcpyHostToDevice), "upload C");
    fio_status s = ensure_ac(r);
    if (s != FIO_OK) return s;
    FIO_CK(plan_eval_cols(ph, d_xdata, N, wd, p->d_warp + (size_t)l * NN, d_ck1, d_ck2, r, d_AC, 0),
           "A_C kernel");
    return FIO_OK;
  };

  // per-wedge scratch of the separation
  int maxnpts = 0;
  for (auto &wd : p->wedges) maxnpts = std::max(maxnpts, wd.npts);
  const int s_val = (int)std::min<long long>(kValidationRows, NN);
  int *d_pk1 = nullptr, *d_pk2 = nullptr, *d_rx = nullptr, *d_gx = nullptr;
  double *d_err = nullptr, *d_nrm = nullptr;
  double2 *d_W = nullptr, *d_P = nullptr, *d_UG = nullptr, *d_T = nullptr;
  long long T_cap = 0;
  auto scratch = [&](void **q, size_t bytes, const char *what) -> fio_status {
    FIO_CK(dev_alloc(q, bytes), what);
    tmp.ptrs.push_back(*q);
    return FIO_OK;
  };
  {
    fio_status s = FIO_OK;
    if (s == FIO_OK) s = scratch((void **)&d_pk1, sizeof(int) * (size_t)maxnpts * 2, "alloc points");
    if (s == FIO_OK) s = scratch((void **)&d_err, sizeof(double) * (size_t)maxnpts * 2, "alloc validation");
    if (s == FIO_OK) s = scratch((void **)&d_rx, sizeof(int) * (size_t)(nrmax + kValidationRows), "alloc rows");
    if (s == FIO_OK) s = scratch((void **)&d_W, sizeof(double2) * (size_t)rmax * rmax, "alloc W");
    if (s == FIO_OK) s = scratch((void **)&d_P, sizeof(double2) * (size_t)rmax * nrmax, "alloc P");
    if (s == FIO_OK) s = scratch((void **)&d_UG, sizeof(double2) * (size_t)kValidationRows * rmax, "alloc U rows");
    if (s != FIO_OK) return s;
  }
  d_pk2 = d_pk1 + maxnpts;
  d_nrm = d_err + maxnpts;
  d_gx = d_rx + nrmax;

  // rows X of U = A_C W (A_C on the device, [x][c]); W is r x q
  auto u_rows = [&](const std::vector<int> &X, int r, int q, const std::vector<cd> &W,
                    std::vector<cd> &out) -> fio_status {
    out.assign(X.size() * (size_t)q, cd(0));
    std::vector<cd> arow(r);
    for (size_t i = 0; i < X.size(); ++i) {
      FIO_CK(cudaMemcpy(arow.data(), d_AC + (size_t)X[i] * r, sizeof(cd) * r, cudaMemcpyDeviceToHost),
             "download A_C row");
      for (int t = 0; t < q; ++t) {
        cd acc = 0;
        for (int c = 0; c < r; ++c) acc += arow[c] * W[(size_t)c * q + t];
        out[i * q + t] = acc;
      }
    }
    return FIO_OK;
  };
  // P = U_R^+ (q x nr) from the SVD of U_R (one-sided Jacobi): U_R W = Y with
  // orthogonal columns of norms s_k, so U_R^+ = W diag(1/s_k^2) Y^H over the
  // s_k above cut * s_1 (Sec. 3.2's pseudo-inverse, without normal equations)
  auto pinv = [&](const std::vector<cd> &UR, int nr, int q, double cut) {
    std::vector<cd> Y = UR, Wv;
    std::vector<double> su;
    svd_jacobi(nr, q, Y, su, Wv);
    std::vector<cd> P((size_t)q * nr, cd(0));
    for (int k = 0; k < q; ++k) {
      if (!(su[k] > cut * su[0])) continue;
      const double inv2 = 1.0 / (su[k] * su[k]);
      for (int t = 0; t < q; ++t) {
        const cd wt = Wv[(size_t)t * q + k] * inv2;
        for (int i = 0; i < nr; ++i) P[(size_t)t * nr + i] += wt * std::conj(Y[(size_t)i * q + k]);
      }
    }
    return P;
  };

  struct Sep {
    std::vector<int> C, R;
    std::vector<cd> W, P;
    std::vector<cd> T;  // exact projection (the sample holds every column): T = S_q V_q^H
    int q = 0;
    double est = 0;
  };
  std::vector<Sep> sep(L);
  p->wedge_err.assign(L, 0.0);
  const double sep_cut = opt.sep_cut > 0 ? opt.sep_cut : kSvdFraction;
  const double sep_target = opt.sep_target > 0 ? opt.sep_target : kValidationTarget;
  const double svd_cut = sep_cut * eps;
  for (int l = 0; l < L; ++l) {
    const WedgeDev &wd = p->wedges[l];
    const int npts = wd.npts;
    FIO_CK(cudaMemcpy(d_pk1, pk1 + wd.pt_off, sizeof(int) * npts, cudaMemcpyHostToDevice), "upload points");
    FIO_CK(cudaMemcpy(d_pk2, pk2 + wd.pt_off, sizeof(int) * npts, cudaMemcpyHostToDevice), "upload points");
    std::vector<int> anchors;  // columns kept from earlier attempts (worst fitted)
    int r = std::min({r0, npts, rank_cap});
    for (int attempt = 0;; ++attempt) {
      // C: the anchors plus uniform random columns (Sec. 3.2, step 1)
      SplitMix64 rng{mix_seed(opt.seed, (uint64_t)l + 1, 3 * (uint64_t)attempt + 1)};
      if ((int)anchors.size() > r) anchors.resize(r);
      std::vector<int> C = anchors;
      std::unordered_set<int> have(C.begin(), C.end());
      for (int c : sample_distinct(npts, std::min(npts, r), rng))
        if ((int)C.size() < r && have.insert(c).second) C.push_back(c);
      while ((int)C.size() < r) {
        const int c = (int)rng.below((uint64_t)npts);
        if (have.insert(c).second) C.push_back(c);
      }
      std::sort(C.begin(), C.end());
      const int rc = (int)C.size();
      // SVD of A_[C] (step 2): A_[C] = Q R by Householder TSQR on the device,
      // R = U_R S V^H by one-sided Jacobi; then A_[C] V = Q U_R S, so
      // U = A_[C] V S^-1 has orthonormal columns.  The singular values keep the
      // absolute accuracy eps_mach s_1 that a Gram matrix would square.
      fio_status s = eval_cols(l, C);
      if (s != FIO_OK) return s;
      if ((s = ensure_qr(rc)) != FIO_OK) return s;
      std::vector<cd> Rm((size_t)rc * rc);
      FIO_CK(plan_tsqr(d_AC, NN, rc, d_qrw, d_stk0, d_stk1, reinterpret_cast<double2 *>(Rm.data()), 0),
             "TSQR kernel");
      FIO_CK(cudaStreamSynchronize(0), "TSQR kernel");
      std::vector<double> sv;
      std::vector<cd> V;
      svd_right_pivoted(rc, Rm, sv, V);
      const double s1 = sv[0];
      int q = 0;
      while (q < rc && sv[q] > svd_cut * s1) ++q;
      q = std::max(q, 1);
      std::vector<cd> Wm((size_t)rc * q);
      for (int i = 0; i < rc; ++i)
        for (int t = 0; t < q; ++t)
          Wm[(size_t)i * q + t] = sv[t] > 0 ? V[(size_t)i * rc + t] / sv[t] : cd(0);
      // rows R and T = U_[R]^+ A_[R] (steps 3-4).  When the sample holds every
      // column of the wedge, A_[C] is the whole wedge block and the projection
      // is exact: T = U^H A = S_q V_q^H, with no row sample.
      const bool exact = rc >= npts;
      std::vector<int> R;
      std::vector<cd> P, Tex;
      if ((s = regrow(&d_T, T_cap, (long long)q * npts, "alloc T")) != FIO_OK) return s;
      if (exact) {
        Tex.assign((size_t)q * npts, cd(0));
        for (int t = 0; t < q; ++t)
          for (int c = 0; c < rc; ++c) Tex[(size_t)t * npts + C[c]] = sv[t] * std::conj(V[(size_t)c * rc + t]);
        FIO_CK(cudaMemcpy(d_T, Tex.data(), sizeof(cd) * Tex.size(), cudaMemcpyHostToDevice), "upload T");
      } else {
        SplitMix64 rr{mix_seed(opt.seed, (uint64_t)l + 1, 3 * (uint64_t)attempt + 2)};
        // the row sample of the least-squares fit: its noise amplification
        // (1 - sqrt(q / nr))^-1 stays near 1.5 or below
        const int nr = (int)std::min<long long>(NN, std::min(nrmax, std::max({rc, 8 * q, 256})));
        R = sample_distinct((int)NN, nr, rr);
        std::vector<cd> UR;
        if ((s = u_rows(R, rc, q, Wm, UR)) != FIO_OK) return s;
        P = pinv(UR, nr, q, svd_cut);
        FIO_CK(cudaMemcpy(d_P, P.data(), sizeof(cd) * q * nr, cudaMemcpyHostToDevice), "upload P");
        FIO_CK(cudaMemcpy(d_rx, R.data(), sizeof(int) * nr, cudaMemcpyHostToDevice), "upload R");
        FIO_CK(plan_form_beta(ph, d_xdata, N, wd, p->d_warp + (size_t)l * NN, d_rx, nr, q, d_P, d_pk1,
                              d_pk2, nullptr, d_T, FIO_FP64, 0),
               "T kernel");
      }
      // validation on fresh rows against every column of the wedge
      SplitMix64 rg{mix_seed(opt.seed, (uint64_t)l + 1, 3 * (uint64_t)attempt + 3)};
      std::vector<int> Gx = sample_distinct((int)NN, s_val, rg);
      std::vector<cd> UG;
      if ((s = u_rows(Gx, rc, q, Wm, UG)) != FIO_OK) return s;
      FIO_CK(cudaMemcpy(d_UG, UG.data(), sizeof(cd) * UG.size(), cudaMemcpyHostToDevice), "upload U rows");
      FIO_CK(cudaMemcpy(d_gx, Gx.data(), sizeof(int) * s_val, cudaMemcpyHostToDevice), "upload rows");
      FIO_CK(plan_validate(ph, d_xdata, N, wd, p->d_warp + (size_t)l * NN, d_gx, s_val, d_UG, d_T, q,
                           d_pk1, d_pk2, d_err, d_nrm, 0),
             "validation kernel");
      std::vector<double> err(npts), nrm(npts);
      FIO_CK(cudaMemcpy(err.data(), d_err, sizeof(double) * npts, cudaMemcpyDeviceToHost), "download");
      FIO_CK(cudaMemcpy(nrm.data(), d_nrm, sizeof(double) * npts, cudaMemcpyDeviceToHost), "download");
      double se = 0, sn = 0;
      for (int i = 0; i < npts; ++i) { se += err[i]; sn += nrm[i]; }
      const double est = std::sqrt(se / std::max(sn, 1e-300));
      const bool ok = (est <= sep_target * eps && 3 * q <= rc) || exact;
      if (trace) {
        double all = 0, tail = 0;
        for (int k = 0; k < rc; ++k) {
          all += sv[k] * sv[k];
          if (k >= q) tail += sv[k] * sv[k];
        }
        std::fprintf(stderr,
                     "fio plan: wedge %d attempt %d r %d q %d est %.3e tail %.3e s_q/s_1 %.3e "
                     "exact %d t %.2fs\n",
                     l, attempt, rc, q, est, std::sqrt(tail / std::max(all, 1e-300)),
                     q < rc ? sv[q] / s1 : 0.0, (int)exact,
                     std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count());
      }
      // no larger sample is allowed once rank_cap columns are taken, unless the
      // whole wedge (at most 2 rank_cap columns) can still be
      const bool capped = rc >= rank_cap && npts > rmax;
      if (ok || capped) {
        if (!ok && est > eps) {
          set_error("wedge " + std::to_string(l) + ": separation error " + std::to_string(est) +
                    " above eps with rank_cap samples");
          return FIO_ERANK;
        }
        sep[l].C = C;
        sep[l].R = R;
        sep[l].W = Wm;
        sep[l].P = P;
        sep[l].T = Tex;
        sep[l].q = q;
        sep[l].est = est;
        p->wedges[l].q = q;
        p->wedge_r[l] = rc;
        p->wedge_err[l] = est;
        break;
      }
      // pivot: keep the worst-fitted columns for the next, doubled sample
      std::vector<int> order(npts);
      std::iota(order.begin(), order.end(), 0);
      std::sort(order.begin(), order.end(), [&](int a, int b) { return err[a] > err[b]; });
      const int add = std::max(1, rc / 4);
      std::unordered_set<int> inC(C.begin(), C.end()), inA(anchors.begin(), anchors.end());
      int added = 0;
      for (int i = 0; i < npts && added < add; ++i)
        if (!inC.count(order[i]) && inA.insert(order[i]).second) {
          anchors.push_back(order[i]);
          ++added;
        }
      r = std::min({2 * r, rank_cap, npts});
      // a wedge of at most 2 rank_cap columns is sampled whole once half of it
      // would be: the exact projection then needs no row sample
      if (2 * r >= npts && npts <= rmax) r = npts;
    }
  }

  for (double2 **q : {&d_qrw, &d_stk0, &d_stk1}) {  // the QR workspace is done
    if (!*q) continue;
    tmp.ptrs.erase(std::find(tmp.ptrs.begin(), tmp.ptrs.end(), (void *)*q));
    cudaFree(*q);
    *q = nullptr;
  }

  // ---- layout of the factors and grids
  long long aoff = 0, boff = 0, gunit = 0, koff = 0;
  long long rc_cols = 0, rc_wn = 0;
  for (int l = 0; l < L; ++l) {
    WedgeDev &wd = p->wedges[l];
    wd.qp = wd.q + (wd.q & 1);
    wd.rc_r = recompute ? (int)sep[l].C.size() : 0;
    wd.rc_col_off = rc_cols;
    wd.rc_w_off = rc_wn;
    rc_cols += wd.rc_r;
    rc_wn += (long long)wd.rc_r * wd.qp;
    wd.alpha_off = aoff;
    wd.beta_off = boff;
    wd.grid_unit = gunit;
    wd.nb1 = (wd.m1 + kBin - 1) / kBin;
    wd.nb2 = (wd.m2 + kBin - 1) / kBin;
    wd.key_off = koff;
    aoff += (long long)wd.qp * NN;
    boff += (long long)wd.qp * wd.npts;
    gunit += (long long)wd.m1 * wd.m2 * wd.qp;
    koff += (long long)wd.nb1 * wd.nb2 * kBin * kBin + 1;
  }
  p->alpha_elems = aoff;
  // recompute mode: gamma^x of alpha_group wedges at a time, in a buffer the
  // size of the largest group; the wedge table d_wedges_rc places each wedge's
  // factors relative to its group
  std::vector<WedgeDev> wrc;
  long long abuf = aoff;
  if (recompute) {
    const int G = opt.alpha_group > 0 ? std::min(opt.alpha_group, L) : std::min(4, L);
    p->grp_first.clear();
    for (int l = 0; l < L; l += G) p->grp_first.push_back(l);
    p->grp_first.push_back(L);
    wrc = rc_wedge_table(p->wedges, p->grp_first, NN, &abuf);
    p->rc_cols = rc_cols;
    p->rc_w_elems = rc_wn;
    p->alpha_elems = abuf;
  }
  p->cstart_elems = koff;
  p->twiddle_elems = (long long)tw.size() / 2;
  p->beta_elems = boff;
  p->grid_units = gunit;
  FIO_CK(dev_alloc(&p->d_alpha, (size_t)abuf * cs), "alloc alpha");
  FIO_CK(dev_alloc(&p->d_beta, (size_t)boff * cs), "alloc beta");
  FIO_CK(dev_alloc(&p->d_grid, (size_t)gunit * max_batch * cs), "alloc grids");
  FIO_CK(dev_alloc(&p->d_fhat, (size_t)NN * max_batch * cs), "alloc spectrum");
  FIO_CK(dev_alloc((void **)&p->d_perm, sizeof(uint32_t) * (size_t)NN * L), "alloc point order");
  FIO_CK(dev_alloc((void **)&p->d_warps, sizeof(uint2) * (size_t)NN * L), "alloc sorted warp");
  FIO_CK(dev_alloc((void **)&p->d_cstart, sizeof(int) * (size_t)koff), "alloc bucket tables");
  FIO_CK(dev_alloc((void **)&p->d_errword, sizeof(int)), "alloc error word");
  FIO_CK(cudaMemset(p->d_errword, 0, sizeof(int)), "clear error word");
  // the padded rank term (t = q when q is odd) must stay exactly zero
  FIO_CK(cudaMemset(p->d_alpha, 0, (size_t)abuf * cs), "clear alpha");
  FIO_CK(cudaMemset(p->d_beta, 0, (size_t)boff * cs), "clear beta");
  FIO_CK(cudaMemcpy(p->d_wedges, p->wedges.data(), sizeof(WedgeDev) * L, cudaMemcpyHostToDevice), "upload wedges");
  {
    void *q = nullptr;
    fio_status s = upload(&q, p->rows, "upload rows");
    p->d_rows = (RowDev *)q;
    if (s != FIO_OK) return s;
    s = upload(&q, p->ffts, "upload fft plans");
    p->d_ffts = (FftPlanDev *)q;
    if (s != FIO_OK) return s;
    if (p->precision == FIO_FP64) {
      s = upload(&p->d_twiddle, tw, "upload twiddles");
    } else {
      std::vector<float> twf(tw.begin(), tw.end());
      s = upload(&p->d_twiddle, twf, "upload twiddles");
    }
    if (s != FIO_OK) return s;
  }

  // ---- pass 2: gamma^x = U (with centre factor and 1/N), gamma^xi = T / phihat
  double *d_dec = nullptr;
  {
    fio_status s = scratch((void **)&d_dec, sizeof(double) * (size_t)maxnpts, "alloc deconvolution");
    if (s != FIO_OK) return s;
  }
  std::vector<std::vector<int>> cstart(L);
  // recompute mode: the x-independent values of every sampled column, and V S^-1
  std::vector<RcCol> rc_col;
  std::vector<cd> rc_w;
  std::vector<float> rc_g;
  const bool tau_g = recompute && ph.kind == FIO_PHASE_TAU_MODES && p->precision == FIO_MIXED;
  for (int l = 0; l < L; ++l) {
    const WedgeDev &wd = p->wedges[l];
    const Sep &sp = sep[l];
    const int rc = (int)sp.C.size(), q = sp.q, nr = (int)sp.R.size();
    FIO_CK(sort_wedge_points(p, l, cstart[l]), "point sort");
    if (recompute) {
      const double th = 2.0 * M_PI * l / L, ct = std::cos(th), st = std::sin(th);
      for (int k = 0; k < rc; ++k) {
        const int k1 = pk1[wd.pt_off + sp.C[k]], k2 = pk2[wd.pt_off + sp.C[k]];
        const double r = std::hypot((double)k1, (double)k2);
        const double dot = ct * k1 + st * k2, cross = ct * k2 - st * k1;
        RcCol c{};
        c.k1 = k1;
        c.k2 = k2;
        c.ctk1 = (float)(ct * k1);
        c.stk2 = (float)(st * k2);
        c.cross2 = (float)(cross * cross);
        c.fk1 = (float)k1;
        c.fk2 = (float)k2;
        c.rsw = (ph.kind == FIO_PHASE_SHIFT_WAVE && r > 0) ? (float)(ph.p[2] * cross * cross / (r + dot)) : 0.f;
        c.ampc = ph.amp_kind == FIO_AMP_SEPARABLE ? (float)(1.0 + ph.a2 * (r > 0 ? k1 / r : 1.0)) : 1.f;
        rc_col.push_back(c);
        for (int t = 0; t < wd.qp; ++t) rc_w.push_back(t < q ? sp.W[(size_t)k * q + t] : cd(0.0));
        if (tau_g) {
          // G_m = |xi| e^{i m theta_l} ((cos m d - cos d) + i (sin m d - m sin d))
          const double d = r > 0 ? std::atan2(cross, dot) : 0.0;
          for (int m = -kTauMmax; m <= kTauMmax; ++m) {
            const double re = -2.0 * std::sin((m + 1) * d / 2) * std::sin((m - 1) * d / 2);
            const double im = std::sin(m * d) - m * std::sin(d);
            const cd gm = r * std::polar(1.0, m * th) * cd(re, im);
            rc_g.push_back((float)gm.real());
            rc_g.push_back((float)gm.imag());
          }
        }
      }
    } else {
      fio_status s = eval_cols(l, sp.C);
      if (s != FIO_OK) return s;
      FIO_CK(cudaMemcpy(d_W, sp.W.data(), sizeof(cd) * rc * q, cudaMemcpyHostToDevice), "upload W");
      FIO_CK(plan_form_alpha(d_AC, N, rc, q, d_W, wd, p->d_warp + (size_t)l * NN,
                             p->d_perm + (size_t)l * NN,
                             (char *)p->d_alpha + (size_t)wd.alpha_off * cs, p->precision, 0),
             "alpha kernel");
    }
    std::vector<double> dec(wd.npts);
    for (int i = 0; i < wd.npts; ++i)
      dec[i] = 1.0 / (kb_phihat_host((double)x1p[l][i] / wd.m1, w, p->kb.beta) *
                      kb_phihat_host((double)x2p[l][i] / wd.m2, w, p->kb.beta));
    char *beta_l = (char *)p->d_beta + (size_t)wd.beta_off * cs;
    if (!sp.T.empty()) {  // exact projection: beta' = T / phihat, formed here
      const size_t n = (size_t)q * wd.npts;
      if (p->precision == FIO_FP64) {
        std::vector<cd> b(n);
        for (size_t e = 0; e < n; ++e) b[e] = sp.T[e] * dec[e % wd.npts];
        FIO_CK(cudaMemcpy(beta_l, b.data(), sizeof(cd) * n, cudaMemcpyHostToDevice), "upload beta");
      } else {
        std::vector<float> b(2 * n);
        for (size_t e = 0; e < n; ++e) {
          const cd v = sp.T[e] * dec[e % wd.npts];
          b[2 * e] = (float)v.real();
          b[2 * e + 1] = (float)v.imag();
        }
        FIO_CK(cudaMemcpy(beta_l, b.data(), sizeof(float) * 2 * n, cudaMemcpyHostToDevice), "upload beta");
      }
      continue;
    }
    FIO_CK(cudaMemcpy(d_P, sp.P.data(), sizeof(cd) * q * nr, cudaMemcpyHostToDevice), "upload P");
    FIO_CK(cudaMemcpy(d_rx, sp.R.data(), sizeof(int) * nr, cudaMemcpyHostToDevice), "upload R");
    FIO_CK(cudaMemcpy(d_pk1, pk1 + wd.pt_off, sizeof(int) * wd.npts, cudaMemcpyHostToDevice), "upload points");
    FIO_CK(cudaMemcpy(d_pk2, pk2 + wd.pt_off, sizeof(int) * wd.npts, cudaMemcpyHostToDevice), "upload points");
    FIO_CK(cudaMemcpy(d_dec, dec.data(), sizeof(double) * wd.npts, cudaMemcpyHostToDevice), "upload deconvolution");
    FIO_CK(plan_form_beta(ph, d_xdata, N, wd, p->d_warp + (size_t)l * NN, d_rx, nr, q, d_P, d_pk1,
                          d_pk2, d_dec, beta_l, p->precision, 0),
           "beta kernel");
  }
  if (recompute) {
    fio_status s = upload((void **)&p->d_rc_col, rc_col, "upload sampled columns");
    if (s != FIO_OK) return s;
    if (p->precision == FIO_FP64) {
      s = upload(&p->d_rc_w, rc_w, "upload V S^-1");
    } else {
      std::vector<float> wf(2 * rc_w.size());
      for (size_t e = 0; e < rc_w.size(); ++e) {
        wf[2 * e] = (float)rc_w[e].real();
        wf[2 * e + 1] = (float)rc_w[e].imag();
      }
      s = upload(&p->d_rc_w, wf, "upload V S^-1");
    }
    if (s != FIO_OK) return s;
    if (tau_g) {
      s = upload(&p->d_rc_g, rc_g, "upload tau column factors");
      if (s != FIO_OK) return s;
    }
    s = upload((void **)&p->d_wedges_rc, wrc, "upload wedge table");
    if (s != FIO_OK) return s;
    // per-x phase data: the plan's own for FP64 plans, single precision otherwise
    const bool xdep = ph.kind == FIO_PHASE_ELLIPSE || ph.kind == FIO_PHASE_TAU_MODES;
    if (p->precision == FIO_FP64) {
      tmp.ptrs.erase(std::find(tmp.ptrs.begin(), tmp.ptrs.end(), d_xdata));
      p->d_rc_x = d_xdata;
      p->rc_x_elems = (long long)plan_xdata_bytes(ph, N);
    } else if (xdep) {
      p->rc_x_elems = (long long)plan_xdata_bytes(ph, N) / 2;  // bytes: float2 for double2
      FIO_CK(dev_alloc(&p->d_rc_x, (size_t)p->rc_x_elems), "alloc phase data");
      FIO_CK(rc_xdata_f32(ph, d_xdata, N, p->d_rc_x, 0), "phase data");
    }
  }
  FIO_CK(cudaDeviceSynchronize(), "plan construction");
  FIO_CK(build_work_lists(p, cstart), "work lists");

  // ---- summary
  p->q_max = 0; p->q_min = 1 << 30; p->r_max = 0;
  double qs = 0;
  for (int l = 0; l < L; ++l) {
    p->q_max = std::max(p->q_max, p->wedges[l].q);
    p->q_min = std::min(p->q_min, p->wedges[l].q);
    p->r_max = std::max(p->r_max, p->wedge_r[l]);
    qs += p->wedges[l].q;
  }
  p->q_mean = qs / L;
  p->sep_err = 0;
  for (double e : p->wedge_err) p->sep_err = std::max(p->sep_err, e);
  p->bytes_total = (sizeof(uint2) + sizeof(uint32_t)) * (size_t)L * NN + sizeof(int) * (size_t)koff +
                   sizeof(int4) * (size_t)p->n_items +
                   sizeof(int2) * (size_t)(p->n_bins + p->n_bins1) + rc_bytes(p) +
                   (size_t)(abuf + boff) * cs + (size_t)gunit * max_batch * cs +
                   (size_t)NN * max_batch * cs + (size_t)NN * L * sizeof(uint2) +
                   tw.size() / 2 * cs + p->rows.size() * sizeof(RowDev) +
                   p->wedges.size() * sizeof(WedgeDev) + p->ffts.size() * sizeof(FftPlanDev);
  // algorithmic bytes of one batch-1 apply: input, spectrum (written and read),
  // output, both factors, warped points, every grid written once and read once
  p->alg_bytes = (unsigned long long)(4 * NN * cs + (aoff + boff) * cs + NN * L * 8 + 2 * gunit * cs);
  p->plan_seconds =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  return FIO_OK;
}

}  // namespace fio
