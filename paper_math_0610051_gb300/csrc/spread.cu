// spread.cu -- S4a of the mixed-precision adjoint (Sec. 3.5 steps 1-2): the
// type-1 spread of conj(alpha'_t(x)) g_b(x) onto the oversampled grids, for all
// B inputs of a launch in one sweep.
//
// A CTA owns the kBin x kBin cells of one bin of one wedge and gathers into each
// of them the contributions of every point whose KB window covers it: the points
// whose window-start cell lies in the (kBin + w - 1)^2 region that ends at the
// bin, found through the plan's bucket table (points are sorted by start cell).
// Every grid cell is written exactly once, by its own bin, with plain stores: no
// atomics and no clearing of the grids, so the adjoint is deterministic.
//
// Warp c owns cell column c of the bin.  Its lanes cover the channels of a cell,
// ch = b qp + t (input b, rank term t), the grid's innermost dimension, so every
// lane of a warp walks the same sequence of points and reads the same weights:
// a lane holds UPL single-term units, ch = lane + 32 j.  This layout serves
// launches whose cells hold more than 32 channels (several inputs); a single
// input takes the bin-pair kernel k_spread_bin, whose lane groups own one column
// each.
// The warp walks the region's start rows top to bottom, keeping in registers the
// w cell rows that the current start row can still reach: a point of start row i
// and start column j (w - 1 or fewer columns left of the cell column) adds
// w1[a1] (w2[a2] v) to row a1 of the window, v = conj(alpha'_t) g_b.  When start
// row i is done, the top cell row is final: it is stored and the window slides.
//
// Candidates come in chunks in region order.  For each chunk the CTA forms the
// KB weights and v for all channels once (alpha' and g are read once per
// launch, whatever B is), then every warp sweeps.  The copies of the next
// chunk's alpha' rows and inputs are started before the sweep and land during
// it (two staging buffers).  A start row may continue in the next chunk; the
// sweep state stays in registers.
//
// A point whose window start disagrees with the bucket it was sorted into is
// recorded in the plan's error word and skipped.
#include <cuda_runtime.h>

#include <algorithm>

#include "apply_common.cuh"
#include "bin_common.cuh"
#include "fio_internal.h"

namespace fio {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSwThreads = kBin * 32;  // one warp per cell column of a bin
constexpr int kSwRegion = (kBin + kMaxKbWidth - 1) * (kBin + kMaxKbWidth - 1);
constexpr int kSwSmem = 212 * 1024;    // dynamic shared memory budget
constexpr int kSwMaxChunk = 512;

// Registers: a lane keeps w x UPL accumulators of two floats; at most 30 of them.
__host__ __device__ constexpr int max_upl(int W) { return 30 / W < 1 ? 1 : (30 / W > 8 ? 8 : 30 / W); }

__device__ __forceinline__ float2 zero_unit() { return make_float2(0.f, 0.f); }

// Per-candidate shared arrays of a chunk: weights [kc][2W] floats, sorted
// position and output index [kc] ints, start column [kc] bytes; then the staged
// alpha' rows [kc][qpmax] and inputs g_b(x) [kc][nbmax] (complex values).
__host__ __device__ constexpr size_t sw_meta_bytes(int kc, int W) {
  return ((size_t)kc * (2 * W * 4 + 4 + 4 + 1) + 15) / 16 * 16;
}

template <int W, int UPL>
__global__ void __launch_bounds__(kSwThreads, 1)
k_spread_sweep(const float2 *__restrict__ gin, float2 *__restrict__ grid,
               const WedgeDev *__restrict__ Wd, const int2 *__restrict__ bins,
               const int *__restrict__ cstart, const float2 *__restrict__ alpha,
               const uint2 *__restrict__ warps, const uint32_t *__restrict__ perm, long long NN,
               int B, KbDev kb, HornerDev hz, int kc, int chp, int qpmax, int nbmax,
               int *errw) {
  using U = float2;  // a unit: one complex term
  __shared__ int sRS[kSwRegion + 1];  // region-ordered first candidate of every start cell
  __shared__ int sGB[kSwRegion];      // sorted position of every start cell's first point
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // v of one chunk, then two buffers of the per-candidate data (weights, sorted
  // position, output index, start column; staged alpha' rows and inputs): the
  // next chunk is staged while this one is swept
  float2 *sV = reinterpret_cast<float2 *>(smem_raw);
  const size_t half = sw_meta_bytes(kc, W) + (size_t)kc * (qpmax + nbmax) * 8;
  auto bufp = [&](int buf) { return smem_raw + (size_t)kc * chp * 8 + buf * half; };

  const int tid = threadIdx.x, lane = tid & 31, cl = tid >> 5;
  const int2 it = bins[blockIdx.x];  // (wedge, bin)
  const int l = it.x;
  const int m1 = Wd[l].m1, m2 = Wd[l].m2, nb2 = Wd[l].nb2, qp = Wd[l].qp;
  const int r0 = (it.y / nb2) * kBin, c0 = (it.y % nb2) * kBin;
  const int H1 = min(kBin, m1 - r0), H2 = min(kBin, m2 - c0);
  const int RH = H1 + W - 1, RW = H2 + W - 1, RC = RH * RW;
  const int *cs = cstart + Wd[l].key_off;
  const int nch = B * qp;
  float2 *gw = grid + Wd[l].grid_unit * B;
  const float2 *al = alpha + Wd[l].alpha_off;
  const uint2 *ws = warps + (long long)l * NN;
  const uint32_t *pm = perm + (long long)l * NN;

  // Start cells (r0 - W + 1 + ri, c0 - W + 1 + rj) of the region, row-major:
  // their buckets, then an exclusive scan of the bucket sizes.
  for (int i = tid; i < RC; i += kSwThreads) {
    const int ri = i / RW, rj = i - ri * RW;
    const int s1 = imodp(r0 - (W - 1) + ri, m1), s2 = imodp(c0 - (W - 1) + rj, m2);
    const long long key = bin_key(s1, s2, nb2);
    const int beg = cs[key];
    sGB[i] = beg;
    sRS[i] = cs[key + 1] - beg;
  }
  __syncthreads();
  if (cl == 0) {
    const int per = (RC + 31) / 32;
    const int a = min(RC, lane * per), e = min(RC, a + per);
    int sum = 0;
    for (int i = a; i < e; ++i) sum += sRS[i];
    int inc = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(kFull, inc, off);
      if (lane >= off) inc += v;
    }
    int run = inc - sum;
    for (int i = a; i < e; ++i) {
      const int cnt = sRS[i];
      sRS[i] = run;
      run += cnt;
    }
    if (lane == 31) sRS[RC] = inc;
  }
  __syncthreads();
  const int total = sRS[RC];
  const int nchunks = max(1, (total + kc - 1) / kc);
  const FastDiv dqp = make_fastdiv((unsigned)qp);

  for (int ch0 = 0; ch0 < nch; ch0 += chp) {
    const int npc = min(chp, nch - ch0);  // channels of this pass
    const int nu = npc;                   // units of this pass
    const FastDiv dnpc = make_fastdiv((unsigned)npc);
    const int b_lo = ch0 / qp, nbp = (ch0 + npc - 1) / qp - b_lo + 1;  // inputs of the pass
    const int k = lane;  // this lane's first unit
    U acc[W][UPL];
#pragma unroll
    for (int a = 0; a < W; ++a)
#pragma unroll
      for (int j = 0; j < UPL; ++j) acc[a][j] = zero_unit();
    int i = 0;  // next start row of the sweep
    // Chunk kk into buffer kk & 1: start cells by binary search, KB weights, and
    // the copies of the candidates' alpha' rows and inputs, all in flight at once.
    auto stage = [&](int kk) {
      unsigned char *bp = bufp(kk & 1);
      float(*sWt)[2 * W] = reinterpret_cast<float(*)[2 * W]>(bp);
      int *sPos = reinterpret_cast<int *>(bp + (size_t)kc * 2 * W * 4);
      int *sX = sPos + kc;
      unsigned char *sCol = reinterpret_cast<unsigned char *>(sX + kc);
      float2 *sA = reinterpret_cast<float2 *>(bp + sw_meta_bytes(kc, W));
      float2 *sGi = sA + (size_t)kc * qpmax;
      const int c = kk * kc;
      const int np = max(0, min(kc, total - c));
      for (int t = tid; t < np; t += kSwThreads) {
        const int idx = c + t;
        int lo = 0, hi = RC - 1;  // the start cell holding candidate idx
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (sRS[mid] <= idx) lo = mid;
          else hi = mid - 1;
        }
        const int pos = sGB[lo] + (idx - sRS[lo]);
        const int ri = lo / RW, rj = lo - ri * RW;
        float wt[2 * W];
        const int2 sc = point_weights<float, W>(ws[pos], m1, m2, kb, hz, wt);
        const bool ok = sc.x == imodp(r0 - (W - 1) + ri, m1) && sc.y == imodp(c0 - (W - 1) + rj, m2);
        if (!ok) atomicOr(errw, 1);
#pragma unroll
        for (int a = 0; a < 2 * W; ++a) sWt[t][a] = ok ? wt[a] : 0.f;
        const int x = (int)pm[pos];
        sPos[t] = pos;
        sX[t] = x;
        sCol[t] = (unsigned char)rj;
        // stage the candidate's alpha' row and inputs: every copy in flight at once
        const float2 *arow = al + (long long)pos * qp;
        for (int u = 0; u < qp; u += 2) cp_async<16>(sA + t * qp + u, arow + u);
        for (int bb = 0; bb < nbp; ++bb)
          cp_async<8>(sGi + t * nbmax + bb, gin + (long long)(b_lo + bb) * NN + x);
      }
    };
    __syncthreads();  // the previous pass is done with every buffer
    stage(0);
    for (int ch = 0; ch < nchunks; ++ch) {
      const int c = ch * kc;
      const int np = max(0, min(kc, total - c));
      unsigned char *bp = bufp(ch & 1);
      const float(*sWt)[2 * W] = reinterpret_cast<const float(*)[2 * W]>(bp);
      const unsigned char *sCol = bp + (size_t)kc * 2 * W * 4 + 2 * (size_t)kc * 4;
      const float2 *sA = reinterpret_cast<const float2 *>(bp + sw_meta_bytes(kc, W));
      const float2 *sGi = sA + (size_t)kc * qpmax;
      cp_async_wait();
      __syncthreads();  // chunk ch is staged; the sweep of chunk ch - 1 is done with v
      // v[t][c] = conj(alpha'_tr(x_t)) g_b(x_t) for the pass's channels ch0 + c = b qp + tr
      for (int e = tid; e < np * npc; e += kSwThreads) {
        const int t = (int)fdiv((unsigned)e, dnpc), cc = ch0 + e - t * npc;
        const int b = (int)fdiv((unsigned)cc, dqp), tr = cc - b * qp;
        sV[e] = cmulc(sGi[t * nbmax + b - b_lo], sA[t * qp + tr]);
      }
      __syncthreads();  // v is complete
      if (ch + 1 < nchunks) stage(ch + 1);  // lands while this chunk is swept
      if (cl >= H2) continue;
      const U *sVu = reinterpret_cast<const U *>(sV);
      // sweep the start rows this chunk reaches
      while (i < RH) {
        const int rb = i * RW + cl;
        const int end = sRS[rb + W];
        const int lo = max(sRS[rb] - c, 0), hi = min(end - c, np);
        {
          for (int t = lo; t < hi; ++t) {
            const float *wr = sWt[t];
            const float w2 = wr[W + (cl + W - 1 - sCol[t])];
            float w1[W];
            if constexpr (W % 2 == 0) {  // rows of 2W floats are 16-byte aligned: vector loads
#pragma unroll
              for (int a = 0; a + 3 < W; a += 4) {
                const float4 q4 = *reinterpret_cast<const float4 *>(wr + a);
                w1[a] = q4.x; w1[a + 1] = q4.y; w1[a + 2] = q4.z; w1[a + 3] = q4.w;
              }
              if constexpr (W % 4 == 2) {
                const float2 q2 = *reinterpret_cast<const float2 *>(wr + W - 2);
                w1[W - 2] = q2.x; w1[W - 1] = q2.y;
              }
            } else {
#pragma unroll
              for (int a = 0; a < W; ++a) w1[a] = wr[a];
            }
            U v[UPL];
#pragma unroll
            for (int j = 0; j < UPL; ++j) {
              const int u = k + 32 * j;
              v[j] = u < nu ? sVu[t * nu + u] : zero_unit();
              uscale(v[j], w2);
            }
#pragma unroll
            for (int a = 0; a < W; ++a)
#pragma unroll
              for (int j = 0; j < UPL; ++j) ufma(acc[a][j], w1[a], v[j]);
          }
        }
        if (end > c + np) break;  // the start row continues in the next chunk
        // start row i is complete: cell row i - (W - 1) is final
        const int rl = i - (W - 1);
        if (rl >= 0) {
          U *dst = reinterpret_cast<U *>(gw + ((long long)(r0 + rl) * m2 + c0 + cl) * nch + ch0);
#pragma unroll
          for (int j = 0; j < UPL; ++j)
            if (k + 32 * j < nu) dst[k + 32 * j] = acc[0][j];
        }
#pragma unroll
        for (int a = 0; a < W - 1; ++a)
#pragma unroll
          for (int j = 0; j < UPL; ++j) acc[a][j] = acc[a + 1][j];
#pragma unroll
        for (int j = 0; j < UPL; ++j) acc[W - 1][j] = zero_unit();
        ++i;
      }
    }
  }
}

// One launch over every bin of every wedge.  A pass covers chp = 32 UPL channels;
// the chunk size kc fills the shared-memory budget.
template <int W, int UPL>
cudaError_t launch_sweep(const fio_plan_s *p, const void *g, void *grid, int B, cudaStream_t s,
                         const WorkRange &wr) {
  const long long NN = (long long)p->N * p->N;
  const int chp = 32 * UPL;
  int qpmax = 2;
  for (const WedgeDev &w : p->wedges) qpmax = std::max(qpmax, w.qp);
  const int nbmax = std::min(B, chp / 2 + 2);  // inputs one pass can touch (qp >= 2)
  const size_t per = 2 * ((size_t)2 * W * 4 + 4 + 4 + 1 + (size_t)(qpmax + nbmax) * 8) + (size_t)chp * 8;
  int kc = (int)std::min<size_t>(kSwMaxChunk, (kSwSmem - 128) / per) / 16 * 16;
  kc = std::max(kc, 16);
  const size_t smem = (size_t)kc * chp * 8 + 2 * (sw_meta_bytes(kc, W) + (size_t)kc * (qpmax + nbmax) * 8);
  cudaError_t e = cudaFuncSetAttribute(k_spread_sweep<W, UPL>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (wr.n_bins1 > 0)
    k_spread_sweep<W, UPL><<<wr.n_bins1, kSwThreads, smem, s>>>(
        (const float2 *)g, (float2 *)grid, wr.wedges, wr.bins1, p->d_cstart,
        (const float2 *)wr.alpha, p->d_warps, p->d_perm, NN, B, make_kbdev(p), p->horner, kc,
        chp, qpmax, nbmax, p->d_errword);
  return cudaGetLastError();
}

// UPL = ceil(channels / 32) single-term units per lane (up to the register
// limit; more channels take several passes).
template <int W>
cudaError_t sweep_w(const fio_plan_s *p, const void *g, void *grid, int B, cudaStream_t s,
                    const WorkRange &wr) {
  int qpmax = 2;
  for (const WedgeDev &w : p->wedges) qpmax = std::max(qpmax, w.qp);
  const int nchmax = B * qpmax;
  if (nchmax >= (1 << 20)) return cudaErrorInvalidValue;  // the channel index divisions need < 2^20
  constexpr int UM = max_upl(W);
  switch (std::min(UM, (nchmax + 31) / 32)) {
    case 1: return launch_sweep<W, 1>(p, g, grid, B, s, wr);
    case 2: return launch_sweep<W, std::min(UM, 2)>(p, g, grid, B, s, wr);
    case 3: return launch_sweep<W, std::min(UM, 3)>(p, g, grid, B, s, wr);
    case 4: return launch_sweep<W, std::min(UM, 4)>(p, g, grid, B, s, wr);
    case 5: return launch_sweep<W, std::min(UM, 5)>(p, g, grid, B, s, wr);
    case 6: return launch_sweep<W, std::min(UM, 6)>(p, g, grid, B, s, wr);
    case 7: return launch_sweep<W, std::min(UM, 7)>(p, g, grid, B, s, wr);
    default: return launch_sweep<W, std::min(UM, 8)>(p, g, grid, B, s, wr);
  }
}

}  // namespace

cudaError_t launch_spread_sweep(const fio_plan_s *p, const void *g, void *grid, int B,
                                cudaStream_t s, const WorkRange &wr) {
  switch (p->kb.w) {
    case 3: return sweep_w<3>(p, g, grid, B, s, wr);
    case 4: return sweep_w<4>(p, g, grid, B, s, wr);
    case 5: return sweep_w<5>(p, g, grid, B, s, wr);
    case 6: return sweep_w<6>(p, g, grid, B, s, wr);
    case 7: return sweep_w<7>(p, g, grid, B, s, wr);
    case 8: return sweep_w<8>(p, g, grid, B, s, wr);
    case 9: return sweep_w<9>(p, g, grid, B, s, wr);
    case 10: return sweep_w<10>(p, g, grid, B, s, wr);
    case 11: return sweep_w<11>(p, g, grid, B, s, wr);
    case 12: return sweep_w<12>(p, g, grid, B, s, wr);
  }
  return cudaErrorNotSupported;
}

}  // namespace fio
