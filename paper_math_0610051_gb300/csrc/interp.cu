// interp.cu -- S3 (type-2 interpolation with the gamma^x multiply and the sums
// over rank terms and wedges, Sec. 3.4 steps 3-4) and S4a (the type-1 spread of
// the adjoint, Sec. 3.5 steps 1-2), on bins of the NUFFT grid.
//
// The plan sorts every wedge's points by the grid cell where their KB window
// starts, bin by bin (kBin x kBin start cells).  The warped points of a wedge
// are a smooth but strongly sheared image of the x grid, so neighbouring x give
// scattered windows; neighbouring sorted points give overlapping ones.  The
// points of one bin touch only its (kBin + w - 1)^2 cell footprint.
//
// S3: a CTA takes a work item (wedge, bin, up to kItemPts sorted points),
// stages the bin's footprint in shared memory cell-major (the rank terms of a
// cell are one contiguous run of 16-byte units: two complex64 terms or one
// complex128), and interpolates warp-cooperatively: a group of lanes owns one
// point, one lane per unit, so a group's loads of a cell are one contiguous run.
// The gamma^x multiply is folded in per lane, the sum over rank terms is a
// segmented shuffle reduction, and the sum over wedges is a vector atomic add
// into the output (each output receives one add per wedge).
//
// S4a: a CTA owns the kBin x kBin cells of one bin and gathers, for each of
// them, the contributions of every point whose window covers it: the points
// whose start cell lies in the (kBin + w - 1)^2 region above and left of the
// bin, found through the plan's bucket table.  Every grid cell is written once,
// by its own bin, with no atomics and no clearing of the grid.
//
// A point whose window start disagrees with the bucket it was sorted into is
// recorded in the plan's error word and skipped.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "apply_common.cuh"
#include "bin_common.cuh"
#include "fio_internal.h"

namespace fio {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kInterpSmemG = 96 * 1024;   // footprint staging buffer of S3
constexpr int kSpreadSmem = 72 * 1024;    // dynamic shared memory budget of S4a
constexpr int kCand = 256;                // candidate points per S4a chunk
constexpr int kChunk = 192;               // points per S3 chunk (weights and alpha staged)
// S4a works on two horizontally adjacent bins at once (32 columns)
constexpr int kSpreadCols = 2 * kBin;
constexpr int kMaxRegion2 = (kBin + kMaxKbWidth - 1) * (kSpreadCols + kMaxKbWidth - 1);
constexpr int kSpreadMaxUnits = 10;  // units per S4a pass: 3 lane groups per warp, <= 11 warps

int host_mod(int a, int m) {
  const int r = a % m;
  return r < 0 ? r + m : r;
}

// ------------------------------------------------------------ point sort ---

__global__ void k_keys(const uint2 *__restrict__ warp_l, long long NN, WedgeDev w, int kbw,
                       uint32_t *__restrict__ keys) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= NN) return;
  const uint2 Y = warp_l[x];
  float b;
  const int s1 = imodp(kb_first<float>(Y.x, w.m1, kbw, &b), w.m1);
  const int s2 = imodp(kb_first<float>(Y.y, w.m2, kbw, &b), w.m2);
  keys[x] = (uint32_t)bin_key(s1, s2, w.nb2);
}

__global__ void k_gather_warp(const uint2 *__restrict__ warp_l, const uint32_t *__restrict__ perm_l,
                              long long NN, uint2 *__restrict__ out) {
  const long long pos = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos < NN) out[pos] = warp_l[perm_l[pos]];
}

// ------------------------------------------------------------- helpers -----

// Start copying `nu` units (starting at complex channel cbase) of every footprint
// cell into sG, cell-major: sG[cell * nu + k] (asynchronous: cp_async_wait and a
// barrier complete it).  Warp wid copies rows wid, wid + 8, ...; a row's units
// are contiguous in global memory when the grid holds one input.
template <typename T>
__device__ __forceinline__ void stage_cells(uint4 *sG, const Cx<T> *gw, int4 tl, int m1, int m2,
                                            long long nch, long long cbase, int nu) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sf2 = 32 / nu, sk = 32 - sf2 * nu;
  for (int f1 = wid; f1 < tl.z; f1 += 8) {
    int g1 = tl.x + f1;
    while (g1 >= m1) g1 -= m1;
    const Cx<T> *rowsrc = gw + (long long)g1 * m2 * nch + cbase;
    uint4 *rowdst = sG + f1 * tl.w * nu;
    int f2 = lane / nu, k = lane - (lane / nu) * nu;
    for (int e = lane; e < tl.w * nu; e += 32) {
      int g2 = tl.y + f2;
      while (g2 >= m2) g2 -= m2;
      cp_async<16>(&rowdst[e], reinterpret_cast<const uint4 *>(rowsrc + (long long)g2 * nch) + k);
      f2 += sf2;
      k += sk;
      if (k >= nu) {
        k -= nu;
        ++f2;
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ T group_sum(T v, int k, int nu) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const T o = __shfl_down_sync(kFull, v, off);
    if (k + off < nu) v += o;
  }
  return v;
}

__device__ __forceinline__ void add_out(float2 *o, float re, float im) {
  atomicAdd(o, make_float2(re, im));
}
__device__ __forceinline__ void add_out(double2 *o, double re, double im) {
  atomicAdd(&o->x, re);
  atomicAdd(&o->y, im);
}

// -------------------------------------------------------------------- S3 ---

// Points that share a window start are interpolated together: a lane group
// takes a task of up to kRun such points, loads every footprint unit of their
// common window once and applies it to each of them.
template <typename T> struct RunLen { static constexpr int value = sizeof(T) == 4 ? 4 : 2; };

template <typename T, int W>
__global__ void __launch_bounds__(256, 2)
k_interp_bin(const Cx<T> *__restrict__ grid, const WedgeDev *__restrict__ Wd,
             const int4 *__restrict__ items, const Cx<T> *__restrict__ alpha,
             const uint2 *__restrict__ warps, const uint32_t *__restrict__ perm,
             Cx<T> *__restrict__ out, long long NN, int B, KbDev kb, HornerDev hz, int smem_g,
             int *errw) {
  using C = Cx<T>;
  using U = typename UnitT<T>::type;
  constexpr int kRun = RunLen<T>::value;
  __shared__ int sKey[kChunk];   // window start (dr kBin + dc) of each point, -1: skip
  __shared__ int sTask[kChunk];  // tasks: first point | count << 16
  __shared__ uint32_t sPm[kChunk];  // output index x of each point
  __shared__ int sNT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  U *sG = reinterpret_cast<U *>(smem_raw);
  T(*sWt)[2 * W] = reinterpret_cast<T(*)[2 * W]>(smem_raw + smem_g);
  U *sAl = reinterpret_cast<U *>(smem_raw + smem_g + kChunk * 2 * W * sizeof(T));  // alpha, one pass
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int4 it = items[blockIdx.x];
  const int l = it.x;
  const int m1 = Wd[l].m1, m2 = Wd[l].m2, nb2 = Wd[l].nb2, qp = Wd[l].qp;
  constexpr int cpu = 16 / (int)sizeof(C);  // rank terms per 16-byte unit
  const int nu = qp / cpu;
  const int r0 = (it.y / nb2) * kBin, c0 = (it.y % nb2) * kBin;
  const int H1 = min(kBin, m1 - r0), H2 = min(kBin, m2 - c0);
  const int4 tl = make_int4(r0, c0, H1 + W - 1, H2 + W - 1);
  // units per pass: the launcher's figure for the largest footprint, so that the
  // alpha buffer (kChunk x CHU units) is never overrun, even in a smaller edge bin
  const int CHU = min(min(nu, 32), smem_g / 16 / ((kBin + W - 1) * (kBin + W - 1)));
  const long long nch = (long long)B * qp;
  const C *gw = grid + Wd[l].grid_unit * B;
  const C *al = alpha + Wd[l].alpha_off;
  const uint2 *ws = warps + (long long)l * NN;
  const uint32_t *pm = perm + (long long)l * NN;
  for (int b = 0; b < B; ++b) {
    for (int u0 = 0; u0 < nu; u0 += CHU) {
      const int nuc = min(CHU, nu - u0);
      const long long cbase = (long long)b * qp + (long long)u0 * cpu;
      __syncthreads();  // the previous pass is done with sG, sWt, sKey, sTask
      stage_cells<T>(reinterpret_cast<uint4 *>(sG), gw, tl, m1, m2, nch, cbase, nuc);
      const int gpw = 32 / nuc;  // lane groups per warp
      const int g = lane / nuc, k = lane - g * nuc;
      const int ngr = 8 * gpw;
      for (int c = it.z; c < it.w; c += kChunk) {
        const int np = min(kChunk, it.w - c);
        if (c != it.z) __syncthreads();  // the previous chunk is done with sWt, sAl, sKey, sTask
        if (tid == 0) sNT = 0;
        // units u0 .. u0 + nuc of the chunk's alpha rows (one contiguous run when
        // nuc = nu): sAl[p * nuc + kk]
        {
          const U *src = reinterpret_cast<const U *>(al + (long long)c * qp) + u0;
          const FastDiv dnu = make_fastdiv((unsigned)nuc);
          for (int e = tid; e < np * nuc; e += 256) {
            const int pt = (int)fdiv((unsigned)e, dnu), kk = e - pt * nuc;
            cp_async<16>(sAl + e, src + pt * nu + kk);
          }
        }
        if (tid < np) {  // overlaps the copies in flight
          int key = -1;
          sPm[tid] = pm[c + tid];
          const int2 sc = point_weights<T, W>(ws[c + tid], m1, m2, kb, hz, sWt[tid]);
          const int dr = sc.x - r0, dc = sc.y - c0;
          if (dr >= 0 && dr < H1 && dc >= 0 && dc < H2) key = dr * kBin + dc;
          else atomicOr(errw, 1);
          sKey[tid] = key;
        }
        cp_async_wait();
        __syncthreads();  // footprint and alpha staged, windows ready
        if (tid < np) {   // runs of equal window start, cut into tasks of <= kRun points
          const int key = sKey[tid];
          if (key >= 0 && (tid == 0 || sKey[tid - 1] != key)) {
            int len = 1;
            while (tid + len < np && sKey[tid + len] == key) ++len;
            for (int s0 = 0; s0 < len; s0 += kRun)
              sTask[atomicAdd(&sNT, 1)] = (tid + s0) | (min(kRun, len - s0) << 16);
          }
        }
        __syncthreads();
        const int ntask = sNT;
        for (int q0 = 0; q0 < ntask; q0 += ngr) {  // uniform per warp: shuffles below
          const int task = q0 + wid * gpw + g;
          const bool act = g < gpw && task < ntask;
          const int tk = act ? sTask[task] : 0;
          const int p0 = tk & 0xffff, cnt = act ? tk >> 16 : 0;
          const int key = act ? sKey[p0] : 0;
          const int dr = key / kBin, dc = key - dr * kBin;
          T w2[kRun][W];
#pragma unroll
          for (int r = 0; r < kRun; ++r)
#pragma unroll
            for (int a = 0; a < W; ++a) w2[r][a] = r < cnt ? sWt[p0 + r][W + a] : T(0);
          U acc[kRun];
#pragma unroll
          for (int r = 0; r < kRun; ++r) acc[r] = uzero<U>();
          if (act) {
#pragma unroll
            for (int a1 = 0; a1 < W; ++a1) {
              const U *pr = sG + ((dr + a1) * tl.w + dc) * nuc + k;
              U rp[kRun];
#pragma unroll
              for (int r = 0; r < kRun; ++r) rp[r] = uzero<U>();
#pragma unroll
              for (int a2 = 0; a2 < W; ++a2) {
                const U gv = pr[a2 * nuc];
#pragma unroll
                for (int r = 0; r < kRun; ++r) ufma(rp[r], w2[r][a2], gv);
              }
#pragma unroll
              for (int r = 0; r < kRun; ++r) ufma4(acc[r], r < cnt ? sWt[p0 + r][a1] : T(0), rp[r]);
            }
          }
#pragma unroll
          for (int r = 0; r < kRun; ++r) {
            T re = 0, im = 0;
            if (r < cnt) {
              const U a = sAl[(p0 + r) * nuc + k];
              if constexpr (sizeof(T) == 4) {
                re = a.x * acc[r].x - a.y * acc[r].y + a.z * acc[r].z - a.w * acc[r].w;
                im = a.x * acc[r].y + a.y * acc[r].x + a.z * acc[r].w + a.w * acc[r].z;
              } else {
                re = a.x * acc[r].x - a.y * acc[r].y;
                im = a.x * acc[r].y + a.y * acc[r].x;
              }
            }
            re = group_sum(re, k, nuc);
            im = group_sum(im, k, nuc);
            if (k == 0 && r < cnt) add_out(out + (long long)b * NN + sPm[p0 + r], re, im);
          }
        }
      }
    }
  }
}

// ------------------------------------------------------------------- S4a ---

// The spread sweeps down the columns of a pair of adjacent bins (16 rows, up to
// 32 columns).  A lane group (one lane per
// 16-byte unit) owns cell column cl and walks the region's start rows in order,
// keeping the w cell rows that a start row can still reach in registers:
// acc[a1] is cell row i - (w - 1) + a1 while start row i is processed.  A point
// of start row i and start column rj within w - 1 of the column adds
// w1[a1] (w2[a2] conj(alpha) g) to acc[a1] for every a1.  After the row, acc[0]
// is complete (no later start row reaches it): it is written out, and the
// window slides down.  Candidates come in chunks of kCand in region order; a
// start row may continue in the next chunk, so the sweep state stays in
// registers across chunks.
template <typename T, int W>
__global__ void __launch_bounds__(384, 2)
k_spread_bin(const Cx<T> *__restrict__ gin, Cx<T> *__restrict__ grid,
             const WedgeDev *__restrict__ Wd, const int2 *__restrict__ bins,
             const int *__restrict__ cstart, const Cx<T> *__restrict__ alpha,
             const uint2 *__restrict__ warps, const uint32_t *__restrict__ perm, long long NN,
             int B, KbDev kb, HornerDev hz, int chu, int *errw) {
  using C = Cx<T>;
  using U = typename UnitT<T>::type;
  __shared__ int sRS[kMaxRegion2 + 1];  // region-ordered first candidate of every start cell
  __shared__ int sGB[kMaxRegion2];      // sorted position of every start cell's first point
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T(*sWt)[2 * W] = reinterpret_cast<T(*)[2 * W]>(smem_raw);  // w1 then w2 of each candidate
  C *sIn = reinterpret_cast<C *>(smem_raw + kCand * 2 * W * sizeof(T));
  int *sPos = reinterpret_cast<int *>(sIn + kCand);
  unsigned char *sCol = reinterpret_cast<unsigned char *>(sPos + kCand);
  U *sV = reinterpret_cast<U *>(
      smem_raw + ((kCand * (2 * W * sizeof(T) + sizeof(C) + sizeof(int) + 1) + 15) / 16 * 16));
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nth = blockDim.x;
  const int2 it = bins[blockIdx.x];  // (wedge, first bin of a pair in one bin row)
  const int l = it.x;
  const int m1 = Wd[l].m1, m2 = Wd[l].m2, nb2 = Wd[l].nb2, qp = Wd[l].qp;
  constexpr int cpu = 16 / (int)sizeof(C);
  const int nu = qp / cpu;
  const int r0 = (it.y / nb2) * kBin, c0 = (it.y % nb2) * kBin;
  const int H1 = min(kBin, m1 - r0), H2 = min(kSpreadCols, m2 - c0);
  const int RH = H1 + W - 1, RW = H2 + W - 1, RC = RH * RW;
  const int *cs = cstart + Wd[l].key_off;
  const long long nch = (long long)B * qp;
  C *gw = grid + Wd[l].grid_unit * B;
  const C *al = alpha + Wd[l].alpha_off;
  const uint2 *ws = warps + (long long)l * NN;
  const uint32_t *pm = perm + (long long)l * NN;

  // Start cells (r0 - W + 1 + ri, c0 - W + 1 + rj) of the region, row-major:
  // their buckets, then an exclusive scan of the bucket sizes.
  for (int i = tid; i < RC; i += nth) {
    const int ri = i / RW, rj = i - ri * RW;
    const int s1 = imodp(r0 - (W - 1) + ri, m1), s2 = imodp(c0 - (W - 1) + rj, m2);
    const long long key = bin_key(s1, s2, nb2);
    const int beg = cs[key];
    sGB[i] = beg;
    sRS[i] = cs[key + 1] - beg;
  }
  __syncthreads();
  if (wid == 0) {
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
  const int nchunks = max(1, (total + kCand - 1) / kCand);

  for (int b = 0; b < B; ++b) {
    for (int u0 = 0; u0 < nu; u0 += chu) {
      const int nuc = min(chu, nu - u0);
      const int gpw = 32 / nuc, g = lane / nuc, k = lane - g * nuc;
      const int cl = wid * gpw + g;  // this group's cell column
      const bool owner = g < gpw && cl < H2;
      U acc[W];
#pragma unroll
      for (int a = 0; a < W; ++a) acc[a] = uzero<U>();
      int i = 0;  // next start row of the sweep
      for (int ch = 0; ch < nchunks; ++ch) {
        const int c = ch * kCand;
        const int np = max(0, min(kCand, total - c));
        __syncthreads();  // the previous chunk is done with the candidate arrays
        for (int t = tid; t < np; t += nth) {
          const int idx = c + t;
          int lo = 0, hi = RC - 1;  // the start cell holding candidate idx
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sRS[mid] <= idx) lo = mid;
            else hi = mid - 1;
          }
          const int pos = sGB[lo] + (idx - sRS[lo]);
          const int ri = lo / RW, rj = lo - ri * RW;
          T wt[2 * W];
          const int2 sc = point_weights<T, W>(ws[pos], m1, m2, kb, hz, wt);
          const bool ok = sc.x == imodp(r0 - (W - 1) + ri, m1) && sc.y == imodp(c0 - (W - 1) + rj, m2);
          if (!ok) atomicOr(errw, 1);
#pragma unroll
          for (int a = 0; a < 2 * W; ++a) sWt[t][a] = ok ? wt[a] : T(0);
          sPos[t] = pos;
          sCol[t] = (unsigned char)rj;
          sIn[t] = gin[(long long)b * NN + pm[pos]];
        }
        __syncthreads();
        // conj(alpha_t) g for units u0 .. u0 + nuc of every candidate: alpha is
        // copied asynchronously into sV, then multiplied in place by the thread
        // that copied it
        {
          const FastDiv dnu = make_fastdiv((unsigned)nuc);
          for (int e = tid; e < np * nuc; e += nth) {
            const int t = (int)fdiv((unsigned)e, dnu), kk = e - t * nuc;
            cp_async<16>(sV + e, al + (long long)sPos[t] * qp + (u0 + kk) * cpu);
          }
          cp_async_wait();
          for (int e = tid; e < np * nuc; e += nth) {
            const C gv = sIn[(int)fdiv((unsigned)e, dnu)];
            if constexpr (sizeof(T) == 4) {
              const float4 a = reinterpret_cast<const float4 *>(sV)[e];
              const C v0 = cmulc(gv, C{a.x, a.y}), v1 = cmulc(gv, C{a.z, a.w});
              reinterpret_cast<float4 *>(sV)[e] = make_float4(v0.x, v0.y, v1.x, v1.y);
            } else {
              double2 *v = reinterpret_cast<double2 *>(sV) + e;
              *v = cmulc(gv, *v);
            }
          }
        }
        __syncthreads();
        if (!owner) continue;
        // sweep the start rows this chunk reaches
        while (i < RH) {
          const int rb = i * RW + cl;
          const int end = sRS[rb + W];
          const int lo = max(sRS[rb] - c, 0), hi = min(end - c, np);
#pragma unroll 2
          for (int t = lo; t < hi; ++t) {
            const T *wr = sWt[t];
            const T w2 = wr[W + (cl + W - 1 - sCol[t])];
            U v = sV[t * nuc + k];
            uscale(v, w2);
#pragma unroll
            for (int a = 0; a < W; ++a) ufma(acc[a], wr[a], v);
          }
          if (end > c + np) break;  // the start row continues in the next chunk
          // start row i is complete: cell row i - (W - 1) is final
          const int rl = i - (W - 1);
          if (rl >= 0)
            *reinterpret_cast<U *>(gw + ((long long)(r0 + rl) * m2 + c0 + cl) * nch +
                                   (long long)b * qp + (long long)(u0 + k) * cpu) = acc[0];
#pragma unroll
          for (int a = 0; a < W - 1; ++a) acc[a] = acc[a + 1];
          acc[W - 1] = uzero<U>();
          ++i;
        }
      }
    }
  }
}

// ------------------------------------------------------------- launchers ---

template <typename T>
int max_units(const fio_plan_s *p) {
  int nu = 1;
  for (const WedgeDev &w : p->wedges) nu = std::max(nu, w.qp * (int)sizeof(T) / 8);
  return nu;  // 16-byte units per cell: qp / 2 complex64 terms or qp complex128 terms
}

template <typename T, int W>
cudaError_t run_bin_kernels(const fio_plan_s *p, const void *in, void *grid, void *out, int B,
                            bool spread, cudaStream_t s, const WorkRange &wr) {
  using C = Cx<T>;
  const long long NN = (long long)p->N * p->N;
  const int numax = std::min(32, max_units<T>(p));
  cudaError_t e;
  if (spread) {
    const size_t fixed =
        (kCand * (2 * W * sizeof(T) + sizeof(C) + sizeof(int) + 1) + 15) / 16 * 16;
    const int chu = std::max(1, std::min(std::min(numax, kSpreadMaxUnits),
                                         (int)((kSpreadSmem - fixed) / ((size_t)kCand * 16))));
    const size_t smem = fixed + (size_t)kCand * 16 * chu;
    // enough lane groups of chu lanes for the columns of a bin pair
    const int gpw = 32 / chu;
    const int threads = 32 * ((kSpreadCols + gpw - 1) / gpw);
    e = cudaFuncSetAttribute(k_spread_bin<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    if (wr.n_bins > 0)
      k_spread_bin<T, W><<<wr.n_bins, threads, smem, s>>>(
          (const C *)in, (C *)grid, wr.wedges, wr.bins, p->d_cstart, (const C *)wr.alpha,
          p->d_warps, p->d_perm, NN, B, make_kbdev(p), p->horner, chu, p->d_errword);
  } else {
    if (wr.clear) e = cudaMemsetAsync(out, 0, sizeof(C) * (size_t)NN * B, s);
    else e = cudaSuccess;
    if (e != cudaSuccess) return e;
    const int cells = (kBin + W - 1) * (kBin + W - 1);
    const int chu = std::max(1, std::min(numax, kInterpSmemG / (16 * cells)));
    const int smem_g = chu * 16 * cells;
    const size_t smem = (size_t)smem_g + kChunk * 2 * W * sizeof(T) + (size_t)kChunk * chu * 16;
    e = cudaFuncSetAttribute(k_interp_bin<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    if (wr.n_items > 0)
      k_interp_bin<T, W><<<wr.n_items, 256, smem, s>>>(
          (const C *)grid, wr.wedges, wr.items, (const C *)wr.alpha, p->d_warps, p->d_perm,
          (C *)out, NN, B, make_kbdev(p), p->horner, smem_g, p->d_errword);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch_w(const fio_plan_s *p, const void *in, void *grid, void *out, int B,
                       bool spread, cudaStream_t s, const WorkRange &wr) {
  switch (p->kb.w) {
    case 3: return run_bin_kernels<T, 3>(p, in, grid, out, B, spread, s, wr);
    case 4: return run_bin_kernels<T, 4>(p, in, grid, out, B, spread, s, wr);
    case 5: return run_bin_kernels<T, 5>(p, in, grid, out, B, spread, s, wr);
    case 6: return run_bin_kernels<T, 6>(p, in, grid, out, B, spread, s, wr);
    case 7: return run_bin_kernels<T, 7>(p, in, grid, out, B, spread, s, wr);
    case 8: return run_bin_kernels<T, 8>(p, in, grid, out, B, spread, s, wr);
    case 9: return run_bin_kernels<T, 9>(p, in, grid, out, B, spread, s, wr);
    case 10: return run_bin_kernels<T, 10>(p, in, grid, out, B, spread, s, wr);
    case 11: return run_bin_kernels<T, 11>(p, in, grid, out, B, spread, s, wr);
    case 12: return run_bin_kernels<T, 12>(p, in, grid, out, B, spread, s, wr);
  }
  return cudaErrorNotSupported;
}

}  // namespace

cudaError_t sort_wedge_points(fio_plan_s *p, int l, std::vector<int> &cs) {
  const WedgeDev &w = p->wedges[l];
  const long long NN = (long long)p->N * p->N;
  const long long nkeys = (long long)w.nb1 * w.nb2 * kBin * kBin;
  uint32_t *d_keys = nullptr;
  cudaError_t e = cudaMalloc(&d_keys, sizeof(uint32_t) * NN);
  if (e != cudaSuccess) return e;
  k_keys<<<(unsigned)((NN + 255) / 256), 256>>>(p->d_warp + l * NN, NN, w, p->kb.w, d_keys);
  std::vector<uint32_t> keys((size_t)NN);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpy(keys.data(), d_keys, sizeof(uint32_t) * NN, cudaMemcpyDeviceToHost);
  cudaFree(d_keys);
  if (e != cudaSuccess) return e;
  // stable counting sort: equal keys keep increasing x
  cs.assign((size_t)nkeys + 1, 0);
  for (long long x = 0; x < NN; ++x) ++cs[keys[x] + 1];
  for (long long k = 0; k < nkeys; ++k) cs[k + 1] += cs[k];
  std::vector<uint32_t> perm((size_t)NN);
  std::vector<int> next(cs.begin(), cs.end() - 1);
  for (long long x = 0; x < NN; ++x) perm[next[keys[x]]++] = (uint32_t)x;
  e = cudaMemcpy(p->d_perm + l * NN, perm.data(), sizeof(uint32_t) * NN, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(p->d_cstart + w.key_off, cs.data(), sizeof(int) * cs.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  k_gather_warp<<<(unsigned)((NN + 255) / 256), 256>>>(p->d_warp + l * NN, p->d_perm + l * NN, NN,
                                                       p->d_warps + l * NN);
  return cudaGetLastError();
}

cudaError_t build_work_lists(fio_plan_s *p, const std::vector<std::vector<int>> &cstart) {
  std::vector<int4> items;
  std::vector<int2> bins, bins1;
  const int W = p->kb.w;
  long long nonempty = 0, total = 0;
  int maxb = 0;
  long long maxc = 0;
  p->item_off.assign(p->L + 1, 0);
  p->bin_off.assign(p->L + 1, 0);
  p->bin1_off.assign(p->L + 1, 0);
  for (int l = 0; l < p->L; ++l) {
    const WedgeDev &w = p->wedges[l];
    const std::vector<int> &cs = cstart[l];
    p->item_off[l] = (int)items.size();
    p->bin_off[l] = (int)bins.size();
    p->bin1_off[l] = (int)bins1.size();
    for (int bin = 0; bin < w.nb1 * w.nb2; ++bin) {
      const int beg = cs[(size_t)bin * kBin * kBin], end = cs[(size_t)(bin + 1) * kBin * kBin];
      const int ipts = item_points(W);
      for (int c = beg; c < end; c += ipts) items.push_back(make_int4(l, bin, c, std::min(end, c + ipts)));
      if ((bin % w.nb2) % 2 == 0) bins.push_back(make_int2(l, bin));  // first bin of a pair
      bins1.push_back(make_int2(l, bin));
      if (end > beg) {
        ++nonempty;
        total += end - beg;
      }
      maxb = std::max(maxb, end - beg);
      if ((bin % w.nb2) % 2 != 0) continue;  // spread candidates: per bin pair
      const int r0 = (bin / w.nb2) * kBin, c0 = (bin % w.nb2) * kBin;
      const int RH = std::min(kBin, w.m1 - r0) + W - 1, RW = std::min(kSpreadCols, w.m2 - c0) + W - 1;
      long long cand = 0;
      for (int i = 0; i < RH; ++i) {
        const int s1 = host_mod(r0 - (W - 1) + i, w.m1);
        for (int j = 0; j < RW; ++j) {
          const long long k = bin_key(s1, host_mod(c0 - (W - 1) + j, w.m2), w.nb2);
          cand += cs[k + 1] - cs[k];
        }
      }
      maxc = std::max(maxc, cand);
    }
  }
  p->n_items = (int)items.size();
  p->n_bins = (int)bins.size();
  p->n_bins1 = (int)bins1.size();
  p->item_off[p->L] = p->n_items;
  p->bin_off[p->L] = p->n_bins;
  p->bin1_off[p->L] = p->n_bins1;
  p->max_bin_pts = maxb;
  p->mean_bin_pts = nonempty ? (double)total / nonempty : 0.0;
  p->max_cand = (int)maxc;
  cudaError_t e = cudaMalloc(&p->d_items, sizeof(int4) * std::max<size_t>(1, items.size()));
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&p->d_bins, sizeof(int2) * std::max<size_t>(1, bins.size()));
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&p->d_bins1, sizeof(int2) * std::max<size_t>(1, bins1.size()));
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(p->d_bins1, bins1.data(), sizeof(int2) * bins1.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  if (!items.empty())
    e = cudaMemcpy(p->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(p->d_bins, bins.data(), sizeof(int2) * bins.size(), cudaMemcpyHostToDevice);
}

WorkRange full_range(const fio_plan_s *p) {
  return WorkRange{p->d_wedges, p->d_alpha, p->d_items, p->n_items, p->d_bins, p->n_bins,
                   p->d_bins1, p->n_bins1, true};
}

WorkRange group_range(const fio_plan_s *p, int g, bool clear) {
  const int l0 = p->grp_first[g], l1 = p->grp_first[g + 1];
  const int i0 = p->item_off[l0], b0 = p->bin_off[l0], c0 = p->bin1_off[l0];
  return WorkRange{p->d_wedges_rc, p->d_alpha, p->d_items + i0, p->item_off[l1] - i0,
                   p->d_bins + b0, p->bin_off[l1] - b0, p->d_bins1 + c0, p->bin1_off[l1] - c0,
                   clear};
}

cudaError_t launch_interp(const fio_plan_s *p, const void *grid, void *out, int B,
                          cudaStream_t s, const WorkRange &wr) {
  if (p->precision == FIO_FP64)
    return dispatch_w<double>(p, nullptr, (void *)grid, out, B, false, s, wr);
  return launch_interp_tasks(p, grid, out, B, s, wr);
}

cudaError_t launch_spread(const fio_plan_s *p, const void *g, void *grid, int B, cudaStream_t s,
                          const WorkRange &wr) {
  if (p->precision == FIO_FP64) return dispatch_w<double>(p, g, grid, nullptr, B, true, s, wr);
  // one lane per channel pays when a cell holds more than 32 channels (several
  // inputs); a single input takes the bin-pair kernel, whose lane groups own a
  // column each
  int qpmax = 2;
  for (const WedgeDev &w : p->wedges) qpmax = std::max(qpmax, w.qp);
  if (B * qpmax <= 32) return dispatch_w<float>(p, g, grid, nullptr, B, true, s, wr);
  return launch_spread_sweep(p, g, grid, B, s, wr);
}

}  // namespace fio
