// interp.cu -- S3 (type-2 interpolation with the gamma^x multiply and the sums
// over rank terms and wedges, Sec. 3.4 steps 3-4) and S4a (the type-1 spread of
// the adjoint, Sec. 3.5 steps 1-2) on 16 x 16 point tiles.
//
// A CTA owns one point tile and walks over every wedge.  For wedge l the tile's
// warped points y'_l(x) m fall in a small box of the NUFFT grid (the tile
// footprint, fixed by the plan), which is staged in shared memory cell-major:
// the rank terms of a cell are one contiguous run of 16-byte units (two
// complex64 terms, or one complex128).
//
// The interpolation is warp-cooperative: a group of lanes owns one point, one
// lane per unit, so the group's loads of a cell are one contiguous run (free of
// bank conflicts) and the warped windows of different points never collide in
// a lane.  Per-point KB weights are computed once per wedge into shared memory;
// the gamma^x multiply is folded in per lane and the sum over rank terms is a
// segmented shuffle reduction.  The spread is the mirror image: each group adds
// its point's weighted values to a shared footprint accumulator (distinct units
// per lane), which is then added to the grid with 16-byte vector atomics
// (neighbouring tiles' footprints overlap).
//
// Every point checks that its window lies inside the footprint; a violation is
// recorded in the plan's error word and the point is skipped.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "apply_common.cuh"
#include "fio_internal.h"

namespace fio {

namespace {

constexpr int kBG = 8;                 // inputs accumulated together per pass
constexpr int kSmemG = 48 * 1024;      // default footprint staging buffer
constexpr int kSmemGMax = 160 * 1024;  // largest staging buffer
constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------- tile footprints ---

__global__ void __launch_bounds__(256) k_tiles(const WedgeDev *__restrict__ Wd,
                                               const uint2 *__restrict__ warp, int N, int nt,
                                               int kbw, int4 *__restrict__ tiles,
                                               uint2 *__restrict__ warpt) {
  __shared__ int ref[2], lo[2], hi[2];
  const int nt2 = nt * nt;
  const int l = blockIdx.x / nt2, tile = blockIdx.x % nt2;
  const int I = tile / nt, J = tile % nt;
  const int tid = threadIdx.x;
  const long long NN = (long long)N * N;
  const WedgeDev w = Wd[l];
  const int n1 = I * kTile + tid / kTile, n2 = J * kTile + tid % kTile;
  const bool valid = n1 < N && n2 < N;
  float bdum;
  if (tid == 0) {
    const uint2 Y = warp[l * NN + (long long)(I * kTile) * N + J * kTile];
    ref[0] = kb_first<float>(Y.x, w.m1, kbw, &bdum);
    ref[1] = kb_first<float>(Y.y, w.m2, kbw, &bdum);
    lo[0] = lo[1] = 1 << 30;
    hi[0] = hi[1] = -(1 << 30);
  }
  __syncthreads();
  uint2 Y = make_uint2(0, 0);
  if (valid) {
    Y = warp[l * NN + (long long)n1 * N + n2];
    const int m[2] = {w.m1, w.m2};
    const int j[2] = {kb_first<float>(Y.x, w.m1, kbw, &bdum), kb_first<float>(Y.y, w.m2, kbw, &bdum)};
    for (int d = 0; d < 2; ++d) {
      // offset from the reference point, centred in [-m/2, m/2)
      const int o = imodp(j[d] - ref[d] + m[d] / 2, m[d]) - m[d] / 2;
      atomicMin(&lo[d], o);
      atomicMax(&hi[d], o);
    }
  }
  warpt[(long long)blockIdx.x * 256 + tid] = Y;  // tile order: [l][tile][point]
  __syncthreads();
  if (tid == 0) {
    const int m[2] = {w.m1, w.m2};
    int r[2], F[2];
    for (int d = 0; d < 2; ++d) {
      F[d] = hi[d] - lo[d] + kbw;
      if (2 * F[d] >= m[d]) {  // spread too wide to centre unambiguously: take every row
        r[d] = 0;
        F[d] = m[d] + kbw - 1;
      } else {
        r[d] = imodp(ref[d] + lo[d], m[d]);
      }
    }
    tiles[blockIdx.x] = make_int4(r[0], r[1], F[0], F[1]);
  }
}

// ------------------------------------------------------------- helpers -----

// KB weights of one axis: Horner polynomials (FP32) or the Bessel form (FP64).
template <typename T, int W>
__device__ __forceinline__ void kb_weights(T base, const KbDev &kb, const HornerDev &hz, T *wgt) {
  if constexpr (sizeof(T) == 4) {
    const float t = 2.0f * (base - (0.5f * W - 1.0f)) - 1.0f;
#pragma unroll
    for (int a = 0; a < W; ++a) wgt[a] = hz.c[hz.deg][a];
    for (int k = hz.deg - 1; k >= 0; --k) {
#pragma unroll
      for (int a = 0; a < W; ++a) wgt[a] = fmaf(wgt[a], t, hz.c[k][a]);
    }
  } else {
    const T tw = T(2) / T(W), beta = T(kb.beta), inv = T(kb.inv_i0b);
#pragma unroll
    for (int a = 0; a < W; ++a) wgt[a] = kb_phi(base - T(a), tw, beta, inv);
  }
}

// Phase 1 of both kernels: thread p computes its point's window offsets inside
// the tile footprint and its 2W weights into shared memory (off = -1: skip).
template <typename T, int W>
__device__ __forceinline__ void point_windows(const uint2 *__restrict__ warpt_tile, const WedgeDev &w,
                                              int4 tl, const KbDev &kb, const HornerDev &hz,
                                              bool valid, T (*sWt)[2 * W], int2 *sOff, int *errw) {
  const int p = threadIdx.x;
  int2 off = make_int2(-1, -1);
  if (valid) {
    T b1, b2;
    const uint2 Y = warpt_tile[p];
    const int j01 = kb_first<T>(Y.x, w.m1, W, &b1);
    const int j02 = kb_first<T>(Y.y, w.m2, W, &b2);
    T w1[W], w2[W];
    kb_weights<T, W>(b1, kb, hz, w1);
    kb_weights<T, W>(b2, kb, hz, w2);
#pragma unroll
    for (int a = 0; a < W; ++a) {
      sWt[p][a] = w1[a];
      sWt[p][W + a] = w2[a];
    }
    const int dr = imodp(j01 - tl.x, w.m1), dc = imodp(j02 - tl.y, w.m2);
    if (dr + W <= tl.z && dc + W <= tl.w) off = make_int2(dr, dc);
    else atomicOr(errw, 1);
  }
  sOff[p] = off;
}

// Copy `nu` units (starting at complex channel cbase) of every footprint cell into
// sG, cell-major: sG[cell * nu + k].  Warp wid copies rows wid, wid + 8, ...; a
// row's units are contiguous in global memory when the grid holds one input.
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
      rowdst[e] = reinterpret_cast<const uint4 *>(rowsrc + (long long)g2 * nch)[k];
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

// -------------------------------------------------------------------- S3 ---

template <typename T, int W>
__global__ void __launch_bounds__(256, 2)
k_interp_tile(const Cx<T> *__restrict__ grid, const WedgeDev *__restrict__ Wd,
              const int4 *__restrict__ tiles, const Cx<T> *__restrict__ alpha,
              const uint2 *__restrict__ warpt, Cx<T> *__restrict__ out, int N, int L, int B,
              int nt, KbDev kb, HornerDev hz, int smem_g, int bgmax, int *errw) {
  using C = Cx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint4 *sG = reinterpret_cast<uint4 *>(smem_raw);
  C(*sAcc)[256] = reinterpret_cast<C(*)[256]>(smem_raw + smem_g);
  T(*sWt)[2 * W] = reinterpret_cast<T(*)[2 * W]>(smem_raw + smem_g + bgmax * 256 * sizeof(C));
  int2 *sOff = reinterpret_cast<int2 *>(smem_raw + smem_g + bgmax * 256 * sizeof(C) +
                                        256 * 2 * W * sizeof(T));
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int tile = blockIdx.x;
  const int I = tile / nt, J = tile % nt;
  const long long NN = (long long)N * N;
  const int nt2 = nt * nt;
  const bool valid = I * kTile + tid / kTile < N && J * kTile + tid % kTile < N;
  constexpr int cpu = 16 / (int)sizeof(C);  // rank terms per 16-byte unit
  for (int b0 = 0; b0 < B; b0 += bgmax) {
    const int BG = min(bgmax, B - b0);
    for (int bb = 0; bb < BG; ++bb) sAcc[bb][tid] = C{0, 0};
    for (int l = 0; l < L; ++l) {
      const WedgeDev &w = Wd[l];
      const int qp = w.qp;
      const int4 tl = tiles[(long long)l * nt2 + tile];
      __syncthreads();  // previous wedge done with sWt, sOff, sG
      point_windows<T, W>(warpt + ((long long)l * nt2 + tile) * 256, w, tl, kb, hz, valid, sWt,
                          sOff, errw);
      const int nu = qp / cpu;
      const int cells = tl.z * tl.w;
      const int umax = smem_g / 16 / cells;     // units per cell that fit the buffer
      const bool direct = umax < 1;             // footprint too large: read global memory
      const int CHU = direct ? min(nu, 32) : min(min(nu, umax), 32);
      const long long nch = (long long)B * qp;
      const C *gw = grid + w.grid_unit * B;
      const C *al_tile = alpha + w.alpha_off + (long long)tile * 256 * qp;
      for (int bb = 0; bb < BG; ++bb) {
        for (int u0 = 0; u0 < nu; u0 += CHU) {
          const int nuc = min(CHU, nu - u0);
          const long long cbase = (long long)(b0 + bb) * qp + (long long)u0 * cpu;
          __syncthreads();
          if (!direct) stage_cells<T>(sG, gw, tl, w.m1, w.m2, nch, cbase, nuc);
          __syncthreads();
          const int gpw = 32 / nuc;               // point groups per warp
          const int g = lane / nuc, k = lane - g * nuc;
          const int stride = 8 * gpw;
          for (int r0 = 0; r0 < 256; r0 += stride) {
            const int p = r0 + wid * gpw + g;
            const bool act = g < gpw && p < 256;
            const int2 off = act ? sOff[p] : make_int2(-1, -1);
            T re = 0, im = 0;
            if (off.x >= 0) {
              const T *wp = sWt[p];
              const int t = (u0 + k) * cpu;
              if constexpr (sizeof(T) == 4) {
                float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
#pragma unroll
                for (int a1 = 0; a1 < W; ++a1) {
                  float rax = 0.f, ray = 0.f, rbx = 0.f, rby = 0.f;
                  const float w1 = wp[a1];
                  if (!direct) {
                    const float4 *pr =
                        reinterpret_cast<const float4 *>(sG) + ((off.x + a1) * tl.w + off.y) * nuc + k;
#pragma unroll
                    for (int a2 = 0; a2 < W; ++a2) {
                      const float4 gv = pr[a2 * nuc];
                      const float w2 = wp[W + a2];
                      rax = fmaf(w2, gv.x, rax);
                      ray = fmaf(w2, gv.y, ray);
                      rbx = fmaf(w2, gv.z, rbx);
                      rby = fmaf(w2, gv.w, rby);
                    }
                  } else {
                    const long long rowoff = (long long)((tl.x + off.x + a1) % w.m1) * w.m2;
                    for (int a2 = 0; a2 < W; ++a2) {
                      const float4 gv = *reinterpret_cast<const float4 *>(
                          gw + (rowoff + (tl.y + off.y + a2) % w.m2) * nch + cbase + 2 * k);
                      const float w2 = wp[W + a2];
                      rax = fmaf(w2, gv.x, rax);
                      ray = fmaf(w2, gv.y, ray);
                      rbx = fmaf(w2, gv.z, rbx);
                      rby = fmaf(w2, gv.w, rby);
                    }
                  }
                  ax = fmaf(w1, rax, ax);
                  ay = fmaf(w1, ray, ay);
                  bx = fmaf(w1, rbx, bx);
                  by = fmaf(w1, rby, by);
                }
                const float4 al = *reinterpret_cast<const float4 *>(al_tile + (long long)p * qp + t);
                re = al.x * ax - al.y * ay + al.z * bx - al.w * by;
                im = al.x * ay + al.y * ax + al.z * by + al.w * bx;
              } else {
                double ax = 0.0, ay = 0.0;
                for (int a1 = 0; a1 < W; ++a1) {
                  double rax = 0.0, ray = 0.0;
                  const double w1 = wp[a1];
                  const long long rowoff = direct ? (long long)((tl.x + off.x + a1) % w.m1) * w.m2 : 0;
#pragma unroll
                  for (int a2 = 0; a2 < W; ++a2) {
                    const double2 gv =
                        direct ? gw[(rowoff + (tl.y + off.y + a2) % w.m2) * nch + cbase + k]
                               : reinterpret_cast<const double2 *>(sG)[((off.x + a1) * tl.w + off.y + a2) * nuc + k];
                    const double w2 = wp[W + a2];
                    rax = fma(w2, gv.x, rax);
                    ray = fma(w2, gv.y, ray);
                  }
                  ax = fma(w1, rax, ax);
                  ay = fma(w1, ray, ay);
                }
                const C al = al_tile[(long long)p * qp + t];
                re = al.x * ax - al.y * ay;
                im = al.x * ay + al.y * ax;
              }
            }
            re = group_sum(re, k, nuc);
            im = group_sum(im, k, nuc);
            if (act && k == 0 && off.x >= 0) {
              sAcc[bb][p].x += re;
              sAcc[bb][p].y += im;
            }
          }
        }
      }
    }
    __syncthreads();
    {
      const int n1 = I * kTile + tid / 16, n2 = J * kTile + tid % 16;
      if (n1 < N && n2 < N)
        for (int bb = 0; bb < BG; ++bb)
          out[(long long)(b0 + bb) * NN + (long long)n1 * N + n2] = sAcc[bb][tid];
    }
  }
}

// ------------------------------------------------------------------- S4a ---

constexpr int kGrp = 8;             // rank terms per gather pass
constexpr int kMaxSortRows = 256;   // footprints with more rows use the unsorted loop

// Accumulate the contributions of point q (weight wt) to one cell for `ng` terms.
template <typename T, int NG>
__device__ __forceinline__ void gather_terms(Cx<T> *acc, const Cx<T> *pairs, int q, T wt) {
#pragma unroll
  for (int k = 0; k < NG; k += 2) {
    const Cx<T> *pp = pairs + ((k >> 1) * 256 + q) * 2;
    Cx<T> s0, s1;
    if constexpr (sizeof(T) == 4) {
      const float4 v4 = *reinterpret_cast<const float4 *>(pp);
      s0 = Cx<T>{v4.x, v4.y};
      s1 = Cx<T>{v4.z, v4.w};
    } else {
      s0 = pp[0];
      s1 = pp[1];
    }
    acc[k].x += wt * s0.x;
    acc[k].y += wt * s0.y;
    acc[k + 1].x += wt * s1.x;
    acc[k + 1].y += wt * s1.y;
  }
}

template <typename T, int W>
__global__ void __launch_bounds__(256, 2)
k_spread_tile(const Cx<T> *__restrict__ gin, Cx<T> *__restrict__ grid,
              const WedgeDev *__restrict__ Wd, const int4 *__restrict__ tiles,
              const Cx<T> *__restrict__ alpha, const uint2 *__restrict__ warpt, int N, int L,
              int B, int nt, KbDev kb, HornerDev hz, int bgmax, int *errw) {
  using C = Cx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C(*sIn)[256] = reinterpret_cast<C(*)[256]>(smem_raw);  // [bgmax]: inputs by point
  C *pairs = reinterpret_cast<C *>(smem_raw + bgmax * 256 * sizeof(C));  // conj(alpha) g, term pairs
  T(*sWt)[2 * W] = reinterpret_cast<T(*)[2 * W]>(smem_raw + (bgmax + kGrp) * 256 * sizeof(C));
  int2 *sOff = reinterpret_cast<int2 *>(smem_raw + (bgmax + kGrp) * 256 * sizeof(C) +
                                        256 * 2 * W * sizeof(T));
  int *sStart = reinterpret_cast<int *>(sOff + 256);      // bucket bounds by footprint row
  short *sSort = reinterpret_cast<short *>(sStart + kMaxSortRows + 1);  // points sorted by row
  const int tid = threadIdx.x;
  const int tile = blockIdx.x;
  const int I = tile / nt, J = tile % nt;
  const long long NN = (long long)N * N;
  const int nt2 = nt * nt;
  const bool valid = I * kTile + tid / kTile < N && J * kTile + tid % kTile < N;
  for (int b0 = 0; b0 < B; b0 += bgmax) {
    const int BG = min(bgmax, B - b0);
    __syncthreads();
    {
      const int n1 = I * kTile + tid / 16, n2 = J * kTile + tid % 16;
      for (int bb = 0; bb < BG; ++bb)
        sIn[bb][tid] = valid ? gin[(long long)(b0 + bb) * NN + (long long)n1 * N + n2] : C{0, 0};
    }
    for (int l = 0; l < L; ++l) {
      const WedgeDev &w = Wd[l];
      const int qp = w.qp;
      const int4 tl = tiles[(long long)l * nt2 + tile];
      const bool sorted = tl.z <= kMaxSortRows;
      __syncthreads();  // previous wedge done with sWt, sOff, sSort, pairs
      point_windows<T, W>(warpt + ((long long)l * nt2 + tile) * 256, w, tl, kb, hz, valid, sWt,
                          sOff, errw);
      const int dr = sOff[tid].x;  // own entry: no barrier needed
      if (sorted)
        for (int r = tid; r <= tl.z; r += 256) sStart[r] = 0;
      __syncthreads();
      if (sorted && dr >= 0) atomicAdd(&sStart[dr + 1], 1);
      __syncthreads();
      if (sorted && tid == 0)
        for (int r = 1; r <= tl.z; ++r) sStart[r] += sStart[r - 1];
      __syncthreads();
      if (sorted && dr >= 0) sSort[atomicAdd(&sStart[dr], 1)] = (short)tid;
      // after the scatter sStart[r] is the end of bucket r (bucket r-1 ends where r begins)
      const long long nch = (long long)B * qp;
      C *gw = grid + w.grid_unit * B;
      const C *al_pt = alpha + w.alpha_off + ((long long)tile * 256 + tid) * qp;
      const int cells = tl.z * tl.w;
      for (int bb = 0; bb < BG; ++bb) {
        for (int t0 = 0; t0 < qp; t0 += kGrp) {
          const int ng = min(kGrp, qp - t0);  // even
          __syncthreads();
          {
            const C g = sIn[bb][tid];
            const bool on = dr >= 0;
            for (int k = 0; k < ng; k += 2) {
              C a0, a1;
              if constexpr (sizeof(T) == 4) {
                const float4 v = *reinterpret_cast<const float4 *>(al_pt + t0 + k);
                a0 = C{v.x, v.y};
                a1 = C{v.z, v.w};
              } else {
                a0 = al_pt[t0 + k];
                a1 = al_pt[t0 + k + 1];
              }
              C *dst = pairs + ((k >> 1) * 256 + tid) * 2;
              dst[0] = on ? cmulc(g, a0) : C{0, 0};  // g conj(alpha_t)
              dst[1] = on ? cmulc(g, a1) : C{0, 0};
            }
          }
          __syncthreads();
          for (int cell = tid; cell < cells; cell += 256) {
            const int r = cell / tl.w, c = cell - r * tl.w;
            int beg = 0, end = 256;
            if (sorted) {
              const int rlo = r - W + 1;  // buckets rlo .. r hold the points covering row r
              beg = rlo > 0 ? sStart[rlo - 1] : 0;
              end = sStart[r];
            }
            C acc[kGrp];
#pragma unroll
            for (int k = 0; k < kGrp; ++k) acc[k] = C{0, 0};
            bool any = false;
            for (int it = beg; it < end; ++it) {
              const int q = sorted ? (int)sSort[it] : it;
              const int2 d = sOff[q];
              if (d.x < 0) continue;
              const unsigned u = (unsigned)(r - d.x), v = (unsigned)(c - d.y);
              if (u < (unsigned)W && v < (unsigned)W) {
                const T wt = sWt[q][u] * sWt[q][W + v];
                any = true;
                if (ng == kGrp) gather_terms<T, kGrp>(acc, pairs, q, wt);
                else
                  for (int k = 0; k < ng; k += 2) {
                    const C *pp = pairs + ((k >> 1) * 256 + q) * 2;
                    acc[k].x += wt * pp[0].x;
                    acc[k].y += wt * pp[0].y;
                    acc[k + 1].x += wt * pp[1].x;
                    acc[k + 1].y += wt * pp[1].y;
                  }
              }
            }
            if (any) {
              C *dst = gw + ((long long)((tl.x + r) % w.m1) * w.m2 + (tl.y + c) % w.m2) * nch +
                       (long long)(b0 + bb) * qp + t0;
#pragma unroll
              for (int k = 0; k < kGrp; k += 2)
                if (k < ng) {
                  if constexpr (sizeof(T) == 4) {
                    atomicAdd(reinterpret_cast<float4 *>(dst + k),
                              make_float4(acc[k].x, acc[k].y, acc[k + 1].x, acc[k + 1].y));
                  } else {
                    atomicAdd(&dst[k].x, acc[k].x);
                    atomicAdd(&dst[k].y, acc[k].y);
                    atomicAdd(&dst[k + 1].x, acc[k + 1].x);
                    atomicAdd(&dst[k + 1].y, acc[k + 1].y);
                  }
                }
            }
          }
        }
      }
    }
  }
}

// ------------------------------------------------------------- launchers ---

int smem_g_for(const fio_plan_s *p) {
  // room for the 99th-percentile footprint with two units per cell (larger ones
  // use fewer units per pass, or global memory), within [kSmemG, kSmemGMax]
  const long long need = 16LL * 2 * ((long long)p->foot_p99 + 1);
  return (int)std::min<long long>(kSmemGMax, std::max<long long>(kSmemG, (need + 15) / 16 * 16));
}

template <typename T, int W>
size_t tile_smem(const fio_plan_s *p, int bgmax) {
  return (size_t)smem_g_for(p) + (size_t)bgmax * 256 * sizeof(Cx<T>) + 256 * 2 * W * sizeof(T) +
         256 * sizeof(int2);
}

template <typename T, int W>
cudaError_t run_tile_kernels(const fio_plan_s *p, const void *in, void *grid, void *out, int B,
                             bool spread, cudaStream_t s) {
  using C = Cx<T>;
  const int nblk = p->ntile * p->ntile;
  const int smem_g = smem_g_for(p);
  const int bgmax = std::min(B, kBG);
  const size_t smem = tile_smem<T, W>(p, bgmax);
  cudaError_t e;
  if (spread) {
    const size_t ssm = (size_t)(bgmax + kGrp) * 256 * sizeof(C) + 256 * 2 * W * sizeof(T) +
                       256 * sizeof(int2) + (kMaxSortRows + 1) * sizeof(int) + 256 * sizeof(short);
    e = cudaFuncSetAttribute(k_spread_tile<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ssm);
    if (e != cudaSuccess) return e;
    k_spread_tile<T, W><<<nblk, 256, ssm, s>>>((const C *)in, (C *)grid, p->d_wedges, p->d_tiles,
                                               (const C *)p->d_alpha, p->d_warpt, p->N, p->L, B,
                                               p->ntile, make_kbdev(p), p->horner, bgmax,
                                               p->d_errword);
  } else {
    e = cudaFuncSetAttribute(k_interp_tile<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    k_interp_tile<T, W><<<nblk, 256, smem, s>>>((const C *)grid, p->d_wedges, p->d_tiles,
                                                (const C *)p->d_alpha, p->d_warpt, (C *)out, p->N,
                                                p->L, B, p->ntile, make_kbdev(p), p->horner,
                                                smem_g, bgmax, p->d_errword);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch_w(const fio_plan_s *p, const void *in, void *grid, void *out, int B,
                       bool spread, cudaStream_t s) {
  switch (p->kb.w) {
    case 3: return run_tile_kernels<T, 3>(p, in, grid, out, B, spread, s);
    case 4: return run_tile_kernels<T, 4>(p, in, grid, out, B, spread, s);
    case 5: return run_tile_kernels<T, 5>(p, in, grid, out, B, spread, s);
    case 6: return run_tile_kernels<T, 6>(p, in, grid, out, B, spread, s);
    case 7: return run_tile_kernels<T, 7>(p, in, grid, out, B, spread, s);
    case 8: return run_tile_kernels<T, 8>(p, in, grid, out, B, spread, s);
    case 9: return run_tile_kernels<T, 9>(p, in, grid, out, B, spread, s);
    case 10: return run_tile_kernels<T, 10>(p, in, grid, out, B, spread, s);
    case 11: return run_tile_kernels<T, 11>(p, in, grid, out, B, spread, s);
    case 12: return run_tile_kernels<T, 12>(p, in, grid, out, B, spread, s);
  }
  return cudaErrorNotSupported;
}

}  // namespace

cudaError_t build_tiles(fio_plan_s *p) {
  const int nt2 = p->ntile * p->ntile;
  k_tiles<<<p->L * nt2, 256>>>(p->d_wedges, p->d_warp, p->N, p->ntile, p->kb.w, p->d_tiles,
                               p->d_warpt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  std::vector<int4> t((size_t)p->L * nt2);
  e = cudaMemcpy(t.data(), p->d_tiles, sizeof(int4) * t.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  // padded plane sizes (16-byte units) of every footprint
  std::vector<int> planes;
  planes.reserve(t.size());
  double sum = 0;
  p->max_foot = 0;
  for (const int4 &v : t) {
    p->max_foot = std::max(p->max_foot, v.z * v.w);
    sum += (double)v.z * v.w;
    planes.push_back(v.z * v.w);
  }
  std::sort(planes.begin(), planes.end());
  p->foot_p99 = planes[std::min(planes.size() - 1, (size_t)(0.99 * planes.size()))];  // cells
  p->mean_foot = sum / (double)t.size();
  return cudaSuccess;
}

cudaError_t launch_interp(const fio_plan_s *p, const void *grid, void *out, int B,
                          cudaStream_t s) {
  if (p->precision == FIO_FP64) return dispatch_w<double>(p, nullptr, (void *)grid, out, B, false, s);
  return dispatch_w<float>(p, nullptr, (void *)grid, out, B, false, s);
}

cudaError_t launch_spread(const fio_plan_s *p, const void *g, void *grid, int B, cudaStream_t s) {
  if (p->precision == FIO_FP64) return dispatch_w<double>(p, g, grid, nullptr, B, true, s);
  return dispatch_w<float>(p, g, grid, nullptr, B, true, s);
}

}  // namespace fio
