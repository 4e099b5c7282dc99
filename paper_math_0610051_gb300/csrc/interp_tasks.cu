// interp_tasks.cu -- S3 of the mixed-precision forward apply (Sec. 3.4 steps
// 3-4): KB interpolation of every grid G_{l t} at the warped points, the
// gamma^x multiply (alpha'), and the sums over rank terms and wedges.
//
// A CTA takes a work item: one bin (kBin x kBin window-start cells) of one wedge
// and up to item_points(w) of its sorted points.  It computes the points' KB
// weights once, cuts the points into tasks (runs of up to kRun points that share
// a window start, so that one load of a window cell serves all of them) and
// sorts the tasks by run length.  Then, for every input b and pass of rank-term
// units, it stages the bin's (kBin + w - 1)^2-cell footprint of the grid in
// shared memory (cell-major, the rank terms of a cell one run of 16-byte units
// of two complex64 terms) while the previous stage computes: the stages are
// double-buffered with cp.async groups.
//
// A lane group owns a task, one lane per unit.  Groups sit on the 8-lane
// quarters of the warp, so that one 16-byte load instruction of a group touches
// distinct banks: up to 8 units a group takes one quarter (4 groups per warp);
// 9 or 10 units take a quarter each plus one or two lanes of the last quarter
// (3 groups); up to 16 take half a warp, up to 32 the whole warp.  The tasks of
// a warp come from the sorted list, so they have the same run length but at
// the list's class boundaries, and the warp runs the body specialised for its
// longest run.  The sum over rank terms is a shuffle reduction inside the
// group, the sum over wedges one vector atomic add per (point, wedge, input)
// into the output, which is cleared first.
//
// A point whose window start disagrees with the bin it was sorted into is
// recorded in the plan's error word and skipped.
#include <cuda_runtime.h>

#include <algorithm>

#include "apply_common.cuh"
#include "bin_common.cuh"
#include "fio_internal.h"

namespace fio {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kItThreads = 512;          // most threads of a CTA (launches use 256 or 512)
constexpr int kRunMax = 4;              // points of one task
constexpr int kItSmem = 220 * 1024;     // dynamic shared memory budget

// Lane layout of the groups for nuc units per cell (see the file comment).
struct GroupLane {
  int G;       // groups per warp
  int g, k;    // this lane's group and unit
  bool on;     // the lane holds a unit
};
__device__ __forceinline__ GroupLane group_lane(int lane, int nuc) {
  GroupLane r;
  if (nuc <= 8) {
    r.G = 4; r.g = lane >> 3; r.k = lane & 7;
  } else if (nuc <= 10) {
    r.G = 3;
    if (lane < 24) { r.g = lane >> 3; r.k = lane & 7; }
    else { const int e = lane - 24; r.g = e % 3; r.k = 8 + e / 3; }
  } else if (nuc <= 16) {
    r.G = 2; r.g = lane >> 4; r.k = lane & 15;
  } else {
    r.G = 1; r.g = 0; r.k = lane;
  }
  r.on = r.k < nuc;
  return r;
}

// Sum of v over the lanes of each group; the result is valid in the group's
// first lane (unit 0).  Lanes without a unit must hold 0.
__device__ __forceinline__ float group_total(float v, int lane, int G) {
  if (G == 3) {  // fold the units 8 and 9 of the last quarter into unit 0
    const int gq = (lane >> 3) % 3;
    const float a = __shfl_sync(kFull, v, 24 + gq), b = __shfl_sync(kFull, v, 27 + gq);
    if (lane < 24 && (lane & 7) == 0) v += a + b;
  }
  const int width = G >= 3 ? 8 : (G == 2 ? 16 : 32);
  for (int off = width >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  return v;
}

// Shared arrays of an item: weights [cap][2W], window start key [cap]
// (dr kBin + dc, -1 to skip), output index [cap], tasks [cap] (first point |
// count << 16); then one or two footprint buffers.
__host__ __device__ constexpr size_t it_item_bytes(int cap, int W) {
  return ((size_t)cap * (2 * W * 4 + 4 + 4 + 4) + 15) / 16 * 16;
}

// Copy `nuc` units (from unit u0) of every footprint cell of input b into sG,
// cell-major: sG[cell * nuc + k].  Warp w copies footprint rows w, w + 16, ...
__device__ __forceinline__ void stage_footprint(float4 *sG, const float2 *gw, int r0, int c0,
                                                int fh, int fw, int m1, int m2, int nch,
                                                int cbase, int nuc) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const FastDiv dnuc = make_fastdiv((unsigned)nuc);
  for (int f1 = wid; f1 < fh; f1 += nwarp) {
    int g1 = r0 + f1;
    if (g1 >= m1) g1 -= m1;
    const float2 *rowsrc = gw + (long long)g1 * m2 * nch + cbase;
    float4 *rowdst = sG + f1 * fw * nuc;
    for (int e = lane; e < fw * nuc; e += 32) {
      const int f2 = (int)fdiv((unsigned)e, dnuc), k = e - f2 * nuc;
      int g2 = c0 + f2;
      if (g2 >= m2) g2 -= m2;
      cp_async<16>(&rowdst[e], reinterpret_cast<const float4 *>(rowsrc + (long long)g2 * nch) + k);
    }
  }
}

// One task of up to R points (R uniform across the warp): the window sums of
// unit k for each point, times alpha', reduced over the group and added to out.
template <int W, int R>
__device__ __forceinline__ void run_task(const float4 *sG, const float (*sWt)[2 * W],
                                         const int *sKey, const uint32_t *sPm, int tk,
                                         const GroupLane &gl, int lane, int fw, int nuc,
                                         const float4 *al4, int qh, int u0, float2 *outb) {
  const int p0 = tk & 0xffff, cnt = tk >> 16;  // cnt = 0: no task for this group
  float4 a[R];
  float2 res[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    a[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gl.on && r < cnt) a[r] = al4[(long long)(p0 + r) * qh + u0 + gl.k];  // in flight meanwhile
  }
  float4 acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (gl.on && cnt > 0) {
    const int key = sKey[p0];
    const int dr = key / kBin, dc = key - dr * kBin;
    float w2[R][W];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int b = 0; b < W; ++b) w2[r][b] = r < cnt ? sWt[p0 + r][W + b] : 0.f;
#pragma unroll
    for (int a1 = 0; a1 < W; ++a1) {
      const float4 *pr = sG + ((dr + a1) * fw + dc) * nuc + gl.k;
      float4 rp[R];
#pragma unroll
      for (int r = 0; r < R; ++r) rp[r] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int a2 = 0; a2 < W; ++a2) {
        const float4 gv = pr[a2 * nuc];
#pragma unroll
        for (int r = 0; r < R; ++r) ufma(rp[r], w2[r][a2], gv);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) ufma(acc[r], r < cnt ? sWt[p0 + r][a1] : 0.f, rp[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    // alpha' times the window sums of this lane's two rank terms
    const float re = a[r].x * acc[r].x - a[r].y * acc[r].y + a[r].z * acc[r].z - a[r].w * acc[r].w;
    const float im = a[r].x * acc[r].y + a[r].y * acc[r].x + a[r].z * acc[r].w + a[r].w * acc[r].z;
    res[r] = make_float2(group_total(re, lane, gl.G), group_total(im, lane, gl.G));
  }
  if (gl.on && gl.k == 0) {
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (r < cnt) atomicAdd(outb + sPm[p0 + r], res[r]);
  }
}

template <int W>
__global__ void __launch_bounds__(kItThreads, 1)
k_interp_tasks(const float2 *__restrict__ grid, const WedgeDev *__restrict__ Wd,
               const int4 *__restrict__ items, const float2 *__restrict__ alpha,
               const uint2 *__restrict__ warps, const uint32_t *__restrict__ perm,
               float2 *__restrict__ out, long long NN, int B, KbDev kb, HornerDev hz, int cap,
               int chu, int nbuf, int *errw) {
  constexpr int FC = (kBin + W - 1) * (kBin + W - 1);  // footprint cells of a full bin
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float(*sWt)[2 * W] = reinterpret_cast<float(*)[2 * W]>(smem_raw);
  int *sKey = reinterpret_cast<int *>(smem_raw + (size_t)cap * 2 * W * 4);
  uint32_t *sPm = reinterpret_cast<uint32_t *>(sKey + cap);
  int *sTask = reinterpret_cast<int *>(sPm + cap);
  float4 *sG0 = reinterpret_cast<float4 *>(smem_raw + it_item_bytes(cap, W));
  const int bstride = FC * chu;  // footprint buffer st mod nbuf starts at sG0 + (st & (nbuf - 1)) bstride
  __shared__ int sNT;

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nthr = blockDim.x, nwarp = nthr >> 5;
  const int4 it = items[blockIdx.x];  // (wedge, bin, first sorted position, end)
  const int l = it.x;
  const int m1 = Wd[l].m1, m2 = Wd[l].m2, nb2 = Wd[l].nb2, qp = Wd[l].qp;
  const int nu = qp >> 1, qh = nu;  // 16-byte units per cell and input
  const int r0 = (it.y / nb2) * kBin, c0 = (it.y % nb2) * kBin;
  const int H1 = min(kBin, m1 - r0), H2 = min(kBin, m2 - c0);
  const int fh = H1 + W - 1, fw = H2 + W - 1;
  const int nch = B * qp;
  const float2 *gw = grid + Wd[l].grid_unit * B;
  const int npass = (nu + chu - 1) / chu;
  const int nst = npass * B;
  // stage st = (unit pass, input b) into buffer st mod nbuf
  auto issue = [&](int st) {
    const int pass = st / B, b = st - pass * B;
    const int u0 = pass * chu, nuc = min(chu, nu - u0);
    stage_footprint(sG0 + (st & (nbuf - 1)) * bstride, gw, r0, c0, fh, fw, m1, m2, nch, b * qp + 2 * u0, nuc);
    cp_async_commit();
  };

  for (int sub = it.z; sub < it.w; sub += cap) {  // the item's points, cap at a time
    const int np = min(cap, it.w - sub);
    const float4 *al4 = reinterpret_cast<const float4 *>(alpha + Wd[l].alpha_off) + (long long)sub * qh;
    const uint2 *ws = warps + (long long)l * NN + sub;
    const uint32_t *pm = perm + (long long)l * NN + sub;
    issue(0);  // the first footprint copy overlaps the weights and tasks below
    // the points' weights and window starts, once for every input and pass
    for (int p = tid; p < np; p += nthr) {
      float wt[2 * W];
      const int2 sc = point_weights<float, W>(ws[p], m1, m2, kb, hz, wt);
      const int dr = sc.x - r0, dc = sc.y - c0;
      int key = -1;
      if (dr >= 0 && dr < H1 && dc >= 0 && dc < H2) key = dr * kBin + dc;
      else atomicOr(errw, 1);
#pragma unroll
      for (int a = 0; a < 2 * W; ++a) sWt[p][a] = wt[a];
      sKey[p] = key;
      sPm[p] = pm[p];
    }
    if (tid == 0) sNT = 0;
    __syncthreads();
    // tasks: runs of equal window start cut into pieces of at most kRunMax
    // points, listed by piece length, longest first
    for (int cls = kRunMax; cls >= 1; --cls) {
      for (int p = tid; p < np; p += nthr) {
        const int key = sKey[p];
        if (key < 0 || (p > 0 && sKey[p - 1] == key)) continue;
        int len = 1;
        while (p + len < np && sKey[p + len] == key) ++len;
        for (int s0 = 0; s0 < len; s0 += kRunMax)
          if (min(kRunMax, len - s0) == cls) sTask[atomicAdd(&sNT, 1)] = (p + s0) | (cls << 16);
      }
      __syncthreads();
    }
    const int ntask = sNT;

    for (int st = 0; st < nst; ++st) {
      if (nbuf > 1 && st + 1 < nst) {
        issue(st + 1);  // double-buffered: the next stage streams in during this one
        cp_async_wait_group<1>();
      } else {
        if (nbuf == 1 && st > 0) issue(st);
        cp_async_wait_group<0>();
      }
      __syncthreads();  // stage st is in shared memory
      const int pass = st / B, b = st - pass * B;
      const int u0 = pass * chu, nuc = min(chu, nu - u0);
      const float4 *sG = sG0 + (st & (nbuf - 1)) * bstride;
      const GroupLane gl = group_lane(lane, nuc);
      float2 *outb = out + (long long)b * NN;
      for (int q0 = 0; q0 < ntask; q0 += nwarp * gl.G) {
        const int task = q0 + wid * gl.G + gl.g;
        const int tk = task < ntask ? sTask[task] : 0;
        switch (__reduce_max_sync(kFull, (unsigned)(tk >> 16))) {
          case 4: run_task<W, 4>(sG, sWt, sKey, sPm, tk, gl, lane, fw, nuc, al4, qh, u0, outb); break;
          case 3: run_task<W, 3>(sG, sWt, sKey, sPm, tk, gl, lane, fw, nuc, al4, qh, u0, outb); break;
          case 2: run_task<W, 2>(sG, sWt, sKey, sPm, tk, gl, lane, fw, nuc, al4, qh, u0, outb); break;
          case 1: run_task<W, 1>(sG, sWt, sKey, sPm, tk, gl, lane, fw, nuc, al4, qh, u0, outb); break;
          default: break;
        }
      }
      __syncthreads();  // every warp is done with this buffer (and, at the end, the tasks)
    }
  }
}

// Two launch shapes: one input with one unit pass (a single stage) runs two
// CTAs of 256 threads per SM with one footprint buffer and items of at most 512
// points, so that one CTA's staging overlaps the other's arithmetic; several
// stages run one CTA of 512 threads per SM with two buffers.
template <int W>
cudaError_t launch_w(const fio_plan_s *p, const void *grid, void *out, int B, cudaStream_t s,
                     const WorkRange &wr) {
  const long long NN = (long long)p->N * p->N;
  constexpr int FC = (kBin + W - 1) * (kBin + W - 1);
  int numax = 1;
  for (const WedgeDev &w : p->wedges) numax = std::max(numax, w.qp / 2);
  const bool single = B == 1 && (size_t)FC * numax * 16 + it_item_bytes(512, W) <= kItSmem / 2;
  const int cap = single ? std::min(512, item_points(W)) : item_points(W);
  const int nbuf = single ? 1 : 2, threads = single ? 256 : kItThreads;
  const size_t budget = single ? kItSmem / 2 : kItSmem;
  const size_t item = it_item_bytes(cap, W);
  const int chu = (int)std::min<size_t>(std::min(numax, 32), (budget - item) / (nbuf * (size_t)FC * 16));
  if (chu < 1) return cudaErrorInvalidConfiguration;
  const size_t smem = item + nbuf * (size_t)FC * chu * 16;
  cudaError_t e = cudaSuccess;
  if (wr.clear) e = cudaMemsetAsync(out, 0, sizeof(float2) * (size_t)NN * B, s);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_interp_tasks<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (wr.n_items > 0)
    k_interp_tasks<W><<<wr.n_items, threads, smem, s>>>(
        (const float2 *)grid, wr.wedges, wr.items, (const float2 *)wr.alpha, p->d_warps,
        p->d_perm, (float2 *)out, NN, B, make_kbdev(p), p->horner, cap, chu, nbuf, p->d_errword);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_interp_tasks(const fio_plan_s *p, const void *grid, void *out, int B,
                                cudaStream_t s, const WorkRange &wr) {
  switch (p->kb.w) {
    case 3: return launch_w<3>(p, grid, out, B, s, wr);
    case 4: return launch_w<4>(p, grid, out, B, s, wr);
    case 5: return launch_w<5>(p, grid, out, B, s, wr);
    case 6: return launch_w<6>(p, grid, out, B, s, wr);
    case 7: return launch_w<7>(p, grid, out, B, s, wr);
    case 8: return launch_w<8>(p, grid, out, B, s, wr);
    case 9: return launch_w<9>(p, grid, out, B, s, wr);
    case 10: return launch_w<10>(p, grid, out, B, s, wr);
    case 11: return launch_w<11>(p, grid, out, B, s, wr);
    case 12: return launch_w<12>(p, grid, out, B, s, wr);
  }
  return cudaErrorNotSupported;
}

}  // namespace fio
