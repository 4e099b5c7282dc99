// fft_engine.cuh -- batched 1D FFTs in shared memory (Stockham autosort,
// mixed radix 2/3/4/5/8/9/16), used by every grid stage of the apply path.
//
// Data of `nl` lines of length n sit in shared memory element-major: element e
// of line l is at buf[e * nl + l].  This is the natural layout of the NUFFT
// grids, whose innermost dimension is the channel (batch, rank term), so the
// lines of a CTA are contiguous in global memory.
//
// Transform convention: X[k] = sum_j x[j] exp(sign * 2 pi i j k / n), sign = +-1,
// unnormalised.  Twiddles come from a table tw[k] = exp(-2 pi i k / n) (k < n)
// that the caller places in shared memory.
#pragma once

#include <cuda_runtime.h>

#include "fio_internal.h"

namespace fio {

template <typename T> struct CxT;
template <> struct CxT<float> { using type = float2; };
template <> struct CxT<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {  // a * conj(b)
  return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return {a.x, -a.y}; }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) {
  return {a.x * s, a.y * s};
}
// i * sign * a
template <typename C> __device__ __forceinline__ C cmul_si(C a, int sign) {
  return sign > 0 ? C{-a.y, a.x} : C{a.y, -a.x};
}

// Packed two-wide FP32 arithmetic (sm_100 and later): each lane rounds like the
// scalar instruction (IEEE, round to nearest), in half the instructions.
union F2U {
  float2 f;
  unsigned long long u;
};
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  F2U A, Bv, Cv, D;
  A.f = a;
  Bv.f = b;
  Cv.f = c;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(D.u) : "l"(A.u), "l"(Bv.u), "l"(Cv.u));
  return D.f;
}
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
  F2U A, Bv, D;
  A.f = a;
  Bv.f = b;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(D.u) : "l"(A.u), "l"(Bv.u));
  return D.f;
}
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
  F2U A, Bv, D;
  A.f = a;
  Bv.f = b;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(D.u) : "l"(A.u), "l"(Bv.u));
  return D.f;
}
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
  F2U A, Bv, D;
  A.f = a;
  Bv.f = b;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(D.u) : "l"(A.u), "l"(Bv.u));
  return D.f;
}
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) { return fadd2(a, b); }
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) { return fsub2(a, b); }
// The complex product stays scalar (two FMUL, two FFMA): a packed form needs the
// operands swizzled, (a.x, a.x), (-a.y, a.y), (b.y, b.x), which costs more ALU
// moves than it saves.

// ---------------------------------------------------------------- butterflies
// V[k] = sum_r v[r] exp(sign 2 pi i r k / R)

template <typename C> __device__ __forceinline__ void bfly2(C *v) {
  C a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <typename C> __device__ __forceinline__ void bfly4(C *v, int sign) {
  C s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
  C s13 = cadd(v[1], v[3]), d13 = cmul_si(csub(v[1], v[3]), sign);
  v[0] = cadd(s02, s13);
  v[2] = csub(s02, s13);
  v[1] = cadd(d02, d13);
  v[3] = csub(d02, d13);
}

template <typename C> __device__ __forceinline__ void bfly3(C *v, int sign) {
  using T = decltype(v[0].x);
  const T c1 = T(-0.5);
  const T s1 = T(0.86602540378443864676372317075294);  // sin(2 pi / 3)
  C t1 = cadd(v[1], v[2]);
  C m = cadd(v[0], cscale(t1, c1));
  C d = cmul_si(cscale(csub(v[1], v[2]), s1), sign);
  v[0] = cadd(v[0], t1);
  v[1] = cadd(m, d);
  v[2] = csub(m, d);
}

template <typename C> __device__ __forceinline__ void bfly5(C *v, int sign) {
  using T = decltype(v[0].x);
  const T c1 = T(0.30901699437494742410229341718282);   // cos(2 pi / 5)
  const T c2 = T(-0.80901699437494742410229341718282);  // cos(4 pi / 5)
  const T s1 = T(0.95105651629515357211643933337938);   // sin(2 pi / 5)
  const T s2 = T(0.58778525229247312916870595463907);   // sin(4 pi / 5)
  C a14 = cadd(v[1], v[4]), d14 = csub(v[1], v[4]);
  C a23 = cadd(v[2], v[3]), d23 = csub(v[2], v[3]);
  C m1 = cadd(v[0], cadd(cscale(a14, c1), cscale(a23, c2)));
  C m2 = cadd(v[0], cadd(cscale(a14, c2), cscale(a23, c1)));
  C n1 = cmul_si(cadd(cscale(d14, s1), cscale(d23, s2)), sign);
  C n2 = cmul_si(csub(cscale(d14, s2), cscale(d23, s1)), sign);
  v[0] = cadd(v[0], cadd(a14, a23));
  v[1] = cadd(m1, n1);
  v[4] = csub(m1, n1);
  v[2] = cadd(m2, n2);
  v[3] = csub(m2, n2);
}

template <typename C> __device__ __forceinline__ void bfly8(C *v, int sign) {
  using T = decltype(v[0].x);
  const T r2 = T(0.70710678118654752440084436210485);
  C e[4] = {v[0], v[2], v[4], v[6]};
  C o[4] = {v[1], v[3], v[5], v[7]};
  bfly4(e, sign);
  bfly4(o, sign);
  // o[k] *= exp(sign 2 pi i k / 8)
  C w1 = {r2, T(sign) * r2}, w3 = {-r2, T(sign) * r2};
  o[1] = cmul(o[1], w1);
  o[2] = cmul_si(o[2], sign);
  o[3] = cmul(o[3], w3);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = cadd(e[k], o[k]);
    v[k + 4] = csub(e[k], o[k]);
  }
}

// DFT_9 as 3 x 3: with r = 3 r1 + r2 and k = k1 + 3 k2,
// V[k] = sum_r2 W3^(r2 k2) w9^(r2 k1) [sum_r1 v[3 r1 + r2] W3^(r1 k1)].
template <typename C> __device__ __forceinline__ void bfly9(C *v, int sign) {
  using T = decltype(v[0].x);
  const T c1 = T(0.76604444311897803520), s1 = T(0.64278760968653932632);   // 2 pi / 9
  const T c2 = T(0.17364817766693034885), s2 = T(0.98480775301220805936);   // 4 pi / 9
  const T c4 = T(-0.93969262078590838405), s4 = T(0.34202014332566873304);  // 8 pi / 9
  C a[3][3];
#pragma unroll
  for (int r2 = 0; r2 < 3; ++r2) {
    a[r2][0] = v[r2];
    a[r2][1] = v[3 + r2];
    a[r2][2] = v[6 + r2];
    bfly3(a[r2], sign);
  }
  const T sg = T(sign);
  a[1][1] = cmul(a[1][1], C{c1, sg * s1});
  a[1][2] = cmul(a[1][2], C{c2, sg * s2});
  a[2][1] = cmul(a[2][1], C{c2, sg * s2});
  a[2][2] = cmul(a[2][2], C{c4, sg * s4});
#pragma unroll
  for (int k1 = 0; k1 < 3; ++k1) {
    C t[3] = {a[0][k1], a[1][k1], a[2][k1]};
    bfly3(t, sign);
    v[k1] = t[0];
    v[k1 + 3] = t[1];
    v[k1 + 6] = t[2];
  }
}

// DFT_16 as 4 x 4: with r = 4 r1 + r2 and k = k1 + 4 k2,
// V[k] = sum_r2 W4^(r2 k2) w16^(r2 k1) [sum_r1 v[4 r1 + r2] W4^(r1 k1)].
template <typename C> __device__ __forceinline__ void bfly16(C *v, int sign) {
  using T = decltype(v[0].x);
  const T c1 = T(0.92387953251128675613), s1 = T(0.38268343236508977173);  // pi / 8
  const T r2 = T(0.70710678118654752440);
  const T sg = T(sign);
  C a[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    a[q][0] = v[q];
    a[q][1] = v[4 + q];
    a[q][2] = v[8 + q];
    a[q][3] = v[12 + q];
    bfly4(a[q], sign);
  }
  // w16^m for m = q k1: 1: (c1, s1), 2: (r2, r2), 3: (s1, c1), 4: i, 6: (-r2, r2), 9: (-c1, -s1)
  a[1][1] = cmul(a[1][1], C{c1, sg * s1});
  a[1][2] = cmul(a[1][2], C{r2, sg * r2});
  a[1][3] = cmul(a[1][3], C{s1, sg * c1});
  a[2][1] = cmul(a[2][1], C{r2, sg * r2});
  a[2][2] = cmul_si(a[2][2], sign);
  a[2][3] = cmul(a[2][3], C{-r2, sg * r2});
  a[3][1] = cmul(a[3][1], C{s1, sg * c1});
  a[3][2] = cmul(a[3][2], C{-r2, sg * r2});
  a[3][3] = cmul(a[3][3], C{-c1, -sg * s1});
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C t[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
    bfly4(t, sign);
    v[k1] = t[0];
    v[k1 + 4] = t[1];
    v[k1 + 8] = t[2];
    v[k1 + 12] = t[3];
  }
}

template <int R, typename C> __device__ __forceinline__ void bfly(C *v, int sign) {
  if constexpr (R == 2) bfly2(v);
  if constexpr (R == 3) bfly3(v, sign);
  if constexpr (R == 4) bfly4(v, sign);
  if constexpr (R == 5) bfly5(v, sign);
  if constexpr (R == 8) bfly8(v, sign);
  if constexpr (R == 9) bfly9(v, sign);
  if constexpr (R == 16) bfly16(v, sign);
}

// One Stockham stage (decimation in time): for butterfly j of each line,
// read v[r] = in[j + r n/R], twiddle by w^(k r) with k = j mod Ns and
// w = exp(sign 2 pi i / (Ns R)), DFT_R, write to out[(j/Ns) Ns R + k + r Ns].
template <int R, typename C>
__device__ __forceinline__ void fft_stage(const C *__restrict__ in, C *__restrict__ out, int n,
                                          int nl, int Ns, int sign, const C *__restrict__ tw) {
  const int nb = n / R;
  const int step = n / (Ns * R);
  for (int it = threadIdx.x; it < nb * nl; it += blockDim.x) {
    const int l = it % nl, j = it / nl;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[(j + r * nb) * nl + l];
    const int k = j % Ns;
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C t = tw[k * r * step];
        if (sign > 0) t.y = -t.y;
        v[r] = cmul(v[r], t);
      }
    }
    bfly<R>(v, sign);
    const int d = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) out[(d + r * Ns) * nl + l] = v[r];
  }
}

// Run all stages of plan `pl` on buffer a (scratch b).  Returns the buffer
// holding the result.  Must be called by all threads of the block; ends with
// __syncthreads().  The caller synchronises before the call.
template <typename C>
__device__ C *fft_exec(C *a, C *b, int n, int nl, const FftPlanDev &pl, int sign, const C *tw) {
  int Ns = 1;
  for (int s = 0; s < pl.nstages; ++s) {
    const int R = pl.radix[s];
    switch (R) {
      case 16: fft_stage<16>(a, b, n, nl, Ns, sign, tw); break;
      case 9: fft_stage<9>(a, b, n, nl, Ns, sign, tw); break;
      case 8: fft_stage<8>(a, b, n, nl, Ns, sign, tw); break;
      case 4: fft_stage<4>(a, b, n, nl, Ns, sign, tw); break;
      case 2: fft_stage<2>(a, b, n, nl, Ns, sign, tw); break;
      case 3: fft_stage<3>(a, b, n, nl, Ns, sign, tw); break;
      case 5: fft_stage<5>(a, b, n, nl, Ns, sign, tw); break;
    }
    __syncthreads();
    C *t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

// ------------------------------------------------------- in-place variant --
// Division by a runtime divisor d <= 4096 for x < 2^20: q = (x ceil(2^40 / d)) >> 40
// is exact (the rounding error x (ceil(2^40/d) d - 2^40) / 2^40 stays below 1).
struct FastDiv {
  unsigned d;
  unsigned long long M;
};
__host__ __device__ inline FastDiv make_fastdiv(unsigned d) {
  return FastDiv{d, ((1ULL << 40) + d - 1) / d};
}
__device__ __forceinline__ unsigned fdiv(unsigned x, const FastDiv &f) {
  return (unsigned)(((unsigned long long)x * f.M) >> 40);
}
// x / R for the radices 2, 3, 4, 5, 8, 9, 16 and x < 2^16 (multiply-shift
// constants ceil(2^17 / 3), ceil(2^18 / 5) and ceil(2^19 / 9), exact on that range).
__device__ __forceinline__ int div_radix(int x, int R) {
  switch (R) {
    case 2: return x >> 1;
    case 4: return x >> 2;
    case 8: return x >> 3;
    case 16: return x >> 4;
    case 3: return (int)(((unsigned)x * 43691u) >> 17);
    case 9: return (int)(((unsigned)x * 58255u) >> 19);
    default: return (int)(((unsigned)x * 52429u) >> 18);
  }
}

// The lines of an in-place transform are shared out with a fixed line per
// thread: thread t < lanes works on line t % nl, items t / nl, t / nl + step, ...
struct LineMap {
  int lanes, l, i0, step;
};
__device__ __forceinline__ LineMap line_map(int nl) {
  LineMap m;
  m.step = blockDim.x / nl;
  m.lanes = m.step * nl;
  m.i0 = threadIdx.x / nl;
  m.l = threadIdx.x - m.i0 * nl;
  return m;
}

// Decimation in frequency on a single shared buffer.  A stage on blocks of
// length m with radix R takes, for j < m/R, x_r = a[j + r m/R] (r < R), forms
// X_k = sum_r x_r exp(sign 2 pi i r k / R), multiplies by exp(sign 2 pi i j k / m)
// and writes it back to a[j + k m/R]: every butterfly reads and writes the same
// R slots, so one buffer and one barrier per stage suffice.  The result is in
// digit-reversed order: frequency k is at fft_dif_pos(k).
template <int R, int SIGN, typename C>
__device__ __forceinline__ void fft_stage_dif(C *a, int n, int nl, int m,
                                              const C *__restrict__ tw, const LineMap &lm) {
  constexpr int sign = SIGN;
  if ((int)threadIdx.x >= lm.lanes) return;
  const int mr = m / R;          // butterfly stride within a block
  const int tws = n / m;         // table step of exp(sign 2 pi i / m)
  const FastDiv dmr = make_fastdiv((unsigned)mr);
  const int nbf = n / R;
  // butterfly idx = b mr + j, advanced by step = sb mr + sj without dividing
  const int sb = (int)fdiv((unsigned)lm.step, dmr), sj = lm.step - sb * mr;
  int b = (int)fdiv((unsigned)lm.i0, dmr), j = lm.i0 - b * mr;
  for (int idx = lm.i0; idx < nbf; idx += lm.step) {
    C *base = a + (b * m + j) * nl + lm.l;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = base[r * mr * nl];
    bfly<R>(v, sign);
    if (j > 0) {
#pragma unroll
      for (int k = 1; k < R; ++k) {
        C t = tw[j * k * tws];
        if (sign > 0) t.y = -t.y;
        v[k] = cmul(v[k], t);
      }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) base[k * mr * nl] = v[k];
    b += sb;
    j += sj;
    if (j >= mr) {
      j -= mr;
      ++b;
    }
  }
}

// Run all stages of plan `pl` in place on a (nl interleaved lines: element e of
// line l at a[e nl + l]), transform sign SIGN (compile time).  Call after a
// barrier; ends with a barrier.
template <int SIGN, typename C>
__device__ void fft_exec_dif(C *a, int n, int nl, const FftPlanDev &pl, const C *tw) {
  const LineMap lm = line_map(nl);
  int m = n;
  for (int s = 0; s < pl.nstages; ++s) {
    const int R = pl.radix[s];
    switch (R) {
      case 16: fft_stage_dif<16, SIGN>(a, n, nl, m, tw, lm); break;
      case 9: fft_stage_dif<9, SIGN>(a, n, nl, m, tw, lm); break;
      case 8: fft_stage_dif<8, SIGN>(a, n, nl, m, tw, lm); break;
      case 4: fft_stage_dif<4, SIGN>(a, n, nl, m, tw, lm); break;
      case 2: fft_stage_dif<2, SIGN>(a, n, nl, m, tw, lm); break;
      case 3: fft_stage_dif<3, SIGN>(a, n, nl, m, tw, lm); break;
      case 5: fft_stage_dif<5, SIGN>(a, n, nl, m, tw, lm); break;
    }
    __syncthreads();
    m /= R;
  }
}

// fft_dif_pos for every k < n into tab (one entry per frequency, shared by all
// lines of the CTA).  Visible to the block after its next barrier.
__device__ __forceinline__ int fft_dif_pos(int k, const FftPlanDev &pl);
__device__ __forceinline__ void fft_dif_table(short *tab, const FftPlanDev &pl) {
  for (int k = threadIdx.x; k < pl.n; k += blockDim.x) tab[k] = (short)fft_dif_pos(k, pl);
}

// Buffer slot of frequency k after fft_exec_dif: with k = d0 + R0 d1 + R0 R1 d2 + ...,
// slot = d0 n/R0 + d1 n/(R0 R1) + ...
__device__ __forceinline__ int fft_dif_pos(int k, const FftPlanDev &pl) {
  int p = 0, span = pl.n;
#pragma unroll 1
  for (int s = 0; s < pl.nstages; ++s) {
    const int R = pl.radix[s];
    span = div_radix(span, R);
    const int q = div_radix(k, R);
    p += (k - q * R) * span;
    k = q;
  }
  return p;
}

}  // namespace fio
