// bin_common.cuh -- device helpers of the bin kernels (S3 interpolation and
// S4a spread): the Kaiser-Bessel weights of a warped point's window and the
// 16-byte units of rank terms with their packed FP32 updates.
#pragma once

#include <cuda_runtime.h>

#include "apply_common.cuh"
#include "fio_internal.h"

namespace fio {

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

// Window start cell (s1, s2) of a warped point and its 2W weights.
template <typename T, int W>
__device__ __forceinline__ int2 point_weights(uint2 Y, int m1, int m2, const KbDev &kb,
                                              const HornerDev &hz, T *wt) {
  T b1, b2;
  const int j01 = kb_first<T>(Y.x, m1, W, &b1);
  const int j02 = kb_first<T>(Y.y, m2, W, &b2);
  kb_weights<T, W>(b1, kb, hz, wt);
  kb_weights<T, W>(b2, kb, hz, wt + W);
  return make_int2(imodp(j01, m1), imodp(j02, m2));
}

// A 16-byte unit of rank terms: two complex64 terms or one complex128 term.
template <typename T> struct UnitT;
template <> struct UnitT<float> { using type = float4; };
template <> struct UnitT<double> { using type = double2; };
__device__ __forceinline__ void ufma(float4 &a, float w, const float4 &v) {
  const float2 ww = make_float2(w, w);
  const float2 lo = ffma2(ww, make_float2(v.x, v.y), make_float2(a.x, a.y));
  const float2 hi = ffma2(ww, make_float2(v.z, v.w), make_float2(a.z, a.w));
  a = make_float4(lo.x, lo.y, hi.x, hi.y);
}
__device__ __forceinline__ void uscale(float4 &v, float w) {
  const float2 ww = make_float2(w, w);
  const float2 lo = fmul2(ww, make_float2(v.x, v.y));
  const float2 hi = fmul2(ww, make_float2(v.z, v.w));
  v = make_float4(lo.x, lo.y, hi.x, hi.y);
}
// A single complex64 term as a unit (the spread of large batches).
__device__ __forceinline__ void ufma(float2 &a, float w, const float2 &v) {
  a = ffma2(make_float2(w, w), v, a);
}
__device__ __forceinline__ void uscale(float2 &v, float w) { v = fmul2(make_float2(w, w), v); }
__device__ __forceinline__ void uscale(double2 &v, double w) {
  v.x *= w;
  v.y *= w;
}
__device__ __forceinline__ void ufma(double2 &a, double w, const double2 &v) {
  a.x = fma(w, v.x, a.x);
  a.y = fma(w, v.y, a.y);
}
template <typename U, typename T> __device__ __forceinline__ void ufma4(U &a, T w, const U &v) {
  ufma(a, w, v);
}
template <typename U> __device__ __forceinline__ U uzero();
template <> __device__ __forceinline__ float4 uzero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <> __device__ __forceinline__ double2 uzero<double2>() { return make_double2(0.0, 0.0); }

}  // namespace fio
