// apply_common.cuh -- device helpers shared by the apply kernels: complex
// type of a precision, periodic index, and the Kaiser-Bessel window of a
// warped point (the interpolation weights of the type-2 / type-1 NUFFT).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "fft_engine.cuh"
#include "fio_internal.h"

namespace fio {

template <typename T> using Cx = typename CxT<T>::type;

__device__ __forceinline__ int imodp(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

constexpr int kThreads = 256;

// ------------------------------------------------ asynchronous staging -----
// cp.async copies global -> shared without passing through registers, so a
// thread can have all of its staging loads in flight at once.  Both addresses
// must be aligned to the copy size.  cp_async_wait() waits for this thread's
// copies; a barrier then makes every thread's copies visible.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}
// Close the group of this thread's copies issued since the last commit; then
// cp_async_wait_group<n>() waits until at most n of its groups are pending.
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N> __device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
// One complex element (8 or 16 bytes).
template <typename C>
__device__ __forceinline__ void cp_async_elem(C *smem, const C *gmem) {
  cp_async<(int)sizeof(C)>(smem, gmem);
}

// ------------------------------------------------------------ KB kernel ----
// phi(s) = I0(beta sqrt(1 - (2s/w)^2)) / I0(beta) for |s| < w/2, else 0.
__device__ __forceinline__ float kb_phi(float s, float two_over_w, float beta, float inv_i0b) {
  float z = s * two_over_w;
  float a = 1.0f - z * z;
  return a > 0.0f ? cyl_bessel_i0f(beta * sqrtf(a)) * inv_i0b : 0.0f;
}
__device__ __forceinline__ double kb_phi(double s, double two_over_w, double beta,
                                         double inv_i0b) {
  double z = s * two_over_w;
  double a = 1.0 - z * z;
  return a > 0.0 ? cyl_bessel_i0(beta * sqrt(a)) * inv_i0b : 0.0;
}

struct KbDev {
  int w;
  double beta, inv_i0b;
};

inline KbDev make_kbdev(const fio_plan_s *p) {
  KbDev kb;
  kb.w = p->kb.w;
  kb.beta = p->kb.beta;
  kb.inv_i0b = 1.0 / std::cyl_bessel_i(0.0, p->kb.beta);
  return kb;
}

// First grid cell of the width-w window of a warped coordinate, before the
// periodic reduction: u = y' m with y' = Y / 2^32, cells j0 .. j0 + w - 1,
// j0 = floor(u - w/2) + 1.  *base receives u - j0 (in [w/2 - 1, w/2)).
template <typename T>
__device__ __forceinline__ int kb_first(uint32_t Y, int m, int w, T *base) {
  const unsigned long long P = (unsigned long long)Y * (unsigned)m;
  const int i = (int)(P >> 32);
  const T f = (T)(uint32_t)P * T(2.3283064365386962890625e-10);  // 2^-32
  const int hw = w >> 1;
  int j0 = i - hw + 1;
  if (w & 1) j0 = i - hw + ((uint32_t)P >= 0x80000000u ? 1 : 0);  // f >= 1/2, exactly
  *base = f + T(i - j0);
  return j0;
}

// The w weights phi(u - j0 - a), a < w, and j0 mod m.
template <typename T>
__device__ __forceinline__ int kb_window(uint32_t Y, int m, const KbDev &kb, T *wgt) {
  T base;
  const int j0 = kb_first<T>(Y, m, kb.w, &base);
  const T tw = T(2.0) / T(kb.w), beta = T(kb.beta), inv = T(kb.inv_i0b);
  for (int a = 0; a < kb.w; ++a) wgt[a] = kb_phi(base - T(a), tw, beta, inv);
  return imodp(j0, m);
}

}  // namespace fio
