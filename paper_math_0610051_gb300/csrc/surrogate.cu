// surrogate.cu -- a learned surrogate of the tau-mode phase offset
// Phi = x.xi + |xi| tau(x, theta): a 4 -> 64 -> 64 -> 3 tanh MLP mapping
// (x1, x2, cos theta, sin theta) to (tau, d tau/d x1, d tau/d x2) (x1 and x2 enter
// the first layer as 2 x - 1), trained on the
// GPU on samples of the plain (exact) evaluation.
//
// The 64 x 64 layer runs on the tensor cores (mma.sync m16n8k16, BF16 operands,
// FP32 accumulation), both forward and in the backward data product
// dz2 W2^T.  The small layers and the weight gradients are FP32 SIMT; the master
// weights are FP32 and Adam updates them.  d tau / d theta (needed for the warped
// points, grad_xi(|xi| tau) = tau xihat + d_theta tau xihat_perp) is the network's
// directional derivative along (0, 0, -sin theta, cos theta), propagated forward
// with the same kernels.
//
// Parameter vector (FP32): W1[4][64], b1[64], W2[64][64], b2[64], W3[64][3], b3[3],
// row-major with the input index first.  Outputs are scaled: the network learns
// (tau / s_tau, d1 tau / s_d, d2 tau / s_d).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "fio_internal.h"

namespace fio {
namespace sur {

constexpr int kH = 64;
constexpr int kNP = 4 * kH + kH + kH * kH + kH + kH * 3 + 3;  // 4675
constexpr int oW1 = 0, oB1 = oW1 + 4 * kH, oW2 = oB1 + kH, oB2 = oW2 + kH * kH,
              oW3 = oB2 + kH, oB3 = oW3 + kH * 3;
constexpr double kTwoPi = 6.283185307179586476925286766559;

// ------------------------------------------------------------ fragments ----

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}

// D += A (16x16, row) * B (16x8, col), BF16 in, FP32 accumulate.
__device__ __forceinline__ void mma16816(float *d, const uint32_t *a, const uint32_t *b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Input c of sample i as the network sees it: x1, x2 in [0, 1) are mapped to
// [-1, 1) so that every input is centred and of unit range.
__device__ __forceinline__ float net_input(const float *__restrict__ X, long long i, int c) {
  const float v = X[4 * i + c];
  return c < 2 ? fmaf(2.0f, v, -1.0f) : v;
}

// Shared copies of the weights: W2 row-major [k][j] and transposed [j][k] in
// BF16 (so that every B fragment is a 32-bit load), the rest in FP32.
struct SmemW {
  __nv_bfloat16 w2[kH * kH];   // [k][j]
  __nv_bfloat16 w2t[kH * kH];  // [j][k]
  float w1[4 * kH], b1[kH], b2[kH], w3[kH * 3], b3[4];
};

__device__ void load_weights(SmemW &S, const float *__restrict__ P) {
  for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) {
    const int k = i / kH, j = i % kH;
    const __nv_bfloat16 v = __float2bfloat16_rn(P[oW2 + i]);
    S.w2[i] = v;
    S.w2t[j * kH + k] = v;
  }
  for (int i = threadIdx.x; i < 4 * kH; i += blockDim.x) S.w1[i] = P[oW1 + i];
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    S.b1[i] = P[oB1 + i];
    S.b2[i] = P[oB2 + i];
  }
  for (int i = threadIdx.x; i < kH * 3; i += blockDim.x) S.w3[i] = P[oW3 + i];
  if (threadIdx.x < 3) S.b3[threadIdx.x] = P[oB3 + threadIdx.x];
  __syncthreads();
}

// B fragment (k16 x n8) of a row-major [K][64] BF16 matrix M stored transposed
// as MT[n][k]: b0 = (M[k0 + 2t][n0 + g], M[k0 + 2t + 1][n0 + g]), b1 at k + 8.
__device__ __forceinline__ void bfrag(const __nv_bfloat16 *MT, int k0, int n0, int g, int t,
                                      uint32_t *b) {
  b[0] = *reinterpret_cast<const uint32_t *>(MT + (n0 + g) * kH + k0 + 2 * t);
  b[1] = *reinterpret_cast<const uint32_t *>(MT + (n0 + g) * kH + k0 + 8 + 2 * t);
}

// Per-warp forward of 16 samples (rows r = g and g + 8 of this lane).
// h1[kk][e]: the lane's layer-1 activations in A-fragment order
//   (e = 0,1: row g, cols 16kk + 2t + {0,1}; e = 2,3: row g + 8; e = 4..7: cols + 8);
// h2[nt][e]: layer-2 activations in C-fragment order (rows g / g + 8, cols 8nt + 2t + {0,1}).
struct Fwd {
  float h1[4][8];
  float h2[8][4];
  float y[2][3];  // rows g, g + 8 (valid in every lane after the reduction)
};

__device__ __forceinline__ void forward16(const SmemW &S, const float (*x)[4], int g, int t,
                                          Fwd &F, const float (*dx)[4] = nullptr,
                                          float *dy0 = nullptr) {
  // layer 1 (K = 4, FP32) and its tangent
  float th1[4][8];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk)
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int row = (e & 2) ? 1 : 0;
      const int col = 16 * kk + 2 * t + (e & 1) + ((e & 4) ? 8 : 0);
      float z = S.b1[col], dz = 0.f;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        z = fmaf(x[row][i], S.w1[i * kH + col], z);
        if (dx) dz = fmaf(dx[row][i], S.w1[i * kH + col], dz);
      }
      const float h = tanhf(z);
      F.h1[kk][e] = h;
      th1[kk][e] = (1.f - h * h) * dz;
    }
  // layer 2 on the tensor cores: z2 = h1 W2 (+ tangent dh1 W2)
  float acc[8][4], tac[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[nt][e] = tac[nt][e] = 0.f;
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    uint32_t a[4], ta[4];
    a[0] = pack_bf16(F.h1[kk][0], F.h1[kk][1]);
    a[1] = pack_bf16(F.h1[kk][2], F.h1[kk][3]);
    a[2] = pack_bf16(F.h1[kk][4], F.h1[kk][5]);
    a[3] = pack_bf16(F.h1[kk][6], F.h1[kk][7]);
    if (dx) {
      ta[0] = pack_bf16(th1[kk][0], th1[kk][1]);
      ta[1] = pack_bf16(th1[kk][2], th1[kk][3]);
      ta[2] = pack_bf16(th1[kk][4], th1[kk][5]);
      ta[3] = pack_bf16(th1[kk][6], th1[kk][7]);
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      uint32_t b[2];
      bfrag(S.w2t, 16 * kk, 8 * nt, g, t, b);
      mma16816(acc[nt], a, b);
      if (dx) mma16816(tac[nt], ta, b);
    }
  }
  // layer 2 activation and layer 3 (FP32, reduced over the 4 lanes of a row)
  float y[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}}, ty[2] = {0.f, 0.f};
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int col = 8 * nt + 2 * t + (e & 1), row = e >> 1;
      const float h = tanhf(acc[nt][e] + S.b2[col]);
      F.h2[nt][e] = h;
#pragma unroll
      for (int o = 0; o < 3; ++o) y[row][o] = fmaf(h, S.w3[col * 3 + o], y[row][o]);
      if (dx) ty[row] = fmaf((1.f - h * h) * tac[nt][e], S.w3[col * 3], ty[row]);
    }
#pragma unroll
  for (int row = 0; row < 2; ++row) {
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      float v = y[row][o];
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      F.y[row][o] = v + S.b3[o];
    }
    if (dx) {
      float v = ty[row];
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      dy0[row] = v;
    }
  }
}

// ------------------------------------------------------------- kernels -----

// Plain-evaluation samples: uniform (x1, x2, theta) from a counter-based hash;
// X = (x1, x2, cos theta, sin theta) in FP32, T = (tau, d1, d2, d_theta) in FP64
// by the literal sum over modes.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {  // SplitMix64 finaliser
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double unif(uint64_t seed, uint64_t i, int c) {
  return (double)(mix64(seed ^ mix64(3 * i + c)) >> 11) * 0x1.0p-53;
}

__global__ void k_samples(const double *__restrict__ modes, int nmodes, int n, uint64_t seed,
                          float *__restrict__ X, double *__restrict__ T) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x1 = unif(seed, i, 0), x2 = unif(seed, i, 1), th = kTwoPi * unif(seed, i, 2);
  double st, ct;
  sincos(th, &st, &ct);
  double tau = 0, d1 = 0, d2 = 0, dt = 0;
  for (int j = 0; j < nmodes; ++j) {
    const double *p = modes + 5 * j;
    double s, c;
    sincos(kTwoPi * (p[1] * x1 + p[2] * x2) + p[3] * th + p[4], &s, &c);
    tau += p[0] * c;
    d1 -= p[0] * s * kTwoPi * p[1];
    d2 -= p[0] * s * kTwoPi * p[2];
    dt -= p[0] * s * p[3];
  }
  X[4 * i] = (float)x1;
  X[4 * i + 1] = (float)x2;
  X[4 * i + 2] = (float)ct;
  X[4 * i + 3] = (float)st;
  T[4 * i] = tau;
  T[4 * i + 1] = d1;
  T[4 * i + 2] = d2;
  T[4 * i + 3] = dt;
}

__global__ void k_scale_targets(const double *__restrict__ T, int n, float s_tau, float s_d,
                                float *__restrict__ Ts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Ts[3 * i] = (float)(T[4 * i] / s_tau);
  Ts[3 * i + 1] = (float)(T[4 * i + 1] / s_d);
  Ts[3 * i + 2] = (float)(T[4 * i + 2] / s_d);
}

// Inference: Y[i] = (tau, d1 tau, d2 tau, d_theta tau) in physical units.
__global__ void __launch_bounds__(128) k_infer(const float *__restrict__ P, const float *__restrict__ X,
                                               int n, float s_tau, float s_d,
                                               float *__restrict__ Y) {
  __shared__ SmemW S;
  load_weights(S, P);
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile * 16 < n; tile += warps) {
    float x[2][4], dx[2][4];
    for (int row = 0; row < 2; ++row) {
      const int i = min(tile * 16 + g + 8 * row, n - 1);
      for (int c = 0; c < 4; ++c) x[row][c] = net_input(X, i, c);
      dx[row][0] = dx[row][1] = 0.f;
      dx[row][2] = -x[row][3];
      dx[row][3] = x[row][2];
    }
    Fwd F;
    float dy0[2];
    forward16(S, x, g, t, F, dx, dy0);
    if (t == 0)
      for (int row = 0; row < 2; ++row) {
        const int i = tile * 16 + g + 8 * row;
        if (i < n) {
          Y[4 * i] = F.y[row][0] * s_tau;
          Y[4 * i + 1] = F.y[row][1] * s_d;
          Y[4 * i + 2] = F.y[row][2] * s_d;
          Y[4 * i + 3] = dy0[row] * s_tau;
        }
      }
  }
}

// Training forward + backward for a mini-batch [i0, i0 + nb): loss sum, and the
// per-sample activations the weight gradients need (H1, H2, DZ1, DZ2: [nb][64],
// DY: [nb][3]).  The data product dh1 = dz2 W2^T runs on the tensor cores, with
// dz2's C fragments reused as A fragments.
__global__ void __launch_bounds__(128) k_train_fb(const float *__restrict__ P,
                                                  const float *__restrict__ X,
                                                  const float *__restrict__ Ts, int i0, int nb,
                                                  float *__restrict__ H1, float *__restrict__ H2,
                                                  float *__restrict__ DZ1,
                                                  float *__restrict__ DZ2,
                                                  float *__restrict__ DY,
                                                  double *__restrict__ loss) {
  __shared__ SmemW S;
  load_weights(S, P);
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int warps = gridDim.x * (blockDim.x >> 5);
  double lsum = 0.0;
  for (int tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile * 16 < nb; tile += warps) {
    float x[2][4];
    bool ok[2];
    for (int row = 0; row < 2; ++row) {
      const int r = tile * 16 + g + 8 * row;
      ok[row] = r < nb;
      const int i = i0 + min(r, nb - 1);
      for (int c = 0; c < 4; ++c) x[row][c] = net_input(X, i, c);
    }
    Fwd F;
    forward16(S, x, g, t, F);
    // dy = 2 (y - T) / nb on rows g, g + 8 (every lane holds them)
    float dy[2][3];
    for (int row = 0; row < 2; ++row) {
      const int r = tile * 16 + g + 8 * row;
      const int i = i0 + min(r, nb - 1);
      for (int o = 0; o < 3; ++o) {
        const float e = ok[row] ? F.y[row][o] - Ts[3 * i + o] : 0.f;
        dy[row][o] = 2.f * e / (float)nb;
        if (t == 0) lsum += (double)e * e;
      }
    }
    // dz2 = (dy W3^T) (1 - h2^2), then dh1 = dz2 W2^T on the tensor cores
    float dz2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int col = 8 * nt + 2 * t + (e & 1), row = e >> 1;
        float dh = 0.f;
        for (int o = 0; o < 3; ++o) dh = fmaf(dy[row][o], S.w3[col * 3 + o], dh);
        const float h = F.h2[nt][e];
        dz2[nt][e] = dh * (1.f - h * h);
      }
    float dh1[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) dh1[nt][e] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      // A = dz2 columns 16kk .. 16kk + 15: C fragments of n-tiles 2kk, 2kk + 1
      uint32_t a[4];
      a[0] = pack_bf16(dz2[2 * kk][0], dz2[2 * kk][1]);
      a[1] = pack_bf16(dz2[2 * kk][2], dz2[2 * kk][3]);
      a[2] = pack_bf16(dz2[2 * kk + 1][0], dz2[2 * kk + 1][1]);
      a[3] = pack_bf16(dz2[2 * kk + 1][2], dz2[2 * kk + 1][3]);
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        uint32_t b[2];
        bfrag(S.w2, 16 * kk, 8 * nt, g, t, b);  // W2^T as [j][k]: its transpose is W2
        mma16816(dh1[nt], a, b);
      }
    }
    // store activations (C-fragment order of the 16 x 64 tiles)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int col = 8 * nt + 2 * t + (e & 1), row = e >> 1;
        const int r = tile * 16 + g + 8 * row;
        if (r >= nb) continue;
        // layer-1 value of (row, col): A-fragment index of column col
        const int kk = col >> 4, cc = col & 15;
        const int ea = (row ? 2 : 0) + (cc & 1) + ((cc & 8) ? 4 : 0);
        const float h1 = F.h1[kk][ea];
        H1[(size_t)r * kH + col] = h1;
        H2[(size_t)r * kH + col] = F.h2[nt][e];
        DZ2[(size_t)r * kH + col] = dz2[nt][e];
        DZ1[(size_t)r * kH + col] = dh1[nt][e] * (1.f - h1 * h1);
      }
    if (t == 0)
      for (int row = 0; row < 2; ++row) {
        const int r = tile * 16 + g + 8 * row;
        if (r < nb)
          for (int o = 0; o < 3; ++o) DY[(size_t)r * 3 + o] = dy[row][o];
      }
  }
  for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
  if (lane == 0) atomicAdd(loss, lsum);
}

// Weight gradients from the stored activations: one thread per parameter,
// FP32 sums over the mini-batch.
__global__ void k_wgrad(const float *__restrict__ X, int i0, int nb, const float *__restrict__ H1,
                        const float *__restrict__ H2, const float *__restrict__ DZ1,
                        const float *__restrict__ DZ2, const float *__restrict__ DY,
                        float *__restrict__ G) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kNP) return;
  float s = 0.f;
  if (p < oB1) {  // W1[i][k] = sum x_i dz1_k
    const int i = p / kH, k = p % kH;
    for (int r = 0; r < nb; ++r) s = fmaf(net_input(X, i0 + r, i), DZ1[(size_t)r * kH + k], s);
  } else if (p < oW2) {
    const int k = p - oB1;
    for (int r = 0; r < nb; ++r) s += DZ1[(size_t)r * kH + k];
  } else if (p < oB2) {  // W2[k][j] = sum h1_k dz2_j
    const int k = (p - oW2) / kH, j = (p - oW2) % kH;
    for (int r = 0; r < nb; ++r) s = fmaf(H1[(size_t)r * kH + k], DZ2[(size_t)r * kH + j], s);
  } else if (p < oW3) {
    const int j = p - oB2;
    for (int r = 0; r < nb; ++r) s += DZ2[(size_t)r * kH + j];
  } else if (p < oB3) {  // W3[j][o] = sum h2_j dy_o
    const int j = (p - oW3) / 3, o = (p - oW3) % 3;
    for (int r = 0; r < nb; ++r) s = fmaf(H2[(size_t)r * kH + j], DY[(size_t)r * 3 + o], s);
  } else {
    const int o = p - oB3;
    for (int r = 0; r < nb; ++r) s += DY[(size_t)r * 3 + o];
  }
  G[p] = s;
}

__global__ void k_adam(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ M,
                       float *__restrict__ V, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kNP) return;
  const float g = G[p];
  const float m = b1 * M[p] + (1.f - b1) * g;
  const float v = b2 * V[p] + (1.f - b2) * g * g;
  M[p] = m;
  V[p] = v;
  P[p] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace sur
}  // namespace fio

using namespace fio;
using namespace fio::sur;

struct fio_surrogate_s {
  int nmodes = 0;
  double *d_modes = nullptr;
  float *d_params = nullptr, *d_m = nullptr, *d_v = nullptr, *d_grad = nullptr;
  float s_tau = 1.f, s_d = 1.f;
  fio_surrogate_info info{};
  int device = 0;
};

namespace {

fio_status sfail(cudaError_t e, const char *what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FIO_ENOMEM : FIO_ECUDA;
}

#define SCK(expr, what)                         \
  do {                                          \
    cudaError_t e_ = (expr);                    \
    if (e_ != cudaSuccess) return sfail(e_, what); \
  } while (0)

struct Tmp {
  std::vector<void *> v;
  ~Tmp() {
    for (void *p : v) cudaFree(p);
  }
  template <typename T> cudaError_t alloc(T **p, size_t n) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(n * sizeof(T), 16));
    if (e == cudaSuccess) v.push_back(q);
    *p = (T *)q;
    return e;
  }
};

// Held-out judge: errors of the network against the plain evaluation.
fio_status judge(fio_surrogate_s *s, int n, uint64_t seed) {
  Tmp tmp;
  float *X, *Y;
  double *T;
  SCK(tmp.alloc(&X, (size_t)n * 4), "judge alloc");
  SCK(tmp.alloc(&Y, (size_t)n * 4), "judge alloc");
  SCK(tmp.alloc(&T, (size_t)n * 4), "judge alloc");
  k_samples<<<nblk(n, 256), 256>>>(s->d_modes, s->nmodes, n, seed, X, T);
  k_infer<<<std::min<unsigned>(nblk(n, 64), 2048), 128>>>(s->d_params, X, n, s->s_tau, s->s_d, Y);
  SCK(cudaGetLastError(), "judge kernels");
  std::vector<float> y((size_t)n * 4);
  std::vector<double> t((size_t)n * 4);
  SCK(cudaMemcpy(y.data(), Y, sizeof(float) * y.size(), cudaMemcpyDeviceToHost), "judge copy");
  SCK(cudaMemcpy(t.data(), T, sizeof(double) * t.size(), cudaMemcpyDeviceToHost), "judge copy");
  double mt = 0, md = 0, mth = 0, rt = 0, rr = 0;
  for (int i = 0; i < n; ++i) {
    const double et = std::abs(y[4 * i] - t[4 * i]);
    const double ed = std::max(std::abs(y[4 * i + 1] - t[4 * i + 1]), std::abs(y[4 * i + 2] - t[4 * i + 2]));
    const double eth = std::abs(y[4 * i + 3] - t[4 * i + 3]);
    mt = std::max(mt, et);
    md = std::max(md, ed);
    mth = std::max(mth, eth);
    rt += et * et;
    rr += t[4 * i] * t[4 * i];
  }
  s->info.heldout_tau_maxerr = mt;
  s->info.heldout_dx_maxerr = md;
  s->info.heldout_dtheta_maxerr = mth;
  s->info.heldout_tau_relrms = std::sqrt(rt / std::max(rr, 1e-300));
  return FIO_OK;
}

}  // namespace

extern "C" {

fio_status fio_surrogate_train(const fio_phase *phase, int nsamples, int epochs, int batch,
                               unsigned long long seed, fio_surrogate *out) {
  if (!out) return FIO_EINVAL;
  *out = nullptr;
  if (!phase || phase->kind != FIO_PHASE_TAU_MODES || phase->nmodes < 1 || !phase->params ||
      nsamples < 1024 || nsamples > (1 << 24) || epochs < 0 || epochs > 10000 || batch < 64 ||
      batch > (1 << 20)) {
    set_error("fio_surrogate_train: needs a tau-mode phase, 1024 <= nsamples <= 2^24, "
              "0 <= epochs <= 10000, 64 <= batch <= 2^20");
    return FIO_EINVAL;
  }
  for (int i = 0; i < 5 * phase->nmodes; ++i)
    if (!std::isfinite(phase->params[i])) {
      set_error("fio_surrogate_train: non-finite phase parameter");
      return FIO_EINVAL;
    }
  const auto t0 = std::chrono::steady_clock::now();
  fio_surrogate_s *s = new fio_surrogate_s();
  cudaGetDevice(&s->device);
  auto fail = [&](fio_status st) {
    fio_surrogate_destroy(s);
    return st;
  };
  s->nmodes = phase->nmodes;
  if (cudaMalloc(&s->d_modes, sizeof(double) * 5 * s->nmodes) != cudaSuccess ||
      cudaMalloc(&s->d_params, sizeof(float) * kNP) != cudaSuccess ||
      cudaMalloc(&s->d_m, sizeof(float) * kNP) != cudaSuccess ||
      cudaMalloc(&s->d_v, sizeof(float) * kNP) != cudaSuccess ||
      cudaMalloc(&s->d_grad, sizeof(float) * kNP) != cudaSuccess) {
    set_error("fio_surrogate_train: device allocation failed");
    return fail(FIO_ENOMEM);
  }
  cudaMemcpy(s->d_modes, phase->params, sizeof(double) * 5 * s->nmodes, cudaMemcpyHostToDevice);
  // Xavier-style initial weights from a seeded SplitMix64 stream
  std::vector<float> p0(kNP, 0.f);
  uint64_t st = seed ^ 0x5A5A5A5AULL;
  auto u01 = [&]() {
    uint64_t z = (st += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-53;
  };
  auto fill = [&](int off, int fan_in, int fan_out, int count) {
    const double a = std::sqrt(6.0 / (fan_in + fan_out));
    for (int i = 0; i < count; ++i) p0[off + i] = (float)((2 * u01() - 1) * a);
  };
  fill(oW1, 4, kH, 4 * kH);
  fill(oW2, kH, kH, kH * kH);
  fill(oW3, kH, 3, kH * 3);
  if (cudaMemcpy(s->d_params, p0.data(), sizeof(float) * kNP, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(s->d_m, 0, sizeof(float) * kNP) != cudaSuccess ||
      cudaMemset(s->d_v, 0, sizeof(float) * kNP) != cudaSuccess) {
    set_error("fio_surrogate_train: upload failed");
    return fail(FIO_ECUDA);
  }
  {
    Tmp tmp;
    float *X, *Ts, *H1, *H2, *DZ1, *DZ2, *DY;
    double *T, *dloss;
    const size_t n = (size_t)nsamples, nb = (size_t)std::min(batch, nsamples);
    if (tmp.alloc(&X, n * 4) || tmp.alloc(&T, n * 4) || tmp.alloc(&Ts, n * 3) ||
        tmp.alloc(&H1, nb * kH) || tmp.alloc(&H2, nb * kH) || tmp.alloc(&DZ1, nb * kH) ||
        tmp.alloc(&DZ2, nb * kH) || tmp.alloc(&DY, nb * 3) || tmp.alloc(&dloss, 1)) {
      set_error("fio_surrogate_train: device allocation failed");
      return fail(FIO_ENOMEM);
    }
    k_samples<<<nblk(n, 256), 256>>>(s->d_modes, s->nmodes, (int)n, seed, X, T);
    // output scales: RMS of tau and of its x-derivatives over the samples
    std::vector<double> th(n * 4);
    if (cudaMemcpy(th.data(), T, sizeof(double) * th.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
      set_error("fio_surrogate_train: sample generation failed");
      return fail(FIO_ECUDA);
    }
    double st2 = 0, sd2 = 0;
    for (size_t i = 0; i < n; ++i) {
      st2 += th[4 * i] * th[4 * i];
      sd2 += 0.5 * (th[4 * i + 1] * th[4 * i + 1] + th[4 * i + 2] * th[4 * i + 2]);
    }
    s->s_tau = (float)std::sqrt(std::max(st2 / n, 1e-30));
    s->s_d = (float)std::sqrt(std::max(sd2 / n, 1e-30));
    k_scale_targets<<<nblk(n, 256), 256>>>(T, (int)n, s->s_tau, s->s_d, Ts);
    const float lr0 = 1e-2f, b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    long long step = 0;
    const long long total = (long long)epochs * ((n + nb - 1) / nb);
    double last = 0;
    for (int ep = 0; ep < epochs; ++ep) {
      cudaMemset(dloss, 0, sizeof(double));
      for (size_t i0 = 0; i0 < n; i0 += nb) {
        const int cnt = (int)std::min(nb, n - i0);
        k_train_fb<<<std::min<unsigned>(nblk(cnt, 64), 1024), 128>>>(
            s->d_params, X, Ts, (int)i0, cnt, H1, H2, DZ1, DZ2, DY, dloss);
        k_wgrad<<<nblk(kNP, 128), 128>>>(X, (int)i0, cnt, H1, H2, DZ1, DZ2, DY, s->d_grad);
        ++step;
        // cosine decay of the learning rate
        const float lr = lr0 * 0.5f * (1.f + std::cos((float)M_PI * (float)step / (float)std::max(total, 1LL)));
        k_adam<<<nblk(kNP, 256), 256>>>(s->d_params, s->d_grad, s->d_m, s->d_v, lr, b1, b2, eps,
                                       1.f - std::pow(b1, (float)step), 1.f - std::pow(b2, (float)step));
      }
      if (ep == epochs - 1) {
        if (cudaMemcpy(&last, dloss, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
          set_error("fio_surrogate_train: training failed");
          return fail(FIO_ECUDA);
        }
      }
    }
    if (cudaDeviceSynchronize() != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      set_error("fio_surrogate_train: training kernels failed");
      return fail(FIO_ECUDA);
    }
    s->info.final_loss = last / (double)n;
    s->info.steps = step;
  }
  s->info.nparams = kNP;
  s->info.nsamples = nsamples;
  s->info.epochs = epochs;
  s->info.tau_scale = s->s_tau;
  s->info.dx_scale = s->s_d;
  s->info.train_seconds =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  fio_status js = judge(s, 1 << 16, seed ^ 0xC0FFEEULL);
  if (js != FIO_OK) return fail(js);
  *out = s;
  return FIO_OK;
}

void fio_surrogate_destroy(fio_surrogate s) {
  if (!s) return;
  cudaFree(s->d_modes);
  cudaFree(s->d_params);
  cudaFree(s->d_m);
  cudaFree(s->d_v);
  cudaFree(s->d_grad);
  delete s;
}

fio_status fio_surrogate_get_info(fio_surrogate s, fio_surrogate_info *info) {
  if (!s || !info) return FIO_EINVAL;
  *info = s->info;
  return FIO_OK;
}

fio_status fio_surrogate_params(fio_surrogate s, float *params, int set) {
  if (!s || !params) return FIO_EINVAL;
  const cudaError_t e =
      set ? cudaMemcpy(s->d_params, params, sizeof(float) * kNP, cudaMemcpyHostToDevice)
          : cudaMemcpy(params, s->d_params, sizeof(float) * kNP, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? FIO_OK : sfail(e, "fio_surrogate_params");
}

fio_status fio_surrogate_eval(fio_surrogate s, int n, const float *x4, float *y4, void *stream) {
  if (!s || n < 1 || !x4 || !y4) return FIO_EINVAL;
  k_infer<<<std::min<unsigned>(nblk(n, 64), 4096), 128, 0, (cudaStream_t)stream>>>(
      s->d_params, x4, n, s->s_tau, s->s_d, y4);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FIO_OK : sfail(e, "fio_surrogate_eval");
}

fio_status fio_surrogate_loss_grad(fio_surrogate s, int n, const float *x4, const float *t3,
                                   float *grad, double *loss) {
  if (!s || n < 1 || !x4 || !t3 || !grad) return FIO_EINVAL;
  Tmp tmp;
  float *H1, *H2, *DZ1, *DZ2, *DY;
  double *dl;
  if (tmp.alloc(&H1, (size_t)n * kH) || tmp.alloc(&H2, (size_t)n * kH) ||
      tmp.alloc(&DZ1, (size_t)n * kH) || tmp.alloc(&DZ2, (size_t)n * kH) ||
      tmp.alloc(&DY, (size_t)n * 3) || tmp.alloc(&dl, 1)) {
    set_error("fio_surrogate_loss_grad: device allocation failed");
    return FIO_ENOMEM;
  }
  cudaMemset(dl, 0, sizeof(double));
  k_train_fb<<<std::min<unsigned>(nblk(n, 64), 1024), 128>>>(s->d_params, x4, t3, 0, n, H1, H2,
                                                            DZ1, DZ2, DY, dl);
  k_wgrad<<<nblk(kNP, 128), 128>>>(x4, 0, n, H1, H2, DZ1, DZ2, DY, grad);
  SCK(cudaDeviceSynchronize(), "fio_surrogate_loss_grad");
  double l = 0;
  SCK(cudaMemcpy(&l, dl, sizeof(double), cudaMemcpyDeviceToHost), "fio_surrogate_loss_grad");
  if (loss) *loss = l / n;
  return FIO_OK;
}

fio_status fio_surrogate_samples(const fio_phase *phase, int n, unsigned long long seed, float *x4,
                                 double *t4) {
  if (!phase || phase->kind != FIO_PHASE_TAU_MODES || n < 1 || !x4 || !t4) return FIO_EINVAL;
  Tmp tmp;
  double *dm;
  SCK(tmp.alloc(&dm, (size_t)5 * phase->nmodes), "fio_surrogate_samples");
  SCK(cudaMemcpy(dm, phase->params, sizeof(double) * 5 * phase->nmodes, cudaMemcpyHostToDevice),
      "fio_surrogate_samples");
  k_samples<<<nblk(n, 256), 256>>>(dm, phase->nmodes, n, seed, x4, t4);
  SCK(cudaDeviceSynchronize(), "fio_surrogate_samples");
  return FIO_OK;
}

int fio_surrogate_nparams(void) { return kNP; }

}  // extern "C"

namespace fio {
// Warped points from a surrogate (used by the plan when the judge allows it):
// y = x + tau xihat_l + d_theta tau xihat_l^perp at theta_l, reduced as in k_warp.
namespace {
__global__ void k_sur_inputs(int N, int L, float *X) {
  const long long NN = (long long)N * N;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= NN * L) return;
  const int l = (int)(idx / NN);
  const long long x = idx % NN;
  double st, ct;
  sincospi(2.0 * l / L, &st, &ct);
  X[4 * idx] = (float)((double)(x / N) / N);
  X[4 * idx + 1] = (float)((double)(x % N) / N);
  X[4 * idx + 2] = (float)ct;
  X[4 * idx + 3] = (float)st;
}
__global__ void k_sur_warp(int N, int L, const WedgeDev *__restrict__ W, const float *__restrict__ Y,
                           uint2 *__restrict__ warp) {
  const long long NN = (long long)N * N;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= NN * L) return;
  const int l = (int)(idx / NN);
  const long long x = idx % NN;
  const WedgeDev w = W[l];
  double st, ct;
  sincospi(2.0 * l / L, &st, &ct);
  const double tau = Y[4 * idx], dt = Y[4 * idx + 3];
  const double y1 = (double)(x / N) / N + tau * ct - dt * st;
  const double y2 = (double)(x % N) / N + tau * st + dt * ct;
  const double yp[2] = {w.Minv[0] * y1 + w.Minv[2] * y2, w.Minv[1] * y1 + w.Minv[3] * y2};
  uint32_t Yf[2];
  for (int d = 0; d < 2; ++d) {
    const double f = yp[d] - floor(yp[d]);
    const double s = rint(f * 4294967296.0);
    Yf[d] = s >= 4294967296.0 ? 0u : (uint32_t)s;
  }
  warp[idx] = make_uint2(Yf[0], Yf[1]);
}
}  // namespace

cudaError_t surrogate_warp(const fio_surrogate_s *s, int N, int L, const WedgeDev *d_w,
                           uint2 *d_warp) {
  const long long n = (long long)N * N * L;
  float *X = nullptr, *Y = nullptr;
  cudaError_t e = cudaMalloc(&X, sizeof(float) * 4 * n);
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&Y, sizeof(float) * 4 * n);
  if (e != cudaSuccess) {
    cudaFree(X);
    return e;
  }
  k_sur_inputs<<<sur::nblk(n, 256), 256>>>(N, L, X);
  // evaluate in chunks below 2^31 samples
  for (long long i0 = 0; i0 < n; i0 += (1LL << 30)) {
    const int cnt = (int)std::min<long long>(n - i0, 1LL << 30);
    sur::k_infer<<<std::min<unsigned>(sur::nblk(cnt, 64), 8192), 128>>>(
        s->d_params, X + 4 * i0, cnt, s->s_tau, s->s_d, Y + 4 * i0);
  }
  k_sur_warp<<<sur::nblk(n, 256), 256>>>(N, L, d_w, Y, d_warp);
  e = cudaDeviceSynchronize();
  cudaFree(X);
  cudaFree(Y);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

const fio_surrogate_info *surrogate_info(const fio_surrogate_s *s) { return &s->info; }

}  // namespace fio
