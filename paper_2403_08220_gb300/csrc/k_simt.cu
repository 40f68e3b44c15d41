// SIMT kernels of the sampler: FP64/FP32 tiled GEMMs with fused epilogues
// (MLP layers, reverse-mode Jacobian products, complement projection and
// field update), the full-KLE prior draw, and small elementwise helpers.
//
// GEMM convention: out = epilogue(A B^T) with A: M x K (row pitch lda) and
// B: N x K (row pitch ldb), i.e. both operands K-contiguous.
#include <algorithm>

#include "dino_internal.h"
#include "philox.cuh"

namespace dino {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4, kGemmThreads = 256;

template <typename T>
__device__ __forceinline__ T act_fn(int kind, T z) {
  if (kind == 1) return tanh(z);
  if (kind == 2) return T(0.5) * z * (T(1) + erf(z * T(0.70710678118654752440)));
  return z;
}

template <typename T>
__device__ __forceinline__ T act_deriv(int kind, T z) {
  if (kind == 1) {
    const T t = tanh(z);
    return T(1) - t * t;
  }
  if (kind == 2)
    return T(0.5) * (T(1) + erf(z * T(0.70710678118654752440))) +
           z * exp(T(-0.5) * z * z) * T(0.39894228040143267794);
  return T(1);
}

// Tiled GEMM: each thread owns a TM x TN block of outputs, strided by 16 so
// that the shared-memory reads of a warp fall in distinct banks.
template <typename T, class Epi>
__global__ void __launch_bounds__(kGemmThreads)
    k_gemm(int M, int N, int K, const T *__restrict__ A, int lda, const T *__restrict__ B,
           int ldb, Epi epi) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += kGemmThreads) {
      const int m = e / BK, k = e % BK, gr = row0 + m, gk = k0 + k;
      As[k][m] = (gr < M && gk < K) ? A[(size_t)gr * lda + gk] : T(0);
    }
    for (int e = tid; e < BN * BK; e += kGemmThreads) {
      const int n = e / BK, k = e % BK, gc = col0 + n, gk = k0 + k;
      Bs[k][n] = (gc < N && gk < K) ? B[(size_t)gc * ldb + gk] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
      if (r < M && c < N) epi(r, c, acc[i][j]);
    }
}

template <typename T>
struct EpiStore {
  T *out;
  int ldo;
  __device__ void operator()(int r, int c, T v) const { out[(size_t)r * ldo + c] = v; }
};

template <typename T>
struct EpiBiasAct {
  const T *bias;
  int act;
  T *out, *der;
  int ldo;
  __device__ void operator()(int r, int c, T v) const {
    const T z = v + bias[c];
    out[(size_t)r * ldo + c] = act_fn(act, z);
    if (der) der[(size_t)r * ldo + c] = act_deriv(act, z);
  }
};

template <typename T>
struct EpiScaleGroup {
  const T *scale;
  int lds, group;
  T *out;
  int ldo;
  __device__ void operator()(int r, int c, T v) const {
    out[(size_t)r * ldo + c] = v * scale[(size_t)(r / group) * lds + c];
  }
};

template <typename T>
struct EpiCoef {
  const double *coef;
  int ldc;
  double cs;
  T *out;
  int ldo;
  __device__ void operator()(int r, int c, T v) const {
    out[(size_t)r * ldo + c] = (T)(coef[(size_t)r * ldc + c] - cs * (double)v);
  }
};

template <typename T>
struct EpiField {
  const int *acc;
  double s, cs;
  T *m;
  const T *Mf;
  int ldm;
  __device__ void operator()(int r, int c, T v) const {
    if (!acc[r]) return;
    const size_t o = (size_t)r * ldm + c;
    m[o] = (T)(s * (double)m[o] + cs * (double)Mf[o]) + v;
  }
};

// FP32 GEMM in 128 x 128 tiles, 8 x 8 outputs per thread (rows 8 ty.., columns
// 8 tx..): per step of the reduction a thread reads two float4 of A and two of
// B from shared memory for 64 FMAs, which balances the shared-memory and FMA
// rates.  Operands are staged K-major ([k][m], [k][n]) in slices of BK2; the
// next slice is loaded into registers while the current one is used.
constexpr int BM2 = 128, BN2 = 128, BK2 = 8;

// With gridDim.z > 1 the CTA at z covers K range [z kchunk, (z + 1) kchunk).
template <class Epi>
__global__ void __launch_bounds__(kGemmThreads)
    k_gemm_f32_big(int M, int N, int K, const float *__restrict__ A, int lda,
                   const float *__restrict__ B, int ldb, Epi epi, int kchunk) {
  __shared__ __align__(16) float As[2][BK2][BM2];
  __shared__ __align__(16) float Bs[2][BK2][BN2];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int row0 = blockIdx.y * BM2, col0 = blockIdx.x * BN2;
  // each thread stages 4 elements of A and 4 of B per slice: (m, k) = (tid / 2, 4 (tid % 2) + q)
  const int lm = tid / 2, lk = 4 * (tid % 2);
  float ra[4], rb[4];
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      As[buf][lk + q][lm] = ra[q];
      Bs[buf][lk + q][lm] = rb[q];
    }
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  // loads past kend read zeros (gk < kend); A and B are read only below K
  auto loadk = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gk = k0 + lk + q;
      const int gr = row0 + lm, gc = col0 + lm;
      ra[q] = (gr < M && gk < kend) ? A[(size_t)gr * lda + gk] : 0.0f;
      rb[q] = (gc < N && gk < kend) ? B[(size_t)gc * ldb + gk] : 0.0f;
    }
  };
  loadk(kbeg);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = kbeg; k0 < kend; k0 += BK2) {
    const bool more = k0 + BK2 < kend;
    if (more) loadk(k0 + BK2);
#pragma unroll
    for (int k = 0; k < BK2; ++k) {
      const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][8 * ty]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][8 * ty + 4]);
      const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][k][8 * tx]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][k][8 * tx + 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int r = row0 + 8 * ty + i, c = col0 + 8 * tx + j;
      if (r < M && c < N) epi(r, c, acc[i][j]);
    }
}

template <typename T, class Epi>
cudaError_t run_gemm(int M, int N, int K, const T *A, int lda, const T *B, int ldb, Epi epi,
                     cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if constexpr (sizeof(T) == 4) {
    dim3 grid((N + BN2 - 1) / BN2, (M + BM2 - 1) / BM2);
    k_gemm_f32_big<Epi><<<grid, kGemmThreads, 0, st>>>(M, N, K, A, lda, B, ldb, epi, K);
  } else {
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    k_gemm<T, Epi><<<grid, kGemmThreads, 0, st>>>(M, N, K, A, lda, B, ldb, epi);
  }
  return cudaGetLastError();
}

// Prior draw: one CTA per chain; X = sqrt(Lambda) .* Z (spectral), Y = X S,
// M = S^T Y, all n x n in shared memory with rows padded to a multiple of 4
// (zero-filled).  Each product is computed in 4 x 4 register tiles: per step
// of the reduction a tile reads one float4 (or double4-as-two-loads) row
// segment of the right operand and four broadcast values of the left one.
constexpr int kPriorThreads = 256;

__host__ __device__ inline int prior_ld(int n) { return (n + 3) / 4 * 4; }

template <typename T>
__global__ void __launch_bounds__(kPriorThreads)
    k_prior_draw(int n, const T *__restrict__ sqrtlam, const T *__restrict__ S, uint64_t seed,
                 uint64_t id_base, uint32_t stream, uint32_t step, T *out, int ldo,
                 __nv_bfloat16 *ms, int ldms, size_t ms_plane, int ms_slices) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int ld = prior_ld(n), nt = ld / 4, NN = ld * ld;
  T *X = reinterpret_cast<T *>(smraw);
  T *Ss = X + NN;
  T *Y = Ss + NN;
  const int c = blockIdx.x, N = n * n;
  const uint32_t chain = (uint32_t)(id_base + (uint64_t)c);
  for (int e = threadIdx.x; e < NN; e += blockDim.x) {
    const int row = e / ld, col = e % ld;
    const bool in = row < n && col < n;
    X[e] = T(0);
    Ss[e] = in ? S[row * n + col] : T(0);
  }
  __syncthreads();
  for (int blk = threadIdx.x; blk < (N + 3) / 4; blk += blockDim.x) {
    const uint4 w = philox_block(seed, stream, step, chain, blk);
    T z[4];
    if constexpr (sizeof(T) == 8) {
      normals4_f64(w, z);
    } else {
      normals4_f32(w, z);
    }
    for (int q = 0; q < 4; ++q) {
      const int m = 4 * blk + q;
      if (m < N) X[(m / n) * ld + m % n] = sqrtlam[m] * z[q];
    }
  }
  __syncthreads();
  // Y[ky][i] = sum_kx X[ky][kx] S[kx][i]
  for (int tt = threadIdx.x; tt < nt * nt; tt += blockDim.x) {
    const int r0 = 4 * (tt / nt), c0 = 4 * (tt % nt);
    T acc[4][4] = {};
    for (int k = 0; k < n; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) a[p] = X[(r0 + p) * ld + k];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Ss[k * ld + c0 + q];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] += a[p] * b[q];
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) Y[(r0 + p) * ld + c0 + q] = acc[p][q];
  }
  __syncthreads();
  // M[j][i] = sum_ky S[ky][j] Y[ky][i]; node p = i + n j
  T *o = out + (size_t)c * ldo;
  for (int tt = threadIdx.x; tt < nt * nt; tt += blockDim.x) {
    const int r0 = 4 * (tt / nt), c0 = 4 * (tt % nt);
    T acc[4][4] = {};
    for (int k = 0; k < n; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) a[p] = Ss[k * ld + r0 + p];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Y[k * ld + c0 + q];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] += a[p] * b[q];
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (r0 + p < n && c0 + q < n) {
          o[(r0 + p) * n + c0 + q] = acc[p][q];
          if constexpr (sizeof(T) == 4) {
            if (ms) {
              __nv_bfloat16 *d = ms + (size_t)c * ldms + (r0 + p) * n + c0 + q;
              float rem = acc[p][q];
              for (int sl = 0; sl < ms_slices; ++sl) {
                const __nv_bfloat16 hb = __float2bfloat16_rn(rem);
                d[sl * ms_plane] = hb;
                // exact widening: the bf16 bits in the upper half of an FP32 word
                rem -= __uint_as_float((uint32_t)__bfloat16_as_ushort(hb) << 16);
              }
            }
          }
        }
  }
}

template <typename T>
__global__ void k_jac_init(int C, int d_y, int w, const T *__restrict__ WL,
                           const T *__restrict__ der, int ldd, T *__restrict__ P) {
  const size_t total = (size_t)C * d_y * w;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t row = e / w;
    const int k = (int)(e % w);
    const size_t c = row / d_y;
    const int i = (int)(row % d_y);
    P[e] = WL[(size_t)i * w + k] * der[c * ldd + k];
  }
}

template <typename T>
__global__ void k_broadcast(int C, size_t n, const T *__restrict__ src, T *__restrict__ out) {
  const size_t total = (size_t)C * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x)
    out[e] = src[e % n];
}

template <typename S, typename D>
__global__ void k_convert(size_t n, const S *__restrict__ src, D *__restrict__ dst) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    dst[e] = (D)src[e];
}

inline int grid_for(size_t n) {
  size_t g = (n + 255) / 256;
  return (int)(g > 152 * 32 ? 152 * 32 : (g ? g : 1));
}

}  // namespace

// Split-K FP32 GEMM for small M x N with long K: partial sums of `splits`
// K ranges go to ws (splits x M x N), then one pass sums them and applies the
// epilogue.
struct EpiPartial {
  float *ws;
  int M, N;
  __device__ void operator()(int r, int c, float v) const {
    ws[((size_t)blockIdx.z * M + r) * N + c] = v;
  }
};

template <class Epi>
__global__ void k_splitk_finish(int M, int N, int splits, const float *__restrict__ ws, Epi epi) {
  const size_t total = (size_t)M * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int z = 0; z < splits; ++z) s += ws[(size_t)z * total + e];
    epi((int)(e / N), (int)(e % N), s);
  }
}

template <class Epi>
cudaError_t run_gemm_splitk_f32(int M, int N, int K, const float *A, int lda, const float *B,
                                int ldb, Epi epi, float *ws, size_t ws_floats, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const int tiles = ((N + BN2 - 1) / BN2) * ((M + BM2 - 1) / BM2);
  int splits = (6 * 152 + tiles - 1) / tiles;
  splits = std::max(1, std::min({splits, 8, (K + 255) / 256}));
  while (splits > 1 && (size_t)splits * M * N > ws_floats) --splits;
  if (splits == 1 || !ws) return run_gemm<float, Epi>(M, N, K, A, lda, B, ldb, epi, st);
  const int kchunk = ((K + splits - 1) / splits + BK2 - 1) / BK2 * BK2;
  dim3 grid((N + BN2 - 1) / BN2, (M + BM2 - 1) / BM2, splits);
  k_gemm_f32_big<EpiPartial>
      <<<grid, kGemmThreads, 0, st>>>(M, N, K, A, lda, B, ldb, EpiPartial{ws, M, N}, kchunk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_splitk_finish<Epi><<<grid_for((size_t)M * N), 256, 0, st>>>(M, N, splits, ws, epi);
  return cudaGetLastError();
}

template <typename T>
cudaError_t gemm_store(int M, int N, int K, const T *A, int lda, const T *B, int ldb, T *out,
                       int ldo, cudaStream_t st) {
  return run_gemm(M, N, K, A, lda, B, ldb, EpiStore<T>{out, ldo}, st);
}

template <typename T>
cudaError_t gemm_bias_act(int M, int N, int K, const T *A, int lda, const T *B, int ldb,
                          const T *bias, int act, T *out, T *der, int ldo, cudaStream_t st) {
  return run_gemm(M, N, K, A, lda, B, ldb, EpiBiasAct<T>{bias, act, out, der, ldo}, st);
}

template <typename T>
cudaError_t gemm_scale_group(int M, int N, int K, const T *A, int lda, const T *B, int ldb,
                             const T *scale, int lds, int group, T *out, int ldo,
                             cudaStream_t st) {
  return run_gemm(M, N, K, A, lda, B, ldb, EpiScaleGroup<T>{scale, lds, group, out, ldo}, st);
}

template <typename T>
cudaError_t gemm_coef(int M, int N, int K, const T *A, int lda, const T *B, int ldb,
                      const double *coef, int ldc, double c, T *out, int ldo, cudaStream_t st,
                      float *ws, size_t ws_floats) {
  if constexpr (sizeof(T) == 4)
    return run_gemm_splitk_f32(M, N, K, A, lda, B, ldb, EpiCoef<T>{coef, ldc, c, out, ldo}, ws,
                               ws_floats, st);
  return run_gemm(M, N, K, A, lda, B, ldb, EpiCoef<T>{coef, ldc, c, out, ldo}, st);
}

template <typename T>
cudaError_t gemm_field(int M, int N, int K, const T *A, int lda, const T *B, int ldb,
                       const int *acc_flag, double s, double c, T *m, const T *Mf, int ldm,
                       cudaStream_t st) {
  return run_gemm(M, N, K, A, lda, B, ldb, EpiField<T>{acc_flag, s, c, m, Mf, ldm}, st);
}

size_t prior_draw_smem_bytes(int n, int elem) {
  return 3 * (size_t)prior_ld(n) * prior_ld(n) * elem;
}

template <typename T>
cudaError_t launch_prior_draw(int C, int n, const T *sqrtlam, const T *S, uint64_t seed,
                              uint64_t id_base, uint32_t stream, uint32_t step, T *out, int ldo,
                              cudaStream_t st, __nv_bfloat16 *ms, int ldms, size_t ms_plane,
                              int ms_slices) {
  if (C <= 0) return cudaSuccess;
  if (ms && (sizeof(T) != 4 || ms_slices < 1 || ldms < n * n)) return cudaErrorInvalidValue;
  const size_t smem = prior_draw_smem_bytes(n, (int)sizeof(T));
  cudaError_t e = cudaFuncSetAttribute(k_prior_draw<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_prior_draw<T><<<C, kPriorThreads, smem, st>>>(n, sqrtlam, S, seed, id_base, stream, step, out,
                                                   ldo, ms, ldms, ms_plane, ms_slices);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_jac_init(int C, int d_y, int w, const T *WL, const T *der, int ldd, T *P,
                            cudaStream_t st) {
  k_jac_init<T><<<grid_for((size_t)C * d_y * w), 256, 0, st>>>(C, d_y, w, WL, der, ldd, P);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_broadcast(int C, size_t n, const T *src, T *out, cudaStream_t st) {
  k_broadcast<T><<<grid_for((size_t)C * n), 256, 0, st>>>(C, n, src, out);
  return cudaGetLastError();
}

cudaError_t launch_copy_f64(size_t n, const double *src, double *dst, cudaStream_t st) {
  k_convert<double, double><<<grid_for(n), 256, 0, st>>>(n, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_f64_to_f32(size_t n, const double *src, float *dst, cudaStream_t st) {
  k_convert<double, float><<<grid_for(n), 256, 0, st>>>(n, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(size_t n, const float *src, double *dst, cudaStream_t st) {
  k_convert<float, double><<<grid_for(n), 256, 0, st>>>(n, src, dst);
  return cudaGetLastError();
}

#define DINO_INST(T)                                                                          \
  template cudaError_t gemm_store<T>(int, int, int, const T *, int, const T *, int, T *, int, \
                                     cudaStream_t);                                           \
  template cudaError_t gemm_bias_act<T>(int, int, int, const T *, int, const T *, int,        \
                                        const T *, int, T *, T *, int, cudaStream_t);         \
  template cudaError_t gemm_scale_group<T>(int, int, int, const T *, int, const T *, int,     \
                                           const T *, int, int, T *, int, cudaStream_t);      \
  template cudaError_t gemm_coef<T>(int, int, int, const T *, int, const T *, int,            \
                                    const double *, int, double, T *, int, cudaStream_t,      \
                                    float *, size_t);                                         \
  template cudaError_t gemm_field<T>(int, int, int, const T *, int, const T *, int,           \
                                     const int *, double, double, T *, const T *, int,        \
                                     cudaStream_t);                                           \
  template cudaError_t launch_prior_draw<T>(int, int, const T *, const T *, uint64_t,         \
                                            uint64_t, uint32_t, uint32_t, T *, int,           \
                                            cudaStream_t, __nv_bfloat16 *, int, size_t, int); \
  template cudaError_t launch_jac_init<T>(int, int, int, const T *, const T *, int, T *,      \
                                          cudaStream_t);                                      \
  template cudaError_t launch_broadcast<T>(int, size_t, const T *, T *, cudaStream_t);

DINO_INST(double)
DINO_INST(float)

}  // namespace dino
