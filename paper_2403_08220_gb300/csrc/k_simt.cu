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

template <typename T, class Epi>
cudaError_t run_gemm(int M, int N, int K, const T *A, int lda, const T *B, int ldb, Epi epi,
                     cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
  k_gemm<T, Epi><<<grid, kGemmThreads, 0, st>>>(M, N, K, A, lda, B, ldb, epi);
  return cudaGetLastError();
}

// Prior draw: one CTA per chain; X = sqrt(Lambda) .* Z (spectral), Y = X S,
// M = S^T Y, all n x n in shared memory with rows padded to a multiple of 4
// (zero-filled).  Each product is computed in 4 x 4 register tiles: per step
// of the reduction a tile reads one float4 (or double4-as-two-loads) row
// segment of the right operand and four broadcast values of the left one.
// FP32 draws with at most kPriorWide tiles use a CTA of kPriorWide threads
// (four CTAs per SM), so that each product takes a single round; otherwise
// kPriorThreads threads loop over the tiles.
constexpr int kPriorThreads = 256;
constexpr int kPriorWide = 320;

__host__ __device__ inline int prior_ld(int n) { return (n + 3) / 4 * 4; }

// Four consecutive values of a padded shared-memory row (16-byte aligned: the
// rows are multiples of 4 values and the arrays start on 16 bytes).
template <typename T>
__device__ __forceinline__ void load4(const T *p, T v[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 x = *reinterpret_cast<const float4 *>(p);
    v[0] = x.x;
    v[1] = x.y;
    v[2] = x.z;
    v[3] = x.w;
  } else {
    const double2 x = reinterpret_cast<const double2 *>(p)[0];
    const double2 y = reinterpret_cast<const double2 *>(p)[1];
    v[0] = x.x;
    v[1] = x.y;
    v[2] = y.x;
    v[3] = y.y;
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT, NT == kPriorWide ? 4 : 1)
    k_prior_draw(int n, const T *__restrict__ sqrtlam, const T *__restrict__ S, uint64_t seed,
                 uint64_t id_base, uint32_t stream, uint32_t step, T *out, int ldo,
                 __nv_bfloat16 *ms, int ldms, size_t ms_plane, int ms_slices,
                 const double *__restrict__ ext_z, const int *__restrict__ only) {
  if (only && !only[blockIdx.x]) return;  // the whole CTA: this chain draws nothing
  extern __shared__ __align__(16) unsigned char smraw[];
  const int ld = prior_ld(n), nt = ld / 4, NN = ld * ld;
  T *X = reinterpret_cast<T *>(smraw);
  T *Ss = X + NN;
  T *Y = Ss + NN;
  const int c = blockIdx.x, N = n * n;
  const uint32_t chain = (uint32_t)(id_base + (uint64_t)c);
  // q / d for 0 <= q < d^2 + 4d, d <= 256, from the FP32 reciprocal: (q + 1/2) / d
  // stays at least 1/(2d) away from an integer, far beyond the rounding error
  // (rounded operations, no contraction)
  const float inv_ld = 1.0f / (float)ld, inv_n = 1.0f / (float)n;
  auto quot = [](int q, float inv) {
    return (int)__fmul_rn(__fadd_rn((float)q, 0.5f), inv);
  };
  for (int e = threadIdx.x; e < NN; e += blockDim.x) {
    const int row = quot(e, inv_ld), col = e - row * ld;
    const bool in = row < n && col < n;
    X[e] = T(0);
    Ss[e] = in ? S[row * n + col] : T(0);
  }
  __syncthreads();
  for (int blk = threadIdx.x; blk < (N + 3) / 4; blk += blockDim.x) {
    T z[4];
    if (ext_z) {
      for (int q = 0; q < 4; ++q)
        z[q] = 4 * blk + q < N ? (T)ext_z[(size_t)c * N + 4 * blk + q] : T(0);
    } else {
      const uint4 w = philox_block(seed, stream, step, chain, blk);
      if constexpr (sizeof(T) == 8) {
        normals4_f64(w, z);
      } else {
        normals4_f32(w, z);
      }
    }
    for (int q = 0; q < 4; ++q) {
      const int m = 4 * blk + q;
      if (m < N) {
        const int j = quot(m, inv_n);
        X[(m - j * n) * ld + j] = sqrtlam[m] * z[q];  // stored transposed
      }
    }
  }
  __syncthreads();
  // Y[ky][i] = sum_kx X[ky][kx] S[kx][i], with X held transposed (X[kx][ky]
  // at kx * ld + ky) so that both operands are read as row segments
  for (int tt = threadIdx.x; tt < nt * nt; tt += blockDim.x) {
    const int r0 = 4 * (tt / nt), c0 = 4 * (tt % nt);
    T acc[4][4] = {};
    for (int k = 0; k < n; ++k) {
      T a[4], b[4];
      load4(X + k * ld + r0, a);
      load4(Ss + k * ld + c0, b);
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
  // M[j][i] = sum_ky S[ky][j] Y[ky][i]; node p = i + n j.  The tiles land in
  // shared memory (X's array, which the first product no longer reads: n^2
  // nodes in order), and the CTA then writes M and its slices with
  // consecutive threads on consecutive nodes.
  T *Mo = X;
  for (int tt = threadIdx.x; tt < nt * nt; tt += blockDim.x) {
    const int r0 = 4 * (tt / nt), c0 = 4 * (tt % nt);
    T acc[4][4] = {};
    for (int k = 0; k < n; ++k) {
      T a[4], b[4];
      load4(Ss + k * ld + r0, a);
      load4(Y + k * ld + c0, b);
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] += a[p] * b[q];
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (r0 + p < n && c0 + q < n) Mo[(r0 + p) * n + c0 + q] = acc[p][q];
  }
  __syncthreads();
  T *o = out + (size_t)c * ldo;
  for (int e = threadIdx.x; e < N; e += blockDim.x) {
    const T v = Mo[e];
    o[e] = v;
    if constexpr (sizeof(T) == 4) {
      if (ms) {
        __nv_bfloat16 *d = ms + (size_t)c * ldms + e;
        float rem = v;
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
                      const double *coef, int ldc, double c, T *out, int ldo, cudaStream_t st) {
  return run_gemm(M, N, K, A, lda, B, ldb, EpiCoef<T>{coef, ldc, c, out, ldo}, st);
}

template <typename T>
cudaError_t gemm_field(int M, int N, int K, const T *A, int lda, const T *B, int ldb,
                       const int *acc_flag, double s, double c, T *m, const T *Mf, int ldm,
                       cudaStream_t st) {
  return run_gemm(M, N, K, A, lda, B, ldb, EpiField<T>{acc_flag, s, c, m, Mf, ldm}, st);
}

template <typename T>
__global__ void k_batched_transpose(int C, int a, int b, const T *__restrict__ src,
                                    T *__restrict__ dst) {
  const size_t blk = (size_t)a * b, n = (size_t)C * blk;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t c = e / blk, rem = e - c * blk, i = rem / a, j = rem - i * a;
    dst[e] = src[c * blk + j * b + i];  // dst (c, i < b, j < a) = src (c, j, i)
  }
}

cudaError_t launch_batched_transpose(int C, int a, int b, const void *src, int f32, void *dst,
                                     cudaStream_t st) {
  const size_t n = (size_t)C * a * b;
  if (n == 0) return cudaSuccess;
  const int grid = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
  if (f32)
    k_batched_transpose<float><<<grid, 256, 0, st>>>(C, a, b, (const float *)src, (float *)dst);
  else
    k_batched_transpose<double><<<grid, 256, 0, st>>>(C, a, b, (const double *)src,
                                                      (double *)dst);
  return cudaGetLastError();
}

// Eight independent FMA chains per thread: with 8 warps per scheduler the
// chains' latency is hidden and the FP32 pipe runs at its issue rate.
constexpr int kFmaIters = 8192;
__global__ void __launch_bounds__(256) k_fma_peak(float seed, float *out) {
  float a[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = seed * (float)(threadIdx.x + q);
  const float b = 0.999999f, c = 1e-7f;
#pragma unroll 4
  for (int it = 0; it < kFmaIters; ++it)
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = fmaf(a[q], b, c);
  float s = 0.0f;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += a[q];
  if (s == 12345.678f) out[0] = s;  // keeps the chains alive
}

cudaError_t measure_fma_peak(cudaStream_t st, float *ms, double *flops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = sms * 8;  // 2048 threads per SM
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  float best = 0.0f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, st);
    k_fma_peak<<<blocks, 256, 0, st>>>(1e-3f, nullptr);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    float t = 0.0f;
    if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
    if (rep > 0 && (best == 0.0f || t < best)) best = t;  // the first launch warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = best;
  *flops = 2.0 * 8.0 * kFmaIters * (double)blocks * 256.0;
  return e;
}

size_t prior_draw_smem_bytes(int n, int elem) {
  return 3 * (size_t)prior_ld(n) * prior_ld(n) * elem;
}

template <typename T>
cudaError_t launch_prior_draw(int C, int n, const T *sqrtlam, const T *S, uint64_t seed,
                              uint64_t id_base, uint32_t stream, uint32_t step, T *out, int ldo,
                              cudaStream_t st, __nv_bfloat16 *ms, int ldms, size_t ms_plane,
                              int ms_slices, const double *ext_z, const int *only) {
  if (C <= 0) return cudaSuccess;
  if (ms && (sizeof(T) != 4 || ms_slices < 1 || ldms < n * n)) return cudaErrorInvalidValue;
  const size_t smem = prior_draw_smem_bytes(n, (int)sizeof(T));
  const int nt = prior_ld(n) / 4;
  auto go = [&](auto kernel, int threads) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kernel<<<C, threads, smem, st>>>(n, sqrtlam, S, seed, id_base, stream, step, out, ldo, ms,
                                     ldms, ms_plane, ms_slices, ext_z, only);
    return cudaGetLastError();
  };
  if constexpr (sizeof(T) == 4)
    if (nt * nt <= kPriorWide) return go(k_prior_draw<T, kPriorWide>, kPriorWide);
  return go(k_prior_draw<T, kPriorThreads>, kPriorThreads);
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

// The SIMT GEMMs serve the FP64 path; the prior draw both paths.
template cudaError_t gemm_store<double>(int, int, int, const double *, int, const double *, int,
                                        double *, int, cudaStream_t);
template cudaError_t gemm_bias_act<double>(int, int, int, const double *, int, const double *,
                                           int, const double *, int, double *, double *, int,
                                           cudaStream_t);
template cudaError_t gemm_scale_group<double>(int, int, int, const double *, int, const double *,
                                              int, const double *, int, int, double *, int,
                                              cudaStream_t);
template cudaError_t gemm_coef<double>(int, int, int, const double *, int, const double *, int,
                                       const double *, int, double, double *, int, cudaStream_t);
template cudaError_t gemm_field<double>(int, int, int, const double *, int, const double *, int,
                                        const int *, double, double, double *, const double *,
                                        int, cudaStream_t);
template cudaError_t launch_jac_init<double>(int, int, int, const double *, const double *, int,
                                             double *, cudaStream_t);
template cudaError_t launch_broadcast<double>(int, size_t, const double *, double *,
                                              cudaStream_t);
#define DINO_INST_DRAW(T)                                                                     \
  template cudaError_t launch_prior_draw<T>(int, int, const T *, const T *, uint64_t,         \
                                            uint64_t, uint32_t, uint32_t, T *, int,           \
                                            cudaStream_t, __nv_bfloat16 *, int, size_t, int, \
                                            const double *, const int *);
DINO_INST_DRAW(double)
DINO_INST_DRAW(float)

}  // namespace dino
