// Markov-chain diagnostics on the device (Sec. 6.2): a recorded trajectory of
// n_c chains x n_s samples x d degrees of freedom, stored per degree of
// freedom and chain so that each series is contiguous:
//   traj[(i n_c + k) max_s + j] = x_{j,k}(i).
//
//   k_diag_record   appends one sample of every chain (from a pool's state or
//                   a caller buffer);
//   k_diag_ess      one CTA per degree of freedom: chain means and variances,
//                   w and v (the 1D covariance estimators), the multi-chain
//                   autocorrelation MACT(t) = 1 - (w - mean_k AC(t,k)) / v lag
//                   pair by lag pair until the pair sum is no longer positive
//                   (the initial positive sequence), ESS% = 1 / (1 + 2 sum_t
//                   MACT(t)) (eq:ess), and the squared jumps of the MSJ;
//   k_diag_center   centred samples and centred chain means (d x n_c n_s and
//                   d x n_c) whose Gram products give W and V
//                   (eq:covariance_estimator);
//   k_jacobi        one-sided Jacobi (Hestenes) on a d x d matrix held by
//                   columns: column pairs are rotated until orthogonal, in
//                   round-robin order so that the d/2 pairs of a round are
//                   disjoint and run on separate warps; for a symmetric
//                   positive semidefinite matrix the final column norms are
//                   its eigenvalues and the accumulated rotations its
//                   eigenvectors;
//   k_sym_sqrt, k_mm  the square root Q diag(sqrt(lambda)) Q^T and the small
//                   products of the Wasserstein MPSRF
//                   Tr(W + V - 2 (W^1/2 V W^1/2)^1/2);
//   k_normals, k_transpose  the encoded prior draws and the stacked transposed
//                   Jacobian of the surrogate-driven DIS basis (eq:mc_ppgnh),
//                   whose eigenproblem the same Jacobi kernel solves.
// Every loop is bounded by the sizes (lags by n_s, Jacobi sweeps by
// kMaxSweeps); no kernel waits on another CTA.
#include <algorithm>

#include "chol.cuh"

namespace dino {
namespace {

constexpr int kEssThreads = 256;
constexpr int kJacobiThreads = 1024;

template <typename T>
__global__ void k_diag_record(int n_c, int d, const T *__restrict__ src, int ld_src,
                              double *__restrict__ traj, int max_s, int j) {
  const size_t n = (size_t)n_c * d;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t k = e / d, i = e - k * d;  // source row k (chain), column i (dof)
    traj[(i * n_c + k) * max_s + j] = (double)src[k * ld_src + i];
  }
}

// Sum over the CTA of two values (every thread gets both); red >= 66 doubles.
__device__ void block_sum2(double &x, double &y, double *red) {
  for (int o = 16; o; o >>= 1) {
    x += __shfl_xor_sync(kFull, x, o);
    y += __shfl_xor_sync(kFull, y, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) {
    red[warp] = x;
    red[32 + warp] = y;
  }
  __syncthreads();
  if (warp == 0) {
    double a = lane < nw ? red[lane] : 0.0, b = lane < nw ? red[32 + lane] : 0.0;
    for (int o = 16; o; o >>= 1) {
      a += __shfl_xor_sync(kFull, a, o);
      b += __shfl_xor_sync(kFull, b, o);
    }
    if (lane == 0) {
      red[64] = a;
      red[65] = b;
    }
  }
  __syncthreads();
  x = red[64];
  y = red[65];
}

// Dynamic shared memory: n_c chain means.
__global__ void __launch_bounds__(kEssThreads)
    k_diag_ess(int n_c, int n_s, const double *__restrict__ traj, int max_s,
               double *__restrict__ means, double *__restrict__ ess, double *__restrict__ sqjump) {
  extern __shared__ double mk[];
  __shared__ double red[72];
  const int i = blockIdx.x;
  const double *X = traj + (size_t)i * n_c * max_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // chain means (warp per chain)
  for (int k = warp; k < n_c; k += nw) {
    double s = 0.0;
    for (int j = lane; j < n_s; j += 32) s += X[(size_t)k * max_s + j];
    s = warp_sum(s);
    if (lane == 0) mk[k] = s / n_s;
  }
  __syncthreads();
  // within-chain sums of squares and squared jumps
  double ss = 0.0, jj = 0.0;
  const size_t tot = (size_t)n_c * n_s;
  for (size_t e = threadIdx.x; e < tot; e += blockDim.x) {
    const int k = (int)(e / n_s), j = (int)(e - (size_t)k * n_s);
    const double x = X[(size_t)k * max_s + j] - mk[k];
    ss += x * x;
    if (j + 1 < n_s) {
      const double dx = X[(size_t)k * max_s + j + 1] - X[(size_t)k * max_s + j];
      jj += dx * dx;
    }
  }
  block_sum2(ss, jj, red);
  double gm = 0.0;
  for (int k = 0; k < n_c; ++k) gm += mk[k];
  gm /= n_c;
  double bs = 0.0;
  for (int k = 0; k < n_c; ++k) bs += (mk[k] - gm) * (mk[k] - gm);
  const double w = ss / ((double)n_c * (n_s - 1));
  const double v = (double)(n_s - 1) / n_s * w + (double)(n_c + 1) / ((double)n_c * (n_c - 1)) * bs;
  // MACT(t) for lag pairs (2m, 2m + 1), MACT(0) = 1, while the pair sum is positive
  double total = 0.0;
  int pairs = 0;
  for (int m = 0; 2 * m + 1 < n_s; ++m) {
    double a0 = 0.0, a1 = 0.0;
    const int t0 = 2 * m, t1 = 2 * m + 1;
    for (size_t e = threadIdx.x; e < tot; e += blockDim.x) {
      const int k = (int)(e / n_s), j = (int)(e - (size_t)k * n_s);
      const double *xs = X + (size_t)k * max_s;
      const double x = xs[j] - mk[k];
      if (t0 > 0 && j + t0 < n_s) a0 += x * (xs[j + t0] - mk[k]);
      if (j + t1 < n_s) a1 += x * (xs[j + t1] - mk[k]);
    }
    block_sum2(a0, a1, red);
    const double r0 = t0 == 0 ? 1.0 : 1.0 - (w - a0 / ((double)n_s * n_c)) / v;
    const double r1 = 1.0 - (w - a1 / ((double)n_s * n_c)) / v;
    const double pair = r0 + r1;
    if (!(pair > 0.0)) break;
    total += pair;
    ++pairs;
  }
  if (threadIdx.x == 0) {
    ess[i] = pairs > 0 ? 1.0 / (2.0 * total - 1.0) : 1.0;
    sqjump[i] = jj;
  }
  for (int k = threadIdx.x; k < n_c; k += blockDim.x) means[(size_t)i * n_c + k] = mk[k];
}

__global__ void k_diag_center(int d, int n_c, int n_s, const double *__restrict__ traj, int max_s,
                              const double *__restrict__ means, double *__restrict__ Xc,
                              double *__restrict__ Mc) {
  const size_t K = (size_t)n_c * n_s, n = (size_t)d * K;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / K, rem = e - i * K, k = rem / n_s, j = rem - k * n_s;
    Xc[e] = traj[(i * n_c + k) * max_s + j] - means[i * n_c + k];
  }
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)d * n_c;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / n_c;
    double g = 0.0;
    for (int k = 0; k < n_c; ++k) g += means[i * n_c + k];
    Mc[e] = means[e] - g / n_c;
  }
}

// W = Wr / (n_c (n_s - 1)), V = (n_s - 1)/n_s W + (n_c + 1)/(n_c (n_c - 1)) Br
__global__ void k_diag_wv(int d, int n_c, int n_s, const double *__restrict__ Wr,
                          const double *__restrict__ Br, double *__restrict__ W,
                          double *__restrict__ V) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x) {
    const double w = Wr[e] / ((double)n_c * (n_s - 1));
    W[e] = w;
    V[e] = (double)(n_s - 1) / n_s * w + (double)(n_c + 1) / ((double)n_c * (n_c - 1)) * Br[e];
  }
}

constexpr int kMaxSweeps = 60;

// One-sided Jacobi on the d columns of G (column i at G + i d); with Q the
// rotations are applied to Q as well (Q = I on entry).  sig[i] = |column i|.
__global__ void __launch_bounds__(kJacobiThreads)
    k_jacobi(int d, double *__restrict__ G, double *__restrict__ Q, double *__restrict__ sig,
             int *__restrict__ sweeps_out) {
  __shared__ int rotated;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n = d + (d & 1);  // players of the round-robin, one dummy if d is odd
  int sweep = 0;
  for (; sweep < kMaxSweeps; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int rnd = 0; rnd < n - 1; ++rnd) {
      for (int pi = warp; pi < n / 2; pi += nw) {
        const int p = pi == 0 ? n - 1 : (rnd + pi) % (n - 1);
        const int q = (rnd - pi + n - 1) % (n - 1);
        if (p >= d || q >= d) continue;
        double *gp = G + (size_t)p * d, *gq = G + (size_t)q * d;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int r = lane; r < d; r += 32) {
          const double x = gp[r], y = gq[r];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (!(fabs(ga) > 1e-15 * sqrt(al * be)) || al == 0.0 || be == 0.0) continue;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        for (int r = lane; r < d; r += 32) {
          const double x = gp[r], y = gq[r];
          gp[r] = c * x - s * y;
          gq[r] = s * x + c * y;
        }
        if (Q) {
          double *qp = Q + (size_t)p * d, *qq = Q + (size_t)q * d;
          for (int r = lane; r < d; r += 32) {
            const double x = qp[r], y = qq[r];
            qp[r] = c * x - s * y;
            qq[r] = s * x + c * y;
          }
        }
        if (lane == 0) rotated = 1;
      }
      __syncthreads();
    }
    const int any = rotated;
    __syncthreads();
    if (!any) break;
  }
  for (int i = warp; i < d; i += nw) {
    const double *g = G + (size_t)i * d;
    double s = 0.0;
    for (int r = lane; r < d; r += 32) s += g[r] * g[r];
    s = warp_sum(s);
    if (lane == 0) sig[i] = sqrt(s);
  }
  if (threadIdx.x == 0 && sweeps_out) *sweeps_out = sweep + 1;
}

__global__ void k_eye(int d, double *__restrict__ Q) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x)
    Q[e] = (e / d == e % d) ? 1.0 : 0.0;
}

// S[a][b] = sum_i sqrt(max(lam_i, 0)) Q(a, i) Q(b, i), Q by columns.
__global__ void k_sym_sqrt(int d, const double *__restrict__ Q, const double *__restrict__ lam,
                           double *__restrict__ S) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x) {
    const int a = e / d, b = e % d;
    double s = 0.0;
    for (int i = 0; i < d; ++i) s += sqrt(fmax(lam[i], 0.0)) * Q[(size_t)i * d + a] * Q[(size_t)i * d + b];
    S[e] = s;
  }
}

// C = A B (row-major d x d)
__global__ void k_mm(int d, const double *__restrict__ A, const double *__restrict__ B,
                     double *__restrict__ C) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x) {
    const int a = e / d, b = e % d;
    double s = 0.0;
    for (int i = 0; i < d; ++i) s += A[(size_t)a * d + i] * B[(size_t)i * d + b];
    C[e] = s;
  }
}

// R_w = Tr W + Tr V - 2 sum_i sqrt(sig_i); out = {R_w, Tr W, Tr V}
__global__ void k_mpsrf_final(int d, const double *__restrict__ W, const double *__restrict__ V,
                              const double *__restrict__ sig, double *__restrict__ out) {
  __shared__ double red[40];
  double tw = 0.0, tv = 0.0, sq = 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    tw += W[(size_t)i * d + i];
    tv += V[(size_t)i * d + i];
    sq += sqrt(fmax(sig[i], 0.0));
  }
  tw = block_sum(tw, red);
  tv = block_sum(tv, red);
  sq = block_sum(sq, red);
  if (threadIdx.x == 0) {
    out[0] = tw + tv - 2.0 * sq;
    out[1] = tw;
    out[2] = tv;
  }
}

int grid_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 152 * 8) + 0; }

// out[i r + q] = normal q of Philox (seed, stream, step 0, "chain" i), i < n
__global__ void k_normals(uint64_t seed, uint32_t stream, int n, int r, double *__restrict__ out) {
  const int nb = (r + 3) / 4;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * nb;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / nb), blk = (int)(e - (size_t)i * nb);
    double z[4];
    normals4_f64(philox_block(seed, stream, 0, (uint32_t)i, blk), z);
    for (int q = 0; q < 4; ++q)
      if (4 * blk + q < r) out[(size_t)i * r + 4 * blk + q] = z[q];
  }
}

// dst[c rows + i] = scale * src[i ld + c]  (rows x cols -> cols x rows, FP64)
template <typename T>
__global__ void k_transpose(int rows, int cols, const T *__restrict__ src, int ld, double scale,
                            double *__restrict__ dst) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)rows * cols;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t c = e / rows, i = e - c * rows;
    dst[e] = scale * (double)src[i * ld + c];
  }
}

}  // namespace

cudaError_t launch_diag_record(int n_c, int d, const void *src, int src_f32, int ld_src,
                               double *traj, int max_s, int j, cudaStream_t st) {
  const size_t n = (size_t)n_c * d;
  if (n == 0) return cudaSuccess;
  if (src_f32)
    k_diag_record<float><<<grid_for(n), 256, 0, st>>>(n_c, d, (const float *)src, ld_src, traj,
                                                      max_s, j);
  else
    k_diag_record<double><<<grid_for(n), 256, 0, st>>>(n_c, d, (const double *)src, ld_src,
                                                       traj, max_s, j);
  return cudaGetLastError();
}

cudaError_t launch_diag_ess(int d, int n_c, int n_s, const double *traj, int max_s, double *means,
                            double *ess, double *sqjump, cudaStream_t st) {
  if (d <= 0) return cudaSuccess;
  if (n_c < 2 || n_s < 2 || (size_t)n_c * 8 > 48 * 1024) return cudaErrorInvalidValue;
  k_diag_ess<<<d, kEssThreads, (size_t)n_c * 8, st>>>(n_c, n_s, traj, max_s, means, ess, sqjump);
  return cudaGetLastError();
}

cudaError_t launch_diag_center(int d, int n_c, int n_s, const double *traj, int max_s,
                               const double *means, double *Xc, double *Mc, cudaStream_t st) {
  k_diag_center<<<grid_for((size_t)d * n_c * n_s), 256, 0, st>>>(d, n_c, n_s, traj, max_s, means,
                                                                 Xc, Mc);
  return cudaGetLastError();
}

cudaError_t launch_diag_wv(int d, int n_c, int n_s, const double *Wr, const double *Br, double *W,
                           double *V, cudaStream_t st) {
  k_diag_wv<<<grid_for((size_t)d * d), 256, 0, st>>>(d, n_c, n_s, Wr, Br, W, V);
  return cudaGetLastError();
}

cudaError_t launch_jacobi(int d, double *G, double *Q, double *sig, int *sweeps,
                          cudaStream_t st) {
  if (d <= 0) return cudaSuccess;
  if (Q) {
    k_eye<<<grid_for((size_t)d * d), 256, 0, st>>>(d, Q);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_jacobi<<<1, kJacobiThreads, 0, st>>>(d, G, Q, sig, sweeps);
  return cudaGetLastError();
}

cudaError_t launch_sym_sqrt(int d, const double *Q, const double *lam, double *S,
                            cudaStream_t st) {
  k_sym_sqrt<<<grid_for((size_t)d * d), 256, 0, st>>>(d, Q, lam, S);
  return cudaGetLastError();
}

cudaError_t launch_small_mm(int d, const double *A, const double *B, double *C, cudaStream_t st) {
  k_mm<<<grid_for((size_t)d * d), 256, 0, st>>>(d, A, B, C);
  return cudaGetLastError();
}

cudaError_t launch_normals(uint64_t seed, uint32_t stream, int n, int r, double *out,
                           cudaStream_t st) {
  if (n <= 0 || r <= 0) return cudaSuccess;
  k_normals<<<grid_for((size_t)n * ((r + 3) / 4)), 256, 0, st>>>(seed, stream, n, r, out);
  return cudaGetLastError();
}

cudaError_t launch_transpose(int rows, int cols, const void *src, int src_f32, int ld,
                             double scale, double *dst, cudaStream_t st) {
  const size_t n = (size_t)rows * cols;
  if (n == 0) return cudaSuccess;
  if (src_f32)
    k_transpose<float><<<grid_for(n), 256, 0, st>>>(rows, cols, (const float *)src, ld, scale, dst);
  else
    k_transpose<double><<<grid_for(n), 256, 0, st>>>(rows, cols, (const double *)src, ld, scale,
                                                     dst);
  return cudaGetLastError();
}

cudaError_t launch_mpsrf_final(int d, const double *W, const double *V, const double *sig,
                               double *out, cudaStream_t st) {
  k_mpsrf_final<<<1, 256, 0, st>>>(d, W, V, sig, out);
  return cudaGetLastError();
}

}  // namespace dino
