// Per-chain reduced-space kernels of the surrogate mMALA step, in FP64.
//
// One CTA per chain keeps the packed lower Cholesky factor L of I + H
// (r (r+1)/2 doubles, row-major: entry (i, j), j <= i, at i (i+1)/2 + j) in
// shared memory and runs every r x r operation of the step on it:
//
//   k_propose   reduced proposal (eq:reduced_space_sampling in Cholesky form)
//               m_r^dag = mu + sqrt(1-s^2) L^-T xi,
//               mu = m_r - (1-s) (I+H)^-1 (m_r + g),
//               and log rho_{0,r}(m_r, m_r^dag) with the geometry at m_r (Sec. 5.4).
//   k_geometry  misfit, gradient, H = J^T J / noise_var + I, its Cholesky
//               factor and half log-determinant at m_r^dag (Alg. 1 lines 3-4),
//               log rho_{0,r}(m_r^dag, m_r), log rho_r^(1) (eq:da_dino_trr_1),
//               the accept test (Alg. 1 line 6) and the state update.
//
// Identities used with L L^T = I + H (exact in real arithmetic):
//   (I+H)^-1 w_a = a - v_a     for w_a = H a - g_a, v_a = (I+H)^-1 (a + g_a),
//   H x = L (L^T x) - x,       x^T H x = |L^T x|^2 - |x|^2.
#include "dino_internal.h"
#include "philox.cuh"

namespace dino {
namespace {

constexpr int kThreads = 256;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kJChunk = 16;  // rows of J staged per pass when forming H

__device__ __forceinline__ int tri(int i) { return i * (i + 1) / 2; }

// Sum over the CTA; `red` holds >= 33 doubles.  Every thread gets the sum.
__device__ double block_sum(double v, double *red) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// x <- L^-1 x.  32-row diagonal blocks are solved by warp 0 with shuffles,
// the rows below each block are updated by the whole CTA.
__device__ void cta_lower_solve(const double *Ls, const double *inv, int r, double *x) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int jb = 0; jb < r; jb += 32) {
    const int nb = min(32, r - jb);
    if (warp == 0) {
      double xl = lane < nb ? x[jb + lane] : 0.0;
      for (int k = 0; k < nb; ++k) {
        const double yk = __shfl_sync(kFull, xl, k) * inv[jb + k];
        if (lane == k)
          xl = yk;
        else if (lane > k && lane < nb)
          xl -= Ls[tri(jb + lane) + jb + k] * yk;
      }
      if (lane < nb) x[jb + lane] = xl;
    }
    __syncthreads();
    for (int i = jb + nb + threadIdx.x; i < r; i += blockDim.x) {
      const double *row = Ls + tri(i) + jb;
      double acc = x[i];
      for (int k = 0; k < nb; ++k) acc -= row[k] * x[jb + k];
      x[i] = acc;
    }
    __syncthreads();
  }
}

// x <- L^-T x (back substitution on the upper factor L^T).
__device__ void cta_upper_solve(const double *Ls, const double *inv, int r, double *x) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int jb = ((r - 1) / 32) * 32; jb >= 0; jb -= 32) {
    const int nb = min(32, r - jb);
    if (warp == 0) {
      double xl = lane < nb ? x[jb + lane] : 0.0;
      for (int k = nb - 1; k >= 0; --k) {
        const double yk = __shfl_sync(kFull, xl, k) * inv[jb + k];
        if (lane == k)
          xl = yk;
        else if (lane < k)
          xl -= Ls[tri(jb + k) + jb + lane] * yk;
      }
      if (lane < nb) x[jb + lane] = xl;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < jb; i += blockDim.x) {
      double acc = x[i];
      for (int k = 0; k < nb; ++k) acc -= Ls[tri(jb + k) + i] * x[jb + k];
      x[i] = acc;
    }
    __syncthreads();
  }
}

// y = L^T x  (y_j = sum_{i >= j} L_ij x_i)
__device__ void cta_upper_matvec(const double *Ls, int r, const double *x, double *y) {
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    double acc = 0.0;
    for (int i = j; i < r; ++i) acc += Ls[tri(i) + j] * x[i];
    y[j] = acc;
  }
  __syncthreads();
}

// y = L x  (y_i = sum_{j <= i} L_ij x_j)
__device__ void cta_lower_matvec(const double *Ls, int r, const double *x, double *y) {
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    const double *row = Ls + tri(i);
    double acc = 0.0;
    for (int j = 0; j <= i; ++j) acc += row[j] * x[j];
    y[i] = acc;
  }
  __syncthreads();
}

// Position (ii, jj) of packed index e in a lower triangle.
__device__ __forceinline__ void tri_pos(int e, int &ii, int &jj) {
  ii = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while (tri(ii + 1) <= e) ++ii;
  while (tri(ii) > e) --ii;
  jj = e - tri(ii);
}

// In-place right-looking Cholesky of the packed matrix; inv[k] = 1 / L_kk.
// A non-positive pivot produces NaN, which the caller turns into a reject.
__device__ void cta_cholesky(double *Ls, double *inv, int r) {
  const int T = blockDim.x;
  for (int k = 0; k < r; ++k) {
    const double dkk = sqrt(Ls[tri(k) + k]);
    const double ik = 1.0 / dkk;
    for (int i = k + 1 + threadIdx.x; i < r; i += T) Ls[tri(i) + k] *= ik;
    __syncthreads();
    if (threadIdx.x == 0) {
      Ls[tri(k) + k] = dkk;
      inv[k] = ik;
    }
    const int n = r - k - 1;
    const int ntri = n * (n + 1) / 2;
    if ((int)threadIdx.x < ntri) {
      int ii, jj;
      tri_pos(threadIdx.x, ii, jj);
      for (int e = threadIdx.x; e < ntri; e += T) {
        const int i = k + 1 + ii, j = k + 1 + jj;
        const int ti = tri(i);
        Ls[ti + j] -= Ls[ti + k] * Ls[tri(j) + k];
        jj += T;
        while (jj > ii) {
          jj -= ii + 1;
          ++ii;
        }
      }
    }
    __syncthreads();
  }
}

// log rho_{0,r}(x -> z) with the geometry (L, g, hld) at x, given v = (I+H)^-1 (x + g).
// Work vectors p, q (length r) are clobbered.
__device__ double log_rho0(const double *Ls, int r, const double *x, const double *gx,
                           const double *v, const double *z, double hld, double s, double dt,
                           double *p, double *q, double *red) {
  const double cs = sqrt(1.0 - s * s);
  cta_upper_matvec(Ls, r, x, p);  // p = L^T x
  cta_lower_matvec(Ls, r, p, q);  // q = (I+H) x
  double t1 = 0.0, t2 = 0.0, nm = 0.0;
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    const double w = q[i] - x[i] - gx[i];      // w = H x - g
    const double mh = (z[i] - s * x[i]) / cs;  // mhat
    t1 += w * (x[i] - v[i]);                   // w^T (I+H)^-1 w
    t2 += mh * w;
    nm += mh * mh;
    p[i] = mh;
  }
  __syncthreads();
  t1 = block_sum(t1, red);
  t2 = block_sum(t2, red);
  nm = block_sum(nm, red);
  cta_upper_matvec(Ls, r, p, q);  // q = L^T mhat
  double t3 = 0.0;
  for (int i = threadIdx.x; i < r; i += blockDim.x) t3 += q[i] * q[i];
  t3 = block_sum(t3, red) - nm;  // mhat^T H mhat
  return -dt / 8.0 * t1 + sqrt(dt) / 2.0 * t2 + hld - 0.5 * t3;
}

__device__ __forceinline__ void split_bf16_store(double x, __nv_bfloat16 *dst, size_t plane,
                                                 int nslice) {
  float rem = (float)x;
  for (int s = 0; s < nslice; ++s) {
    const __nv_bfloat16 h = __float2bfloat16_rn(rem);
    dst[s * plane] = h;
    rem -= __bfloat162float(h);
  }
}

__global__ void __launch_bounds__(kThreads) k_propose(ReducedArgs a) {
  extern __shared__ double sm[];
  const int c = blockIdx.x, r = a.r;
  const size_t lsz = tri_size(r);
  double *Ls = sm;
  double *inv = Ls + lsz;
  double *va = inv + r, *vg = va + r, *vv = vg + r, *vx = vv + r, *vp = vx + r, *vq = vp + r;
  double *red = vq + r;
  const double *Lg = a.L + (size_t)c * lsz;
  for (size_t e = threadIdx.x; e < lsz; e += blockDim.x) Ls[e] = Lg[e];
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    va[i] = a.mr[(size_t)c * r + i];
    vg[i] = a.g[(size_t)c * r + i];
    vv[i] = va[i] + vg[i];
  }
  const uint32_t chain = (uint32_t)(a.id_base + (uint64_t)c);
  for (int blk = threadIdx.x; blk < (r + 3) / 4; blk += blockDim.x) {
    double n4[4];
    normals4_f64(philox_block(a.seed, STREAM_XI, a.step, chain, blk), n4);
    for (int q = 0; q < 4; ++q)
      if (4 * blk + q < r) vx[4 * blk + q] = n4[q];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < r; i += blockDim.x) inv[i] = 1.0 / Ls[tri(i) + i];
  __syncthreads();
  cta_lower_solve(Ls, inv, r, vv);
  cta_upper_solve(Ls, inv, r, vv);  // vv = (I+H)^-1 (a + g)
  cta_upper_solve(Ls, inv, r, vx);  // vx = L^-T xi
  const double s = a.s, cs = sqrt(1.0 - s * s);
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    const double mu = va[i] - (1.0 - s) * vv[i];
    const double b = mu + cs * vx[i];
    vx[i] = b;
    a.mu[(size_t)c * r + i] = mu;
    a.b[(size_t)c * r + i] = b;
    if (a.b_bf16)
      split_bf16_store(b, a.b_bf16 + (size_t)c * a.b_ld + i, a.b_plane, a.b_slices);
  }
  __syncthreads();
  const double lq = log_rho0(Ls, r, va, vg, vv, vx, a.hld[c], s, a.dt, vp, vq, red);
  if (threadIdx.x == 0) a.lq_fwd[c] = lq;
}

template <typename TJ>
__global__ void __launch_bounds__(kThreads) k_geometry(ReducedArgs a, int mode) {
  extern __shared__ double sm[];
  const int c = blockIdx.x, r = a.r, dy = a.d_y;
  const size_t lsz = tri_size(r);
  double *Ls = sm;
  double *inv = Ls + lsz;
  double *vb = inv + r, *vg = vb + r, *va = vg + r, *vv = va + r, *vp = vv + r, *vq = vp + r;
  double *res = vq + r;
  double *red = res + dy;
  TJ *Jc = reinterpret_cast<TJ *>(red + 34);
  const TJ *J = reinterpret_cast<const TJ *>(a.J) + (size_t)c * dy * r;
  const TJ *f = reinterpret_cast<const TJ *>(a.f) + (size_t)c * dy;
  const double inv_nv = 1.0 / a.noise_var;
  const double phi_a = mode ? a.phi[c] : 0.0;  // read before any thread may overwrite it

  for (int i = threadIdx.x; i < r; i += blockDim.x) vb[i] = a.b[(size_t)c * r + i];
  double ph = 0.0;
  for (int i = threadIdx.x; i < dy; i += blockDim.x) {
    const double rs = (double)f[i] - a.y[i];
    res[i] = rs;
    ph += rs * rs;
  }
  const double phi_b = 0.5 * block_sum(ph, red) * inv_nv;  // includes a sync
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < dy; ++i) acc += (double)J[(size_t)i * r + j] * res[i];
    vg[j] = acc * inv_nv;  // g = J^T (f - y) / noise_var
  }
  // I + J^T J / noise_var, accumulated over chunks of kJChunk rows of J
  for (int i0 = 0; i0 < dy; i0 += kJChunk) {
    const int nr = min(kJChunk, dy - i0);
    for (int e = threadIdx.x; e < nr * r; e += blockDim.x) Jc[e] = J[(size_t)i0 * r + e];
    __syncthreads();
    if ((int)threadIdx.x < (int)lsz) {
      int ii, jj;
      tri_pos(threadIdx.x, ii, jj);
      for (int e = threadIdx.x; e < (int)lsz; e += blockDim.x) {
        TJ acc = 0;
        for (int k = 0; k < nr; ++k) acc += Jc[k * r + ii] * Jc[k * r + jj];
        const double h = (double)acc * inv_nv;
        if (i0 == 0)
          Ls[e] = (ii == jj ? 1.0 : 0.0) + h;
        else
          Ls[e] += h;
        jj += blockDim.x;
        while (jj > ii) {
          jj -= ii + 1;
          ++ii;
        }
      }
    }
    __syncthreads();
  }
  if (dy == 0) {
    for (size_t e = threadIdx.x; e < lsz; e += blockDim.x) Ls[e] = 0.0;
    __syncthreads();
    for (int i = threadIdx.x; i < r; i += blockDim.x) Ls[tri(i) + i] = 1.0;
    __syncthreads();
  }
  cta_cholesky(Ls, inv, r);
  double ld = 0.0;
  for (int i = threadIdx.x; i < r; i += blockDim.x) ld += log(Ls[tri(i) + i]);
  const double hld_b = block_sum(ld, red);

  double *Lg = a.L + (size_t)c * lsz;
  if (mode == 0) {
    for (size_t e = threadIdx.x; e < lsz; e += blockDim.x) Lg[e] = Ls[e];
    for (int i = threadIdx.x; i < r; i += blockDim.x) {
      a.g[(size_t)c * r + i] = vg[i];
      a.mr[(size_t)c * r + i] = vb[i];
    }
    if (threadIdx.x == 0) {
      a.phi[c] = phi_b;
      a.hld[c] = hld_b;
    }
    return;
  }

  // log rho_{0,r}(b -> a) with the geometry at b
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    va[i] = a.mr[(size_t)c * r + i];
    vv[i] = vb[i] + vg[i];
  }
  __syncthreads();
  cta_lower_solve(Ls, inv, r, vv);
  cta_upper_solve(Ls, inv, r, vv);  // vv = (I+H_b)^-1 (b + g_b)
  const double lq_rev = log_rho0(Ls, r, vb, vg, vv, va, hld_b, a.s, a.dt, vp, vq, red);
  const double lr = phi_a - phi_b + lq_rev - a.lq_fwd[c];
  const uint32_t chain = (uint32_t)(a.id_base + (uint64_t)c);
  const double log_u = log(word_to_uniform(philox_block(a.seed, STREAM_U, a.step, chain, 0).x));
  const bool finite = isfinite(lr);
  const bool accept = finite && log_u <= fmin(0.0, lr);
  for (int i = threadIdx.x; i < r; i += blockDim.x)
    a.coef[(size_t)c * r + i] = vb[i] - a.s * va[i];
  if (threadIdx.x == 0) {
    a.log_rho[c] = lr;
    a.log_u[c] = log_u;
    a.acc[c] = accept ? 1 : 0;
    if (accept) {
      a.acc_count[c] += 1;
      atomicAdd(&a.counters[0], 1ull);
      a.phi[c] = phi_b;
      a.hld[c] = hld_b;
    }
    if (!finite) atomicAdd(&a.counters[1], 1ull);
    atomicAdd(a.sum_alpha, finite ? exp(fmin(0.0, lr)) : 0.0);
  }
  if (accept) {
    for (size_t e = threadIdx.x; e < lsz; e += blockDim.x) Lg[e] = Ls[e];
    for (int i = threadIdx.x; i < r; i += blockDim.x) {
      a.g[(size_t)c * r + i] = vg[i];
      a.mr[(size_t)c * r + i] = vb[i];
    }
  }
}

}  // namespace

size_t propose_smem_bytes(int r) { return (tri_size(r) + 7 * (size_t)r + 40) * sizeof(double); }

size_t geometry_smem_bytes(int r, int d_y, int jf_f32) {
  return (tri_size(r) + 7 * (size_t)r + d_y + 34) * sizeof(double) +
         (size_t)kJChunk * r * (jf_f32 ? sizeof(float) : sizeof(double)) + 16;
}

cudaError_t launch_propose(const ReducedArgs &a, cudaStream_t st) {
  const size_t smem = propose_smem_bytes(a.r);
  cudaError_t e = cudaFuncSetAttribute(k_propose, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_propose<<<a.C, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_geometry(const ReducedArgs &a, int mode, cudaStream_t st) {
  const size_t smem = geometry_smem_bytes(a.r, a.d_y, a.jf_f32);
  cudaError_t e;
  if (a.jf_f32) {
    e = cudaFuncSetAttribute(k_geometry<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    k_geometry<float><<<a.C, kThreads, smem, st>>>(a, mode);
  } else {
    e = cudaFuncSetAttribute(k_geometry<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    k_geometry<double><<<a.C, kThreads, smem, st>>>(a, mode);
  }
  return cudaGetLastError();
}

}  // namespace dino
