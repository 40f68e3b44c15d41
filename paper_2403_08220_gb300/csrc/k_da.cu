// The second, true-model stage of delayed-acceptance surrogate mMALA
// (Algorithm 1, lines 7-13).
//
// The first stage (the geometry kernels with ReducedArgs::da set) tests
// rho_r^(1) (eq:da_dino_trr_1) and, for a chain that passes, stages the
// proposal's surrogate state (factor in the spare slot, Phi~, half log det,
// g) without committing it.  The full proposal m^dagger = s m + sqrt(1-s^2) M
// + Psi_r (m_r^dagger - s m_r - sqrt(1-s^2) Psi_r^* M) of Prop. 5.1 is never
// formed here: the true map of this library is G(m) = f_t(E_t m) (a larger
// MLP on an r_t-dimensional encoding of the full field), and E_t m^dagger is
// linear in what the step already has,
//   E_t m^dagger = s (E_t m) + sqrt(1-s^2) (E_t M) + (E_t Psi_r) coef2,
// with E_t m kept as chain state (mt), E_t M a projection of the prior draw
// and coef2 the complement coefficient of the field update.
//
//   k_da_assemble  xt = s mt + cs EtM + EtDc (and its bf16 slices for the
//                  tensor-core MLP);
//   k_da_misfit    Phi = |f_t - y|^2 / (2 noise_var) (the initial state);
//   k_da_decide    Phi(m^dagger), log rho^(2) = Phi(m_j) - Phi(m^dagger)
//                  + Phi~(m_r^dagger) - Phi~(m_r,j) (eq:da_dino_trr_2), the
//                  test against the stage's own uniform (Philox stream U2)
//                  and, for a chain that passes both stages, the commit of
//                  the staged state; the flags it leaves drive the field
//                  update.
#include <algorithm>

#include "chol.cuh"

namespace dino {
namespace {

constexpr int kDaThreads = 128;

template <typename T>
__global__ void k_da_assemble(int C, int r_t, double s, double cs, const double *__restrict__ mt,
                              const T *__restrict__ EtM, const T *__restrict__ EtDc,
                              double *__restrict__ xt, __nv_bfloat16 *xb, int ldx, size_t plane,
                              int nslice) {
  const size_t n = (size_t)C * r_t;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    double v = s * mt[e];
    if (EtM) v += cs * (double)EtM[e];
    if (EtDc) v += (double)EtDc[e];
    xt[e] = v;
    if (xb) {
      const size_t c = e / r_t, i = e - c * r_t;
      split_bf16_store(v, xb + c * ldx + i, plane, nslice);
    }
  }
}

template <typename T>
__device__ double misfit_sum(const T *f, const double *y, int dy, double *red) {
  double ph = 0.0;
  for (int i = threadIdx.x; i < dy; i += blockDim.x) {
    const double rs = (double)f[i] - y[i];
    ph += rs * rs;
  }
  return block_sum(ph, red);
}

template <typename T>
__global__ void __launch_bounds__(kDaThreads) k_da_misfit(int dy, const T *__restrict__ ft,
                                                          const double *__restrict__ y,
                                                          double inv_nv, double *phi_t) {
  __shared__ double red[40];
  const int c = blockIdx.x;
  const double ph = misfit_sum(ft + (size_t)c * dy, y, dy, red);
  if (threadIdx.x == 0) phi_t[c] = 0.5 * ph * inv_nv;
}

template <typename T, typename TJ>
__global__ void __launch_bounds__(kDaThreads) k_da_decide(DaArgs a) {
  __shared__ double red[40];
  __shared__ int flag;
  const int c = blockIdx.x, r = a.r, dy = a.d_y;
  const double ph = misfit_sum(reinterpret_cast<const T *>(a.ft) + (size_t)c * dy, a.y, dy, red);
  if (threadIdx.x == 0) {
    const double phi_new = 0.5 * ph / a.noise_var;
    const uint32_t chain = (uint32_t)(a.id_base + (uint64_t)c);
    const double log_u2 =
        a.ext_log_u2 ? a.ext_log_u2[c]
                     : log(word_to_uniform(philox_block(a.seed, STREAM_U2, a.step, chain, 0).x));
    bool accept = false;
    double lr2 = nan("");
    a.stage1[c] = a.acc[c];
    if (a.acc[c]) {
      lr2 = a.phi_t[c] - phi_new + a.phi_st[c] - a.phi[c];
      const bool finite = isfinite(lr2);
      accept = finite && log_u2 <= fmin(0.0, lr2);
      if (!finite) atomicAdd(&a.counters[1], 1ull);
    }
    a.log_rho2[c] = lr2;
    a.log_u2[c] = log_u2;
    a.acc[c] = accept ? 1 : 0;
    if (accept) {
      a.acc_count[c] += 1;
      atomicAdd(&a.counters[0], 1ull);
      a.phi[c] = a.phi_st[c];
      a.hld[c] = a.hld_st[c];
      a.phi_t[c] = phi_new;
      a.cur[c] ^= 1;
    }
    flag = accept ? 1 : 0;
  }
  __syncthreads();
  if (!flag) return;
  for (int k = threadIdx.x; k < r; k += blockDim.x) {
    a.mr[(size_t)c * r + k] = a.b[(size_t)c * r + k];
    if (a.g_st) a.g[(size_t)c * r + k] = a.g_st[(size_t)c * r + k];
    if (a.a_df) a.a_df[(size_t)c * r + k] = a.b_df[(size_t)c * r + k];
  }
  for (int k = threadIdx.x; k < a.r_t; k += blockDim.x)
    a.mt[(size_t)c * a.r_t + k] = a.xt[(size_t)c * a.r_t + k];
  if (a.Js) {
    const TJ *J = reinterpret_cast<const TJ *>(a.J) + (size_t)c * dy * r;
    TJ *Js = reinterpret_cast<TJ *>(a.Js) + (size_t)c * dy * r;
    for (size_t e = threadIdx.x; e < (size_t)dy * r; e += blockDim.x) Js[e] = J[e];
  }
}

}  // namespace

cudaError_t launch_da_assemble(int C, int r_t, double s, double cs, const double *mt,
                               const void *EtM, const void *EtDc, int in_f32, double *xt,
                               __nv_bfloat16 *xb, int ldx, size_t plane, int nslice,
                               cudaStream_t st) {
  if (C <= 0 || r_t <= 0) return cudaSuccess;
  if (xb && (nslice < 1 || ldx < r_t)) return cudaErrorInvalidValue;
  const size_t n = (size_t)C * r_t;
  const int grid = (int)std::min<size_t>((n + 255) / 256, 152 * 8);
  if (in_f32)
    k_da_assemble<float><<<grid, 256, 0, st>>>(C, r_t, s, cs, mt, (const float *)EtM,
                                                (const float *)EtDc, xt, xb, ldx, plane, nslice);
  else
    k_da_assemble<double><<<grid, 256, 0, st>>>(C, r_t, s, cs, mt, (const double *)EtM,
                                                 (const double *)EtDc, xt, xb, ldx, plane, nslice);
  return cudaGetLastError();
}

cudaError_t launch_da_misfit(int C, int d_y, const void *ft, int f32, const double *y,
                             double noise_var, double *phi_t, cudaStream_t st) {
  if (C <= 0) return cudaSuccess;
  if (f32)
    k_da_misfit<float><<<C, kDaThreads, 0, st>>>(d_y, (const float *)ft, y, 1.0 / noise_var, phi_t);
  else
    k_da_misfit<double><<<C, kDaThreads, 0, st>>>(d_y, (const double *)ft, y, 1.0 / noise_var,
                                                  phi_t);
  return cudaGetLastError();
}

cudaError_t launch_da_decide(const DaArgs &a, cudaStream_t st) {
  if (a.C <= 0) return cudaSuccess;
  if (a.ft_f32 && a.j_f32)
    k_da_decide<float, float><<<a.C, kDaThreads, 0, st>>>(a);
  else if (a.ft_f32)
    k_da_decide<float, double><<<a.C, kDaThreads, 0, st>>>(a);
  else if (a.j_f32)
    k_da_decide<double, float><<<a.C, kDaThreads, 0, st>>>(a);
  else
    k_da_decide<double, double><<<a.C, kDaThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace dino
