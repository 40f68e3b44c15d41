// Per-chain kernels of the eigen proposal map (eq:reduced_space_sampling with
// the eigendecomposition of the Gauss-Newton matrix, Algorithm 1 line 4),
// for d_y < r.
//
// With K = J / sigma, H = K^T K and M = I + K K^T = U diag(nu) U^T (nu >= 1),
// the nonzero eigenpairs of H are (nu_i - 1, K^T U_i / sqrt(nu_i - 1)), so
// the symmetric root (I + H)^-1/2 = P diag((d + 1)^-1/2) P^T acts as
//   (I + H)^-1/2 xi = xi + K^T U diag(phi) U^T K xi,
//   phi_i = (nu_i^-1/2 - 1) / (nu_i - 1) = -1 / (sqrt(nu_i) (1 + sqrt(nu_i))),
// and K (I + H)^-1/2 xi = U diag(nu^-1/2) U^T K xi.  With u = K x - eps and
// v = M^-1 u = U diag(1/nu) U^T u (the Woodbury identities of the perturbation
// map's kernels) the proposal from x is
//   mu = s x + (1 - s) K^T v,   m_r^dag = mu + sqrt(1 - s^2) (I + H)^-1/2 xi,
//   K mhat = ((1 - s)(u - v) + sqrt(1 - s^2) U diag(nu^-1/2) U^T K xi) / sqrt(1 - s^2),
// log det(I + H) = sum_i log nu_i and w^T (I + H)^-1 w = |u|^2 - u^T v, so
// log rho_{0,r} (Sec. 5.4) again needs only d_y-vectors.
//
// M is eigendecomposed per chain by one-sided Jacobi in shared memory (the
// columns of M V are rotated until orthogonal; their norms are nu and V = U),
// in FP64 on both precision paths.  The state slot holds U (d_y x d_y, by
// columns), nu, u, v and t1 = |u|^2 - u^T v; J at the state is kept in Js as
// on the perturbation-map path.
#include "chol.cuh"

namespace dino {
namespace {

constexpr int kEigThreads = 256;
constexpr int kEigSweeps = 40;

struct EigSlot {
  size_t U, nu, u, v, t1;
  __host__ __device__ explicit EigSlot(int dy) {
    U = 0;
    nu = (size_t)dy * dy;
    u = nu + dy;
    v = u + dy;
    t1 = v + dy;
  }
};

// shared layout (doubles): Md[d^2] Vd[d^2] nu, Kb, Ka, u, w, vv, ys[d] | vb va [r] | red, flag
struct EigLayout {
  size_t Md, Vd, nu, Kb, Ka, u, w, vv, ys, vb, va, red, flag, tail;
  __host__ __device__ EigLayout(int r, int dy) {
    const size_t dd = (size_t)dy * dy;
    Md = 0;
    Vd = dd;
    nu = 2 * dd;
    Kb = nu + dy;
    Ka = Kb + dy;
    u = Ka + dy;
    w = u + dy;
    vv = w + dy;
    ys = vv + dy;
    vb = ys + dy;
    va = vb + r;
    red = va + r;
    flag = red + kRed;
    tail = flag + 2;
  }
};

// y = K x (d_y values, / sigma applied): warp per row of J
template <typename TJ>
__device__ void k_times(const TJ *J, int dy, int r, double inv_sigma, const double *x, double *y) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < dy; i += nw) {
    const TJ *Ji = J + (size_t)i * r;
    double acc = 0.0;
    for (int k = lane; k < r; k += 32) acc += (double)Ji[k] * x[k];
    acc = warp_sum(acc);
    if (lane == 0) y[i] = acc * inv_sigma;
  }
  __syncthreads();
}

// One-sided Jacobi on the dense d x d matrix Md (by columns) with the
// rotations accumulated in Vd (= I on entry); nu[i] = |column i of Md V|.
__device__ void eig_jacobi(int d, double *Md, double *Vd, double *nu, int *flag) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n = d + (d & 1);
  for (int sweep = 0; sweep < kEigSweeps; ++sweep) {
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int rnd = 0; rnd < n - 1; ++rnd) {
      for (int pi = warp; pi < n / 2; pi += nw) {
        const int p = pi == 0 ? n - 1 : (rnd + pi) % (n - 1);
        const int q = (rnd - pi + n - 1) % (n - 1);
        if (p >= d || q >= d) continue;
        double *gp = Md + (size_t)p * d, *gq = Md + (size_t)q * d;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int k = lane; k < d; k += 32) {
          al += gp[k] * gp[k];
          be += gq[k] * gq[k];
          ga += gp[k] * gq[k];
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (!(fabs(ga) > 1e-15 * sqrt(al * be))) continue;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
        double *vp = Vd + (size_t)p * d, *vq = Vd + (size_t)q * d;
        for (int k = lane; k < d; k += 32) {
          const double x = gp[k], y = gq[k];
          gp[k] = c * x - sn * y;
          gq[k] = sn * x + c * y;
          const double a = vp[k], b = vq[k];
          vp[k] = c * a - sn * b;
          vq[k] = sn * a + c * b;
        }
        if (lane == 0) *flag = 1;
      }
      __syncthreads();
    }
    const int any = *flag;
    __syncthreads();
    if (!any) break;
  }
  for (int i = warp; i < d; i += nw) {
    double s = 0.0;
    for (int k = lane; k < d; k += 32) s += Md[(size_t)i * d + k] * Md[(size_t)i * d + k];
    s = warp_sum(s);
    if (lane == 0) nu[i] = sqrt(s);
  }
  __syncthreads();
}

// out = U diag(f) U^T x over d-vectors (U by columns in Vd); tmp: d doubles
__device__ void u_diag_ut(int d, const double *Vd, const double *f, const double *x, double *tmp,
                          double *out) {
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < d; ++k) acc += Vd[(size_t)i * d + k] * x[k];  // (U^T x)_i
    tmp[i] = acc * f[i];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < d; ++i) acc += Vd[(size_t)i * d + k] * tmp[i];
    out[k] = acc;
  }
  __syncthreads();
}

template <typename TJ>
__global__ void __launch_bounds__(kEigThreads) k_eig_geometry(ReducedArgs a, int mode) {
  extern __shared__ __align__(16) double sm[];
  const int c = blockIdx.x, r = a.r, dy = a.d_y;
  const EigLayout lay(r, dy);
  const EigSlot sl(dy);
  double *Md = sm + lay.Md, *Vd = sm + lay.Vd, *nu = sm + lay.nu, *Kb = sm + lay.Kb,
         *Ka = sm + lay.Ka, *u = sm + lay.u, *wv = sm + lay.w, *vv = sm + lay.vv,
         *ys = sm + lay.ys, *vb = sm + lay.vb, *va = sm + lay.va, *red = sm + lay.red;
  int *flag = reinterpret_cast<int *>(sm + lay.flag);
  const size_t ldS = (((size_t)dy * dy + 3 * (size_t)dy + 1) + 1) & ~(size_t)1;
  const int slot = mode == 0 ? a.cur[c] : 1 - a.cur[c];
  double *Sg = a.L + (size_t)slot * a.L_slot + (size_t)c * ldS;
  const TJ *J = reinterpret_cast<const TJ *>(a.J) + (size_t)c * dy * r;
  const TJ *f = reinterpret_cast<const TJ *>(a.f) + (size_t)c * dy;
  const double inv_nv = 1.0 / a.noise_var, inv_sigma = sqrt(inv_nv);

  for (int k = threadIdx.x; k < r; k += blockDim.x) {
    vb[k] = a.b[(size_t)c * r + k];
    va[k] = mode == 1 ? a.mr[(size_t)c * r + k] : 0.0;
  }
  double ph = 0.0;
  for (int i = threadIdx.x; i < dy; i += blockDim.x) {
    const double rs = (double)f[i] - a.y[i];
    ys[i] = rs * inv_sigma;  // eps = (f - y) / sigma
    ph += rs * rs;
  }
  const double phi_b = 0.5 * block_sum(ph, red) * inv_nv;
  if (a.Kb_pre) {
    for (int i = threadIdx.x; i < dy; i += blockDim.x) {
      Kb[i] = a.Kb_pre[(size_t)c * dy + i];
      Ka[i] = mode == 1 ? a.Ka_pre[(size_t)c * dy + i] : 0.0;
    }
    __syncthreads();
  } else {
    k_times<TJ>(J, dy, r, inv_sigma, vb, Kb);
    k_times<TJ>(J, dy, r, inv_sigma, va, Ka);
  }
  // M = I + K K^T (dense, by columns; symmetric), V = I
  for (int e = threadIdx.x; e < dy * dy; e += blockDim.x) {
    const int i = e / dy, j = e - i * dy;
    double g;
    if (a.G) {
      const int hi = i > j ? i : j, lo = i > j ? j : i;  // the lower triangle is stored
      g = (double)a.G[((size_t)c * dy + hi) * a.ldg + lo] * inv_nv;
    } else {
      double acc = 0.0;
      for (int k = 0; k < r; ++k) acc += (double)J[(size_t)i * r + k] * (double)J[(size_t)j * r + k];
      g = acc * inv_nv;
    }
    Md[e] = g + (i == j ? 1.0 : 0.0);
    Vd[e] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  eig_jacobi(dy, Md, Vd, nu, flag);
  double uu = 0.0, ld = 0.0;
  for (int i = threadIdx.x; i < dy; i += blockDim.x) {
    u[i] = Kb[i] - ys[i];
    uu += u[i] * u[i];
    ld += log(nu[i]);
    wv[i] = 1.0 / nu[i];
  }
  uu = block_sum(uu, red);
  const double hld_b = 0.5 * block_sum(ld, red);
  u_diag_ut(dy, Vd, wv, u, ys, vv);  // v = M^-1 u
  double uv = 0.0;
  for (int i = threadIdx.x; i < dy; i += blockDim.x) uv += u[i] * vv[i];
  const double t1 = uu - block_sum(uv, red);

  auto store_slot = [&]() {
    for (int e = threadIdx.x; e < dy * dy; e += blockDim.x) Sg[sl.U + e] = Vd[e];
    for (int i = threadIdx.x; i < dy; i += blockDim.x) {
      Sg[sl.nu + i] = nu[i];
      Sg[sl.u + i] = u[i];
      Sg[sl.v + i] = vv[i];
    }
    if (threadIdx.x == 0) Sg[sl.t1] = t1;
  };
  auto take_state = [&]() {
    TJ *Js = reinterpret_cast<TJ *>(a.Js) + (size_t)c * dy * r;
    for (size_t e = threadIdx.x; e < (size_t)dy * r; e += blockDim.x) Js[e] = J[e];
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
      a.mr[(size_t)c * r + k] = vb[k];
      if constexpr (sizeof(TJ) == 4)
        if (a.a_df) a.a_df[(size_t)c * r + k] = a.b_df[(size_t)c * r + k];
    }
  };
  if (mode == 0) {
    store_slot();
    take_state();
    if (threadIdx.x == 0) {
      a.phi[c] = phi_b;
      a.hld[c] = hld_b;
    }
    return;
  }
  const double s = a.s, cs = sqrt(1.0 - s * s);
  double t2 = 0.0, t3 = 0.0, unused = 0.0;
  for (int i = threadIdx.x; i < dy; i += blockDim.x) {
    const double km = (Ka[i] - s * Kb[i]) / cs;  // K mhat for b -> a
    t2 += km * u[i];
    t3 += km * km;
  }
  block_sum3(t2, t3, unused, red);
  if (threadIdx.x == 0) {
    const double lq_rev = -a.dt / 8.0 * t1 + sqrt(a.dt) / 2.0 * t2 + hld_b - 0.5 * t3;
    const double lr = a.phi[c] - phi_b + lq_rev - a.lq_fwd[c];
    *flag = accept_test(a, c, lr, phi_b, hld_b) ? 1 : 0;
  }
  __syncthreads();
  const bool accept = *flag != 0;
  for (int k = threadIdx.x; k < r; k += blockDim.x) a.coef[(size_t)c * r + k] = vb[k] - s * va[k];
  if (accept) {
    store_slot();
    if (!a.da) take_state();
  }
}

template <typename TJ>
__global__ void __launch_bounds__(kEigThreads) k_eig_propose(ReducedArgs a) {
  extern __shared__ __align__(16) double sm[];
  const int c = blockIdx.x, r = a.r, dy = a.d_y;
  const EigLayout lay(r, dy);
  const EigSlot sl(dy);
  const size_t ldS = (((size_t)dy * dy + 3 * (size_t)dy + 1) + 1) & ~(size_t)1;
  const double *Sg = a.L + (size_t)a.cur[c] * a.L_slot + (size_t)c * ldS;
  double *Vd = sm + lay.Vd, *nu = sm + lay.nu, *Kx = sm + lay.Kb, *zd = sm + lay.Ka,
         *u = sm + lay.u, *fv = sm + lay.w, *vv = sm + lay.vv, *tmp = sm + lay.ys,
         *xa = sm + lay.vb, *xi = sm + lay.va, *red = sm + lay.red;
  double *kz = sm + lay.Md;  // d_y-vector: U diag(nu^-1/2) U^T K xi
  const TJ *J = reinterpret_cast<const TJ *>(a.Js) + (size_t)c * dy * r;
  const double inv_sigma = sqrt(1.0 / a.noise_var);
  const double s = a.s, cs = sqrt(1.0 - s * s);
  for (int e = threadIdx.x; e < dy * dy; e += blockDim.x) Vd[e] = Sg[sl.U + e];
  for (int i = threadIdx.x; i < dy; i += blockDim.x) {
    nu[i] = Sg[sl.nu + i];
    u[i] = Sg[sl.u + i];
    vv[i] = Sg[sl.v + i];
  }
  const uint32_t chain = (uint32_t)(a.id_base + (uint64_t)c);
  for (int k = threadIdx.x; k < r; k += blockDim.x) xa[k] = a.mr[(size_t)c * r + k];
  for (int blk = threadIdx.x; blk < (r + 3) / 4; blk += blockDim.x) {
    double n4[4];
    if (a.ext_xi) {
      for (int q = 0; q < 4; ++q)
        n4[q] = 4 * blk + q < r ? a.ext_xi[(size_t)c * r + 4 * blk + q] : 0.0;
    } else {
      normals4_f64(philox_block(a.seed, STREAM_XI, a.step, chain, blk), n4);
    }
    for (int q = 0; q < 4; ++q)
      if (4 * blk + q < r) xi[4 * blk + q] = n4[q];
  }
  __syncthreads();
  k_times<TJ>(J, dy, r, inv_sigma, xi, Kx);  // K xi
  for (int i = threadIdx.x; i < dy; i += blockDim.x) {
    const double sq = sqrt(nu[i]);
    fv[i] = -1.0 / (sq * (1.0 + sq));  // phi_i
  }
  __syncthreads();
  u_diag_ut(dy, Vd, fv, Kx, tmp, zd);  // z = U diag(phi) U^T K xi
  for (int i = threadIdx.x; i < dy; i += blockDim.x) fv[i] = 1.0 / sqrt(nu[i]);
  __syncthreads();
  u_diag_ut(dy, Vd, fv, Kx, tmp, kz);  // K (I + H)^-1/2 xi
  // K^T z and K^T v: thread per column of J (coalesced across threads)
  for (int k = threadIdx.x; k < r; k += blockDim.x) {
    double az = 0.0, av = 0.0;
    for (int i = 0; i < dy; ++i) {
      const double jk = (double)J[(size_t)i * r + k];
      az += jk * zd[i];
      av += jk * vv[i];
    }
    const double mk = s * xa[k] + (1.0 - s) * av * inv_sigma;
    const double bk = mk + cs * (xi[k] + az * inv_sigma);
    a.mu[(size_t)c * r + k] = mk;
    a.b[(size_t)c * r + k] = bk;
    if constexpr (sizeof(TJ) == 4)
      if (a.b_df) a.b_df[(size_t)c * r + k] = DF::from(bk);
    if (a.b_bf16) split_bf16_store(bk, a.b_bf16 + (size_t)c * a.b_ld + k, a.b_plane, a.b_slices);
  }
  double t2 = 0.0, t3 = 0.0, unused = 0.0;
  for (int i = threadIdx.x; i < dy; i += blockDim.x) {
    const double km = ((1.0 - s) * (u[i] - vv[i]) + cs * kz[i]) / cs;  // K mhat
    t2 += km * u[i];
    t3 += km * km;
  }
  block_sum3(t2, t3, unused, red);
  if (threadIdx.x == 0)
    a.lq_fwd[c] = -a.dt / 8.0 * Sg[sl.t1] + sqrt(a.dt) / 2.0 * t2 + a.hld[c] - 0.5 * t3;
}

}  // namespace

size_t eig_slot_stride(int d_y) {
  return (((size_t)d_y * d_y + 3 * (size_t)d_y + 1) + 1) & ~(size_t)1;
}

size_t eig_smem_bytes(int r, int d_y) { return EigLayout(r, d_y).tail * sizeof(double); }

cudaError_t launch_eig_geometry(const ReducedArgs &a, int mode, cudaStream_t st) {
  const size_t smem = eig_smem_bytes(a.r, a.d_y);
  if (a.jf_f32) {
    cudaError_t e = cudaFuncSetAttribute(k_eig_geometry<float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_eig_geometry<float><<<a.C, kEigThreads, smem, st>>>(a, mode);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_eig_geometry<double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_eig_geometry<double><<<a.C, kEigThreads, smem, st>>>(a, mode);
  }
  return cudaGetLastError();
}

cudaError_t launch_eig_propose(const ReducedArgs &a, cudaStream_t st) {
  const size_t smem = eig_smem_bytes(a.r, a.d_y);
  if (a.jf_f32) {
    cudaError_t e = cudaFuncSetAttribute(k_eig_propose<float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_eig_propose<float><<<a.C, kEigThreads, smem, st>>>(a);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_eig_propose<double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_eig_propose<double><<<a.C, kEigThreads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace dino
