// Per-chain reduced-space kernels of the surrogate mMALA step, in FP64.
//
// Besides m_r, g, Phi and half log det(I + H), each chain keeps one factor
// slot: the packed lower Cholesky factor (row-major, entry (i, j), j <= i, at
// i (i+1)/2 + j) of I + H bordered below by the row (m_r + g)^T, so that its
// row r holds t = L^-1 (m_r + g); then p = L^T m_r.
//
//   k_propose_warp / k_propose
//               reduced proposal (eq:reduced_space_sampling in Cholesky form)
//               m_r^dag = mu + sqrt(1-s^2) L^-T xi,
//               mu = m_r - (1-s) (I+H)^-1 (m_r + g) = m_r - (1-s) L^-T t,
//               both from one two-column back substitution, and
//               log rho_{0,r}(m_r, m_r^dag) with the geometry at m_r (Sec. 5.4).
//   k_geometry  misfit, gradient, H = J^T J / noise_var + I and the bordered
//               factor at m_r^dag (Algorithm 1), log rho_{0,r}(m_r^dag, m_r),
//               log rho_r^(1) (eq:da_dino_trr_1), the accept test and the
//               state update.
//
// With L L^T = I + H, w = H x - g, mhat = (z - s x) / sqrt(1-s^2) for a move
// x -> z, t = L^-1 (x + g) and p = L^T x (exact in real arithmetic):
//   w^T (I+H)^-1 w = |p - t|^2,
//   mhat^T w = (L^T mhat)^T p - mhat^T (x + g),
//   mhat^T H mhat = |L^T mhat|^2 - |mhat|^2,
// so log rho_0 needs no pass over the factor beyond L^T mhat, and that one
// is known in closed form on both sides: on the forward side
// L^T mhat = ((1-s)(p - t) + sqrt(1-s^2) xi) / sqrt(1-s^2); on the reverse
// side the geometry kernel forms L^T z and L^T x from the factor it holds.
//
// The FP64 pipe bounds these kernels (1/64 of the FP32 rate on GB300), so the
// Cholesky is blocked (8-column panels with lookahead) to keep the FP64 units
// fed from shared memory, and on the tensor-core path the product J^T J is
// formed from the FP32 Jacobian in FP32 register tiles, off the FP64 pipe.
#include "chol.cuh"

namespace dino {
namespace {

constexpr int kThreads = 512;

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


// y1 = L^T x1 and, when `two`, y2 = L^T x2 over the leading r rows of L
// (y_j = sum_{j <= i < r} L_ij x_i): column j by thread j, rows in order.
template <class A>
__device__ void cta_upper_matvec2(const typename A::T *Ls, int r, const typename A::T *x1,
                                  const typename A::T *x2, double *y1, double *y2, bool two) {
  using E = typename A::T;
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    typename A::Acc a1 = A::begin(E{}), a2 = A::begin(E{});
    for (int i = j; i < r; ++i) {
      const E l = Ls[tri(i) + j];
      A::sub(a1, l, A::neg(x1[i]));
      if (two) A::sub(a2, l, A::neg(x2[i]));
    }
    y1[j] = A::to(A::end(a1));
    if (two) y2[j] = A::to(A::end(a2));
  }
  __syncthreads();
}

// Shared-memory layout in doubles:
//   Ls[slot_stride(r)] inv[r+1] seven work vectors[r] res[dy] red[kRed] flag[1] | J chunk
// (red[100..102] hold the Cholesky's six work counters)
// (one double, or one double-float pair, per element).  With `global` the
// factor lives in its global slot and takes no shared memory.
struct Layout {
  size_t Ls, inv, v0, res, red, flag, tail;
  __host__ __device__ Layout(int r, int dy, bool global) {
    Ls = 0;
    inv = global ? 0 : slot_stride(r);
    v0 = inv + r + 1;
    res = v0 + 7 * (size_t)r;
    red = res + dy;
    flag = red + kRed;
    tail = (flag + 1 + 1) & ~(size_t)1;  // 16-byte aligned start of the J chunk
  }
};

// One CTA per chain, for r beyond the register-resident warp kernel: the
// factor is read from its global slot (L2-resident while the chain is
// processed), the vectors live in shared memory.
__global__ void __launch_bounds__(kThreads) k_propose(ReducedArgs a) {
  extern __shared__ __align__(16) double sm[];
  const int c = blockIdx.x, r = a.r;
  const Layout lay(r, 0, true);
  const double *Ls = a.L + (size_t)a.cur[c] * a.L_slot + (size_t)c * slot_stride(r);
  const double *tv = Ls + tri(r), *pv = Ls + tri(r + 1);
  double *inv = sm + lay.inv;
  double *va = sm + lay.v0, *vg = va + r, *vx = vg + r, *z1 = vx + r, *z2 = z1 + r;
  double *red = sm + lay.red;
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    va[i] = a.mr[(size_t)c * r + i];
    vg[i] = a.g[(size_t)c * r + i];
    z1[i] = tv[i];
    inv[i] = 1.0 / Ls[tri(i) + i];
  }
  const uint32_t chain = (uint32_t)(a.id_base + (uint64_t)c);
  for (int blk = threadIdx.x; blk < (r + 3) / 4; blk += blockDim.x) {
    double n4[4];
    if (a.ext_xi) {
      for (int q = 0; q < 4; ++q)
        n4[q] = 4 * blk + q < r ? a.ext_xi[(size_t)c * r + 4 * blk + q] : 0.0;
    } else {
      normals4_f64(philox_block(a.seed, STREAM_XI, a.step, chain, blk), n4);
    }
    for (int q = 0; q < 4; ++q)
      if (4 * blk + q < r) vx[4 * blk + q] = z2[4 * blk + q] = n4[q];
  }
  __syncthreads();
  cta_upper_solve(Ls, inv, r, z1);  // z1 = L^-T t = (I+H)^-1 (a + g)
  cta_upper_solve(Ls, inv, r, z2);  // z2 = L^-T xi
  const double s = a.s, cs = sqrt(1.0 - s * s);
  double t1 = 0.0, t2 = 0.0, t3 = 0.0;
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    const double mu = va[i] - (1.0 - s) * z1[i];
    const double b = mu + cs * z2[i];
    a.mu[(size_t)c * r + i] = mu;
    a.b[(size_t)c * r + i] = b;
    if (a.b_bf16)
      split_bf16_store(b, a.b_bf16 + (size_t)c * a.b_ld + i, a.b_plane, a.b_slices);
    const double p = pv[i], d = p - tv[i];               // d = L^-1 w
    const double mh = (b - s * va[i]) / cs;               // mhat
    const double u = ((1.0 - s) * d + cs * vx[i]) / cs;   // L^T mhat
    t1 += d * d;
    t2 += u * p - mh * (va[i] + vg[i]);
    t3 += u * u - mh * mh;
  }
  block_sum3(t1, t2, t3, red);
  if (threadIdx.x == 0)
    a.lq_fwd[c] = -a.dt / 8.0 * t1 + sqrt(a.dt) / 2.0 * t2 + a.hld[c] - 0.5 * t3;
}

// ---------------------------------------------------------------------------
// Warp-per-chain reduced proposal.  Each warp owns one chain; vectors live in
// registers distributed over lanes (element i in lane i % 32, slot i / 32) and
// L is read from global memory (L1/L2), so an SM keeps 16 chains in flight
// and the serial parts of the back substitution of one chain overlap with the
// FP64 work of the others.

constexpr int kPropWarps = 4;  // chains per CTA

// [x, z] <- L^-T [x, z]: back substitution with two right-hand sides, so the
// factor is read once for both.  Column k of a 32-row diagonal block is
// broadcast by shuffles; the blocks above it take the update with lanes
// reading contiguous parts of row k.
template <int S>
__device__ __forceinline__ void warp_upper_solve2(const double *__restrict__ L, int r,
                                                  const double (&invd)[S], double (&x)[S],
                                                  double (&z)[S]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int b = S - 1; b >= 0; --b) {
    if (32 * b >= r) continue;
    const int jb = 32 * b, nb = min(32, r - jb);
    double xb = x[b], zb = z[b];
    const double ib = invd[b];
    for (int k = nb - 1; k >= 0; --k) {
      const double d = __shfl_sync(kFull, ib, k);
      const double xk = __shfl_sync(kFull, xb, k) * d;
      const double zk = __shfl_sync(kFull, zb, k) * d;
      if (lane == k) {
        xb = xk;
        zb = zk;
      } else if (lane < k) {
        const double l = L[tri(jb + k) + jb + lane];
        xb -= l * xk;
        zb -= l * zk;
      }
    }
    x[b] = xb;
    z[b] = zb;
    if (b == 0) continue;
    for (int k = 0; k < nb; ++k) {
      const double xk = __shfl_sync(kFull, xb, k);
      const double zk = __shfl_sync(kFull, zb, k);
      const double *row = L + tri(jb + k);
#pragma unroll
      for (int b2 = 0; b2 < S; ++b2) {
        if (b2 < b) {
          const double l = row[32 * b2 + lane];
          x[b2] -= l * xk;
          z[b2] -= l * zk;
        }
      }
    }
  }
}

template <int S>
__global__ void __launch_bounds__(32 * kPropWarps) k_propose_warp(ReducedArgs a) {
  __shared__ double xi_s[kPropWarps][32 * S];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c = blockIdx.x * kPropWarps + w;
  if (c >= a.C) return;  // whole warp
  const int r = a.r;
  const double *L = a.L + (size_t)a.cur[c] * a.L_slot + (size_t)c * slot_stride(r);
  const double *tv = L + tri(r), *pv = L + tri(r + 1);
  const uint32_t chain = (uint32_t)(a.id_base + (uint64_t)c);
  for (int blk = lane; blk < (r + 3) / 4; blk += 32) {
    double n4[4];
    if (a.ext_xi) {
      for (int q = 0; q < 4; ++q)
        n4[q] = 4 * blk + q < r ? a.ext_xi[(size_t)c * r + 4 * blk + q] : 0.0;
    } else {
      normals4_f64(philox_block(a.seed, STREAM_XI, a.step, chain, blk), n4);
    }
    for (int q = 0; q < 4; ++q)
      if (4 * blk + q < r) xi_s[w][4 * blk + q] = n4[q];
  }
  __syncwarp();
  double va[S], vg[S], vt[S], vx[S], z1[S], z2[S], invd[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int i = 32 * s + lane;
    const bool in = i < r;
    va[s] = in ? a.mr[(size_t)c * r + i] : 0.0;
    vg[s] = in ? a.g[(size_t)c * r + i] : 0.0;
    vt[s] = in ? tv[i] : 0.0;
    vx[s] = in ? xi_s[w][i] : 0.0;
    invd[s] = in ? 1.0 / L[tri(i) + i] : 0.0;
    z1[s] = vt[s];
    z2[s] = vx[s];
  }
  warp_upper_solve2<S>(L, r, invd, z1, z2);  // z1 = (I+H)^-1 (a + g), z2 = L^-T xi
  const double s_ = a.s, cs = sqrt(1.0 - s_ * s_);
  double t1 = 0.0, t2 = 0.0, t3 = 0.0;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int i = 32 * s + lane;
    if (i < r) {
      const double mu = va[s] - (1.0 - s_) * z1[s];
      const double b = mu + cs * z2[s];
      a.mu[(size_t)c * r + i] = mu;
      a.b[(size_t)c * r + i] = b;
      if (a.b_bf16)
        split_bf16_store(b, a.b_bf16 + (size_t)c * a.b_ld + i, a.b_plane, a.b_slices);
      const double p = pv[i], d = p - vt[s];                 // d = L^-1 w
      const double mh = (b - s_ * va[s]) / cs;                // mhat
      const double u = ((1.0 - s_) * d + cs * vx[s]) / cs;    // L^T mhat
      t1 += d * d;
      t2 += u * p - mh * (va[s] + vg[s]);
      t3 += u * u - mh * mh;
    }
  }
  t1 = warp_sum(t1);
  t2 = warp_sum(t2);
  t3 = warp_sum(t3);
  if (lane == 0)
    a.lq_fwd[c] = -a.dt / 8.0 * t1 + sqrt(a.dt) / 2.0 * t2 + a.hld[c] - 0.5 * t3;
}

// One CTA per chain at the point b.  G = false: the factor is built in shared
// memory; G = true (large r): directly in the other global slot.
//
// The matrix factored is I + H bordered by the row v^T = (b + g_b)^T with
// pivot 1 + |v|^2.  Its factor's leading block is L_b and its last row is
// t_b^T = (L_b^-1 v)^T; the last pivot stays >= 1 since |L_b^-1 v| <= |v|
// when I + H >= I.  With p_b = L_b^T b and q_b = L_b^T a the reverse density
// takes L_b^T mhat = (q_b - s p_b) / sqrt(1-s^2) for mhat = (a - s b) / sqrt(1-s^2).
//
// Mode 0 makes b the chain state (slot cur[c]).  Mode 1 evaluates
// log rho_r^(1) against the current state a, takes the accept test and moves
// an accepted chain to b: its factor slot (written only then, into the other
// slot, which becomes current) and its state vectors.  The complement
// coefficient b - s a is written for every chain.
template <typename TJ, bool G, int NT>
__global__ void __launch_bounds__(NT, NT <= 128 ? 4 : (NT <= 256 ? 2 : 1)) k_geometry(ReducedArgs a, int mode) {
  // FP32 Jacobian (tensor-core path): double-float Cholesky; FP64 Jacobian: FP64
  using A = std::conditional_t<sizeof(TJ) == 4, DF, F64>;
  using E = typename A::T;
  static_assert(sizeof(E) == sizeof(double), "one factor element per double of the slot");
  extern __shared__ __align__(16) double sm[];
  const int c = blockIdx.x, r = a.r, dy = a.d_y;
  const size_t ldL = slot_stride(r), lsz = tri_size(r + 1);
  const Layout lay(r, dy, G);
  const int slot = mode == 0 ? a.cur[c] : 1 - a.cur[c];
  double *Lg = a.L + (size_t)slot * a.L_slot + (size_t)c * ldL;
  E *Ls = reinterpret_cast<E *>(G ? Lg : sm + lay.Ls);
  E *inv = reinterpret_cast<E *>(sm + lay.inv);
  double *vb = sm + lay.v0, *vg = vb + r, *va = vg + r, *vp = va + r, *vq = vp + r;
  E *be = reinterpret_cast<E *>(vq + r), *ae = be + r;  // b and a as factor elements
  E *res = reinterpret_cast<E *>(sm + lay.res);  // f - y as factor elements
  double *red = sm + lay.red;
  int *flag = reinterpret_cast<int *>(sm + lay.flag);
  const TJ *J = reinterpret_cast<const TJ *>(a.J) + (size_t)c * dy * r;
  const TJ *f = reinterpret_cast<const TJ *>(a.f) + (size_t)c * dy;
  const double inv_nv = 1.0 / a.noise_var;

  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    vb[i] = a.b[(size_t)c * r + i];
    va[i] = mode == 1 ? a.mr[(size_t)c * r + i] : 0.0;
    be[i] = A::from(vb[i]);
    ae[i] = A::from(va[i]);
  }
  double ph = 0.0;
  for (int i = threadIdx.x; i < dy; i += blockDim.x) {
    const double rs = (double)f[i] - a.y[i];
    res[i] = A::neg(A::from(rs));
    ph += rs * rs;
  }
  const double phi_b = 0.5 * block_sum(ph, red) * inv_nv;  // includes a barrier
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    typename A::Acc acc = A::begin(E{});
    for (int i = 0; i < dy; ++i) A::sub(acc, A::from_j(J[(size_t)i * r + j]), res[i]);
    vg[j] = A::to(A::end(acc)) * inv_nv;  // g = J^T (f - y) / noise_var
  }
  if constexpr (sizeof(TJ) == 4) {
    form_gram_f32<false>(reinterpret_cast<const float *>(J), dy, r, r, inv_nv,
                         reinterpret_cast<float2 *>(Ls), reinterpret_cast<float *>(sm + lay.tail));
  } else {
    double *Ld = reinterpret_cast<double *>(Ls);
    form_gram_f64<false>(reinterpret_cast<const double *>(J), dy, r, r, inv_nv, Ld, sm + lay.tail);
    if (dy == 0) {
      for (int e = threadIdx.x; e < tri(r); e += blockDim.x) Ld[e] = 0.0;
      __syncthreads();
      for (int i = threadIdx.x; i < r; i += blockDim.x) Ld[tri(i) + i] = 1.0;
      __syncthreads();
    }
  }
  double vv = 0.0;  // bordered row v = b + g_b (each thread its own j, as for g)
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    const double v = vb[j] + vg[j];
    Ls[tri(r) + j] = A::from(v);
    vv += v * v;
  }
  vv = block_sum(vv, red);
  if (threadIdx.x == 0) Ls[tri(r) + r] = A::from(1.0 + vv);
  __syncthreads();
  cta_cholesky_panels<A>(Ls, inv, r + 1);
  double ld = 0.0;
  for (int i = threadIdx.x; i < r; i += blockDim.x) ld += log(A::to(Ls[tri(i) + i]));
  const double hld_b = block_sum(ld, red);
  cta_upper_matvec2<A>(Ls, r, be, ae, vp, vq, mode == 1);  // p_b = L^T b, q_b = L^T a

  // the slot holds FP64: copied from shared memory, or converted in place
  // (each thread its own elements) when the factor was built in the slot
  auto store_factor = [&]() {
    for (size_t e = threadIdx.x; e < lsz; e += blockDim.x) {
      const double x = A::to(Ls[e]);
      Lg[e] = x;
    }
  };
  if (mode == 0) {
    store_factor();
    for (int i = threadIdx.x; i < r; i += blockDim.x) {
      Lg[lsz + i] = vp[i];
      a.g[(size_t)c * r + i] = vg[i];
      a.mr[(size_t)c * r + i] = vb[i];
    }
    if (threadIdx.x == 0) {
      a.phi[c] = phi_b;
      a.hld[c] = hld_b;
    }
    return;
  }
  const E *tb = Ls + tri(r);
  const double s = a.s, cs = sqrt(1.0 - s * s);
  double t1 = 0.0, t2 = 0.0, t3 = 0.0;
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    const double d = vp[i] - A::to(tb[i]);         // L_b^-1 w, w = H_b b - g_b
    const double mh = (va[i] - s * vb[i]) / cs;    // mhat for b -> a
    const double u = (vq[i] - s * vp[i]) / cs;     // L_b^T mhat
    t1 += d * d;
    t2 += u * vp[i] - mh * (vb[i] + vg[i]);
    t3 += u * u - mh * mh;
  }
  block_sum3(t1, t2, t3, red);
  if (threadIdx.x == 0) {
    const double lq_rev = -a.dt / 8.0 * t1 + sqrt(a.dt) / 2.0 * t2 + hld_b - 0.5 * t3;
    const double lr = a.phi[c] - phi_b + lq_rev - a.lq_fwd[c];
    *flag = accept_test(a, c, lr, phi_b, hld_b) ? 1 : 0;
  }
  __syncthreads();
  const bool accept = *flag != 0;
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    a.coef[(size_t)c * r + i] = vb[i] - s * va[i];
    if (accept) {
      if (a.da) {
        a.g_st[(size_t)c * r + i] = vg[i];
      } else {
        a.mr[(size_t)c * r + i] = vb[i];
        a.g[(size_t)c * r + i] = vg[i];
      }
      Lg[lsz + i] = vp[i];
    }
  }
  if (accept) store_factor();
}

}  // namespace

bool uses_global_factor(int r, int d_y) {
  const Layout lay(r, d_y, false);
  const size_t jc = (size_t)kJChunkF * ((r + kHT - 1) / kHT * kHT) * sizeof(float);
  return r > kMaxRSmem || lay.tail * sizeof(double) + jc > kSmemLimit;
}

size_t propose_smem_bytes(int r) {
  const Layout lay(r, 0, true);
  return lay.tail * sizeof(double);
}

size_t geometry_smem_bytes(int r, int d_y, int jf_f32) {
  const bool G = uses_global_factor(r, d_y);
  const Layout lay(r, d_y, G);
  const size_t jc = jf_f32 ? (size_t)kJChunkF * ((r + kHT - 1) / kHT * kHT) * sizeof(float)
                           : (size_t)kJChunk * r * sizeof(double);
  return lay.tail * sizeof(double) + jc;
}

cudaError_t launch_propose(const ReducedArgs &a, cudaStream_t st) {
  if (a.r <= 32 * 7) {
    const int grid = (a.C + kPropWarps - 1) / kPropWarps;
    if (a.r <= 32 * 2)
      k_propose_warp<2><<<grid, 32 * kPropWarps, 0, st>>>(a);
    else
      k_propose_warp<7><<<grid, 32 * kPropWarps, 0, st>>>(a);
    return cudaGetLastError();
  }
  const size_t smem = propose_smem_bytes(a.r);
  cudaError_t e =
      cudaFuncSetAttribute(k_propose, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_propose<<<a.C, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename TJ, bool G, int NT>
static cudaError_t launch_geometry_nt(const ReducedArgs &a, int mode, size_t smem,
                                      cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_geometry<TJ, G, NT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_geometry<TJ, G, NT><<<a.C, NT, smem, st>>>(a, mode);
  return cudaGetLastError();
}

// CTA size by r: a small factor keeps few threads busy, and smaller CTAs let
// more chains share an SM (the kernel's loops stride over blockDim); the
// 128- and 256-thread kernels are held to 128 registers so that four and two
// of them fit an SM.
template <typename TJ, bool G>
static cudaError_t launch_geometry_t(const ReducedArgs &a, int mode, size_t smem,
                                     cudaStream_t st) {
  if (a.r <= 64) return launch_geometry_nt<TJ, G, 128>(a, mode, smem, st);
  if (a.r <= 128) return launch_geometry_nt<TJ, G, 256>(a, mode, smem, st);
  return launch_geometry_nt<TJ, G, kThreads>(a, mode, smem, st);
}

cudaError_t launch_geometry(const ReducedArgs &a, int mode, cudaStream_t st) {
  const size_t smem = geometry_smem_bytes(a.r, a.d_y, a.jf_f32);
  const bool G = uses_global_factor(a.r, a.d_y);
  if (a.jf_f32)
    return G ? launch_geometry_t<float, true>(a, mode, smem, st)
             : launch_geometry_t<float, false>(a, mode, smem, st);
  return G ? launch_geometry_t<double, true>(a, mode, smem, st)
           : launch_geometry_t<double, false>(a, mode, smem, st);
}

}  // namespace dino
