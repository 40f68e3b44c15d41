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
//
// The FP64 pipe bounds both kernels (1/64 of the FP32 rate on GB300), so the
// Cholesky is blocked (8-column panels, 3 barriers per panel) to keep the
// FP64 units fed from shared memory, and on the tensor-core path the product
// J^T J is formed from the FP32 Jacobian in FP32 register tiles, off the FP64
// pipe.  Factors move from HBM into shared memory by TMA bulk copies.
#include "dino_internal.h"
#include "philox.cuh"

namespace dino {
namespace {

constexpr int kThreads = 512;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kJChunk = 16;    // rows of an FP64 J staged per pass when forming H
constexpr int kJChunkF = 32;   // rows of an FP32 J staged per pass
constexpr int kNB = 8;         // Cholesky panel width
constexpr int kHT = 4;         // FP32 register tile edge for J^T J
constexpr int kHMaxTiles = 3;  // tiles per thread: ceil(52*53/2 / 512) for r <= 208
constexpr uint32_t kSpinLimit = 1u << 24;

__device__ __forceinline__ int tri(int i) { return i * (i + 1) / 2; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

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

__device__ __forceinline__ bool mbar_try0(uint32_t bar) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar)
      : "memory");
  return done != 0;
}

__device__ bool mbar_wait0_bounded(uint32_t bar) {
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    if (mbar_try0(bar)) return true;
    if (it > 32) __nanosleep(64);
  }
  return false;
}

// TMA bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// from global to shared memory.  Thread 0 issues and waits with a bounded
// spin; the verdict is shared through `flag`.  On timeout it raises bit 4 of
// `err`, waits once more (bounded) for the copies in flight, and every thread
// gets false.
__device__ bool cta_bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *mbar,
                              int *flag, int *err) {
  if (threadIdx.x == 0) {
    const uint32_t bar = smem_u32(mbar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
    const char *s = static_cast<const char *>(src);
    const uint32_t d = smem_u32(dst);
    for (uint32_t off = 0; off < bytes; off += 65536u) {
      const uint32_t n = bytes - off < 65536u ? bytes - off : 65536u;
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
          "[%3];" ::"r"(d + off),
          "l"(s + off), "r"(n), "r"(bar)
          : "memory");
    }
    const bool ok = mbar_wait0_bounded(bar);
    if (!ok) {
      atomicOr(err, 4);
      mbar_wait0_bounded(bar);
    }
    *flag = ok ? 1 : 0;
  }
  __syncthreads();
  return *flag != 0;
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

// Factor the 8 x 8 diagonal block at kb (size nb) by one warp: pivots from
// y = x^(-1/2), an FP32 estimate refined by two Newton-Raphson steps on
// 1/y^2 - x = 0 (y <- y (3 - x y^2) / 2), then the block's own column scaling
// and rank-1 updates.  inv[k] = 1 / L_kk.
__device__ __forceinline__ void warp_factor_diag(double *Ls, double *inv, int kb, int nb,
                                                 int lane) {
  for (int q = 0; q < nb; ++q) {
    const int kq = kb + q;
    const double xkk = Ls[tri(kq) + kq];
    double id = (double)rsqrtf((float)xkk);
    id = id * (1.5 - 0.5 * xkk * id * id);
    id = id * (1.5 - 0.5 * xkk * id * id);
    const double d = xkk * id;
    __syncwarp();
    if (lane == 0) {
      Ls[tri(kq) + kq] = d;
      inv[kq] = id;
    }
    if (lane > q && lane < nb) Ls[tri(kb + lane) + kq] *= id;
    __syncwarp();
    for (int e = lane; e < nb * nb; e += 32) {
      const int i = e / nb, j = e % nb;
      if (j > q && j <= i)
        Ls[tri(kb + i) + kb + j] -= Ls[tri(kb + i) + kq] * Ls[tri(kb + j) + kq];
    }
    __syncwarp();
  }
}

// Rows i >= row0 of the panel at kb: L[i, kb:kb+nb] <- L[i, kb:kb+nb] L_bb^-T.
__device__ __forceinline__ void panel_solve(double *Ls, const double *inv, int r, int kb, int nb,
                                            int row0, int t0, int T) {
  for (int i = row0 + t0; i < r; i += T) {
    double *row = Ls + tri(i) + kb;
    double x[kNB];
#pragma unroll
    for (int q = 0; q < kNB; ++q) {
      if (q < nb) {
        double acc = row[q];
        const double *lq = Ls + tri(kb + q) + kb;
#pragma unroll
        for (int p = 0; p < q; ++p) acc -= x[p] * lq[p];
        x[q] = acc * inv[kb + q];
      }
    }
#pragma unroll
    for (int q = 0; q < kNB; ++q)
      if (q < nb) row[q] = x[q];
  }
}

// Rank-nb update from the panel at kb of the entries (i, j), j0 <= j <= i < r
// and j < j1: the triangle below j0 when j1 >= r, or a column strip.
// Threads t0, t0 + T, ... share the entries evenly; each thread works on two
// entries at a time so that two independent FMA chains hide the FP64 latency.
struct StripPos {
  int ii, jj;
};

__device__ __forceinline__ void strip_advance(StripPos &p, int step, int w) {
  p.jj += step;
  while (true) {
    const int len = p.ii + 1 < w ? p.ii + 1 : w;
    if (p.jj < len) break;
    p.jj -= len;
    ++p.ii;
  }
}

__device__ __forceinline__ void trailing_update(double *Ls, int r, int kb, int nb, int j0, int j1,
                                                int t0, int T) {
  const int n = r - j0;
  const int w = min(j1, r) - j0;  // strip width (w == n: whole triangle)
  const int full = w * (w + 1) / 2 + (n - w) * w;
  if (t0 >= full) return;
  StripPos p;
  {
    const int tw = w * (w + 1) / 2;
    if (t0 < tw) {
      tri_pos(t0, p.ii, p.jj);
    } else {
      p.ii = w + (t0 - tw) / w;
      p.jj = (t0 - tw) % w;
    }
  }
  for (int e = t0; e < full; e += 2 * T) {
    StripPos q = p;
    const bool two = e + T < full;
    if (two) strip_advance(q, T, w);
    const int i1 = j0 + p.ii, c1 = j0 + p.jj;
    const int i2 = j0 + q.ii, c2 = j0 + q.jj;
    const double *li1 = Ls + tri(i1) + kb, *lj1 = Ls + tri(c1) + kb;
    const double *li2 = Ls + tri(i2) + kb, *lj2 = Ls + tri(c2) + kb;
    double *a1 = Ls + tri(i1) + c1;
    double *a2 = Ls + tri(i2) + c2;
    double acc1 = *a1, acc2 = two ? *a2 : 0.0;
    if (nb == kNB) {
      double x1[kNB], y1[kNB], x2[kNB], y2[kNB];
#pragma unroll
      for (int k = 0; k < kNB; ++k) {
        x1[k] = li1[k];
        y1[k] = lj1[k];
        x2[k] = two ? li2[k] : 0.0;
        y2[k] = two ? lj2[k] : 0.0;
      }
#pragma unroll
      for (int k = 0; k < kNB; ++k) {
        acc1 -= x1[k] * y1[k];
        acc2 -= x2[k] * y2[k];
      }
    } else {
      for (int k = 0; k < nb; ++k) acc1 -= li1[k] * lj1[k];
      if (two)
        for (int k = 0; k < nb; ++k) acc2 -= li2[k] * lj2[k];
    }
    *a1 = acc1;
    if (two) *a2 = acc2;
    p = q;
    strip_advance(p, two ? T : 0, w);
  }
}

// In-place right-looking Cholesky of the packed matrix in 8-column panels
// with a one-panel lookahead and warp specialisation.  Per panel:
//   (A) all threads: the next panel's columns take this panel's rank-8 update;
//   (B) warps 0-3 factor the next diagonal block (warp 0) and then solve the
//       rows below it against that block, while warps 4.. apply this panel's
//       update to the rest of the trailing triangle.
// Two CTA barriers per panel; the serial diagonal work and the panel solve
// run in the shadow of the trailing update.  Per element this is the same
// sequence of fused multiply-adds as the column-at-a-time algorithm.  A
// non-positive pivot produces NaN, which the caller turns into a reject.
constexpr int kPanelThreads = 128;  // warps 0-3

__device__ __forceinline__ void panel_group_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kPanelThreads) : "memory");
}

__device__ void cta_cholesky(double *Ls, double *inv, int r) {
  const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (warp == 0) warp_factor_diag(Ls, inv, 0, min(kNB, r), lane);
  __syncthreads();
  panel_solve(Ls, inv, r, 0, min(kNB, r), min(kNB, r), tid, T);
  __syncthreads();
  for (int kb = 0; kb < r; kb += kNB) {
    const int nb = min(kNB, r - kb);
    const int nk = kb + nb;  // next panel
    if (nk >= r) break;
    const int nb2 = min(kNB, r - nk);
    trailing_update(Ls, r, kb, nb, nk, nk + nb2, tid, T);  // (A)
    __syncthreads();
    if (tid < kPanelThreads) {  // (B) panel group
      if (warp == 0) warp_factor_diag(Ls, inv, nk, nb2, lane);
      panel_group_sync();
      panel_solve(Ls, inv, r, nk, nb2, nk + nb2, tid, kPanelThreads);
    } else if (nk + nb2 < r) {  // (B) update group
      trailing_update(Ls, r, kb, nb, nk + nb2, r, tid - kPanelThreads, T - kPanelThreads);
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

// Shared-memory layout in doubles:
//   Ls[ldL] inv[r] six work vectors[r] res[dy] red[34] mbar[1] flag[1] | J chunk
struct Layout {
  size_t Ls, inv, v0, res, red, mbar, flag, tail;
  // with `global` the factor lives in global memory and takes no shared memory
  __host__ __device__ Layout(int r, int dy, size_t ldL, bool global = false) {
    Ls = 0;
    inv = global ? 0 : ldL;
    v0 = inv + r;
    res = v0 + 6 * (size_t)r;
    red = res + dy;
    mbar = (red + 34 + 1) & ~(size_t)1;  // 8-byte mbarrier, kept 16-byte aligned
    flag = mbar + 1;
    tail = (flag + 1 + 1) & ~(size_t)1;  // 16-byte aligned start of the J chunk
  }
};

// One CTA per chain.  G = false: the factor is bulk-copied into shared
// memory; G = true (large r): the CTA works on the chain's factor in global
// memory (L2-resident while the chain is processed).
template <bool G>
__global__ void __launch_bounds__(kThreads) k_propose(ReducedArgs a) {
  extern __shared__ __align__(16) double sm[];
  const int c = blockIdx.x, r = a.r;
  const size_t ldL = l_stride(r);
  const Layout lay(r, 0, ldL, G);
  double *Lcur = a.L + (size_t)a.cur[c] * a.L_slot + (size_t)c * ldL;
  double *Ls = G ? Lcur : sm + lay.Ls;
  double *inv = sm + lay.inv;
  double *va = sm + lay.v0, *vg = va + r, *vv = vg + r, *vx = vv + r, *vp = vx + r, *vq = vp + r;
  double *red = sm + lay.red;
  if (!G && !cta_bulk_load(Ls, Lcur, (uint32_t)(ldL * 8),
                           reinterpret_cast<uint64_t *>(sm + lay.mbar),
                           reinterpret_cast<int *>(sm + lay.flag), a.err))
    return;
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    va[i] = a.mr[(size_t)c * r + i];
    vg[i] = a.g[(size_t)c * r + i];
    vv[i] = va[i] + vg[i];
    inv[i] = 1.0 / Ls[tri(i) + i];
  }
  const uint32_t chain = (uint32_t)(a.id_base + (uint64_t)c);
  for (int blk = threadIdx.x; blk < (r + 3) / 4; blk += blockDim.x) {
    double n4[4];
    normals4_f64(philox_block(a.seed, STREAM_XI, a.step, chain, blk), n4);
    for (int q = 0; q < 4; ++q)
      if (4 * blk + q < r) vx[4 * blk + q] = n4[q];
  }
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

// ---------------------------------------------------------------------------
// Warp-per-chain reduced proposal.  Each warp owns one chain; vectors live in
// registers distributed over lanes (element i in lane i % 32, slot i / 32) and
// L is read from global memory (L1/L2), so an SM keeps 16 chains in flight
// and the serial parts of the triangular solves of one chain overlap with the
// FP64 work of the others.

constexpr int kPropWarps = 4;  // chains per CTA

template <int S>
__device__ __forceinline__ void warp_lower_solve(const double *__restrict__ L, int r,
                                                 const double (&invd)[S], double (&t)[S]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int b = 0; b < S; ++b) {
    if (32 * b >= r) break;
    const int jb = 32 * b, nb = min(32, r - jb);
    double tb = t[b];
    const double ib = invd[b];
    for (int k = 0; k < nb; ++k) {
      const double yk = __shfl_sync(kFull, tb, k) * __shfl_sync(kFull, ib, k);
      if (lane == k)
        tb = yk;
      else if (lane > k && lane < nb)
        tb -= L[tri(jb + lane) + jb + k] * yk;
    }
    t[b] = tb;
#pragma unroll
    for (int b2 = b + 1; b2 < S; ++b2) {
      if (32 * b2 >= r) break;
      const int i = 32 * b2 + lane;
      const double *row = L + tri(i) + jb;
      double acc = t[b2];
      for (int k = 0; k < nb; ++k) {
        const double yk = __shfl_sync(kFull, tb, k);
        if (i < r) acc -= row[k] * yk;
      }
      t[b2] = acc;
    }
  }
}

template <int S>
__device__ __forceinline__ void warp_upper_solve(const double *__restrict__ L, int r,
                                                 const double (&invd)[S], double (&t)[S]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int b = S - 1; b >= 0; --b) {
    if (32 * b >= r) continue;
    const int jb = 32 * b, nb = min(32, r - jb);
    double tb = t[b];
    const double ib = invd[b];
    for (int k = nb - 1; k >= 0; --k) {
      const double xk = __shfl_sync(kFull, tb, k) * __shfl_sync(kFull, ib, k);
      if (lane == k)
        tb = xk;
      else if (lane < k)
        tb -= L[tri(jb + k) + jb + lane] * xk;
    }
    t[b] = tb;
#pragma unroll
    for (int b2 = 0; b2 < b; ++b2) {
      const int i = 32 * b2 + lane;
      double acc = t[b2];
      for (int k = 0; k < nb; ++k) acc -= L[tri(jb + k) + i] * __shfl_sync(kFull, tb, k);
      t[b2] = acc;
    }
  }
}

// y = L^T x: for each row i of L (coalesced across lanes j <= i)
template <int S>
__device__ __forceinline__ void warp_upper_matvec(const double *__restrict__ L, int r,
                                                  const double (&x)[S], double (&y)[S]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < S; ++s) y[s] = 0.0;
#pragma unroll
  for (int b = 0; b < S; ++b) {
    if (32 * b >= r) break;
    const int nb = min(32, r - 32 * b);
    for (int k = 0; k < nb; ++k) {
      const int i = 32 * b + k;
      const double xi = __shfl_sync(kFull, x[b], k);
      const double *row = L + tri(i);
#pragma unroll
      for (int s = 0; s <= b; ++s) {
        const int j = 32 * s + lane;
        if (j <= i) y[s] += row[j] * xi;
      }
    }
  }
}

// y = L x: each lane its own rows, contiguous along the row
template <int S>
__device__ __forceinline__ void warp_lower_matvec(const double *__restrict__ L, int r,
                                                  const double (&x)[S], double (&y)[S]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    y[s] = 0.0;
    if (32 * s >= r) continue;
    const int i = 32 * s + lane;
    const double *row = L + tri(min(i, r - 1));
    double acc = 0.0;
#pragma unroll
    for (int b = 0; b <= s; ++b) {
      for (int k = 0; k < 32; ++k) {
        const int j = 32 * b + k;
        const double xj = __shfl_sync(kFull, x[b], k);
        if (i < r && j <= i) acc += row[j] * xj;
      }
    }
    y[s] = acc;
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

template <int S>
__global__ void __launch_bounds__(32 * kPropWarps) k_propose_warp(ReducedArgs a) {
  __shared__ double xi_s[kPropWarps][32 * S];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c = blockIdx.x * kPropWarps + w;
  if (c >= a.C) return;  // whole warp
  const int r = a.r;
  const double *L = a.L + (size_t)a.cur[c] * a.L_slot + (size_t)c * l_stride(r);
  const uint32_t chain = (uint32_t)(a.id_base + (uint64_t)c);
  for (int blk = lane; blk < (r + 3) / 4; blk += 32) {
    double n4[4];
    normals4_f64(philox_block(a.seed, STREAM_XI, a.step, chain, blk), n4);
    for (int q = 0; q < 4; ++q)
      if (4 * blk + q < r) xi_s[w][4 * blk + q] = n4[q];
  }
  __syncwarp();
  double va[S], vg[S], vv[S], vx[S], vp[S], vq[S], invd[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int i = 32 * s + lane;
    const bool in = i < r;
    va[s] = in ? a.mr[(size_t)c * r + i] : 0.0;
    vg[s] = in ? a.g[(size_t)c * r + i] : 0.0;
    vv[s] = va[s] + vg[s];
    vx[s] = in ? xi_s[w][i] : 0.0;
    invd[s] = in ? 1.0 / L[tri(i) + i] : 0.0;
  }
  warp_lower_solve<S>(L, r, invd, vv);
  warp_upper_solve<S>(L, r, invd, vv);  // vv = (I+H)^-1 (a + g)
  warp_upper_solve<S>(L, r, invd, vx);  // vx = L^-T xi
  const double s_ = a.s, cs = sqrt(1.0 - s_ * s_);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int i = 32 * s + lane;
    const double mu = va[s] - (1.0 - s_) * vv[s];
    const double b = mu + cs * vx[s];
    vx[s] = i < r ? b : 0.0;
    if (i < r) {
      a.mu[(size_t)c * r + i] = mu;
      a.b[(size_t)c * r + i] = b;
      if (a.b_bf16)
        split_bf16_store(b, a.b_bf16 + (size_t)c * a.b_ld + i, a.b_plane, a.b_slices);
    }
  }
  // log rho_{0,r}(a -> b) with the geometry at a
  warp_upper_matvec<S>(L, r, va, vp);  // p = L^T a
  warp_lower_matvec<S>(L, r, vp, vq);  // q = (I+H) a
  double t1 = 0.0, t2 = 0.0, nm = 0.0;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int i = 32 * s + lane;
    if (i < r) {
      const double wv = vq[s] - va[s] - vg[s];        // w = H a - g
      const double mh = (vx[s] - s_ * va[s]) / cs;    // mhat
      t1 += wv * (va[s] - vv[s]);
      t2 += mh * wv;
      nm += mh * mh;
      vp[s] = mh;
    } else {
      vp[s] = 0.0;
    }
  }
  t1 = warp_sum(t1);
  t2 = warp_sum(t2);
  nm = warp_sum(nm);
  warp_upper_matvec<S>(L, r, vp, vq);  // q = L^T mhat
  double t3 = 0.0;
#pragma unroll
  for (int s = 0; s < S; ++s) t3 += vq[s] * vq[s];
  t3 = warp_sum(t3) - nm;
  if (lane == 0)
    a.lq_fwd[c] = -a.dt / 8.0 * t1 + sqrt(a.dt) / 2.0 * t2 + a.hld[c] - 0.5 * t3;
}

// I + J^T J / noise_var into the packed shared matrix, from an FP64 J:
// chunks of kJChunk rows, FP64 products accumulated in shared memory.
__device__ void form_h_f64(const double *J, int dy, int r, double inv_nv, double *Ls,
                           double *Jc) {
  const int lsz = tri(r);
  for (int i0 = 0; i0 < dy; i0 += kJChunk) {
    const int nr = min(kJChunk, dy - i0);
    for (int e = threadIdx.x; e < nr * r; e += blockDim.x) Jc[e] = J[(size_t)i0 * r + e];
    __syncthreads();
    if ((int)threadIdx.x < lsz) {
      int ii, jj;
      tri_pos(threadIdx.x, ii, jj);
      for (int e = threadIdx.x; e < lsz; e += blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < nr; ++k) acc += Jc[k * r + ii] * Jc[k * r + jj];
        const double h = acc * inv_nv;
        Ls[e] = (i0 == 0 ? (ii == jj ? 1.0 : 0.0) : Ls[e]) + h;
        jj += blockDim.x;
        while (jj > ii) {
          jj -= ii + 1;
          ++ii;
        }
      }
    }
    __syncthreads();
  }
}

// The same from an FP32 J: each thread accumulates up to kHMaxTiles 4 x 4
// tiles of J^T J in FP32 registers over all d_y rows (chunks of kJChunkF
// rows staged in shared memory, padded to a multiple of 4 columns), then
// writes I + H once in FP64.  Large r takes several rounds of tiles.
__device__ void form_h_f32(const float *J, int dy, int r, double inv_nv, double *Ls,
                           float *Jc) {
  const int nt = (r + kHT - 1) / kHT, rp = nt * kHT;
  const int ntiles = nt * (nt + 1) / 2;
  if (dy == 0) {
    for (int e = threadIdx.x; e < tri(r); e += blockDim.x) Ls[e] = 0.0;
    __syncthreads();
    for (int i = threadIdx.x; i < r; i += blockDim.x) Ls[tri(i) + i] = 1.0;
    __syncthreads();
    return;
  }
  for (int t0 = 0; t0 < ntiles; t0 += kHMaxTiles * blockDim.x) {
    int ti[kHMaxTiles], tj[kHMaxTiles];
    float acc[kHMaxTiles][kHT][kHT];
#pragma unroll
    for (int s = 0; s < kHMaxTiles; ++s) {
      const int t = t0 + threadIdx.x + s * blockDim.x;
      if (t < ntiles) {
        tri_pos(t, ti[s], tj[s]);
      } else {
        ti[s] = -1;
        tj[s] = 0;
      }
#pragma unroll
      for (int p = 0; p < kHT; ++p)
#pragma unroll
        for (int q = 0; q < kHT; ++q) acc[s][p][q] = 0.0f;
    }
    for (int i0 = 0; i0 < dy; i0 += kJChunkF) {
      const int nr = min(kJChunkF, dy - i0);
      for (int e = threadIdx.x; e < nr * rp; e += blockDim.x) {
        const int k = e / rp, j = e % rp;
        Jc[e] = j < r ? J[(size_t)(i0 + k) * r + j] : 0.0f;
      }
      __syncthreads();
      for (int k = 0; k < nr; ++k) {
        const float *row = Jc + k * rp;
#pragma unroll
        for (int s = 0; s < kHMaxTiles; ++s) {
          if (ti[s] < 0) continue;
          const float4 x = *reinterpret_cast<const float4 *>(row + kHT * ti[s]);
          const float4 y = *reinterpret_cast<const float4 *>(row + kHT * tj[s]);
          const float xa[4] = {x.x, x.y, x.z, x.w}, ya[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
          for (int p = 0; p < kHT; ++p)
#pragma unroll
            for (int q = 0; q < kHT; ++q) acc[s][p][q] = fmaf(xa[p], ya[q], acc[s][p][q]);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int s = 0; s < kHMaxTiles; ++s) {
      if (ti[s] < 0) continue;
#pragma unroll
      for (int p = 0; p < kHT; ++p)
#pragma unroll
        for (int q = 0; q < kHT; ++q) {
          const int i = kHT * ti[s] + p, j = kHT * tj[s] + q;
          if (i < r && j <= i)
            Ls[tri(i) + j] = (i == j ? 1.0 : 0.0) + (double)acc[s][p][q] * inv_nv;
        }
    }
  }
  __syncthreads();
}

// G = false: the factor is built in shared memory and copied to its slot;
// G = true (large r): built directly in its global slot.  Mode 0 writes the
// chain state (slot cur[c]); mode 1 writes the geometry at the proposal into
// the other slot and the candidate buffers, for the accept kernel.
template <typename TJ, bool G>
__global__ void __launch_bounds__(kThreads) k_geometry(ReducedArgs a, int mode) {
  extern __shared__ __align__(16) double sm[];
  const int c = blockIdx.x, r = a.r, dy = a.d_y;
  const size_t ldL = l_stride(r);
  const Layout lay(r, dy, ldL, G);
  const int slot = mode == 0 ? a.cur[c] : 1 - a.cur[c];
  double *Lg = a.L + (size_t)slot * a.L_slot + (size_t)c * ldL;
  double *Ls = G ? Lg : sm + lay.Ls;
  double *inv = sm + lay.inv;
  double *vb = sm + lay.v0, *vg = vb + r;
  double *res = sm + lay.res;
  double *red = sm + lay.red;
  const TJ *J = reinterpret_cast<const TJ *>(a.J) + (size_t)c * dy * r;
  const TJ *f = reinterpret_cast<const TJ *>(a.f) + (size_t)c * dy;
  const double inv_nv = 1.0 / a.noise_var;

  for (int i = threadIdx.x; i < r; i += blockDim.x) vb[i] = a.b[(size_t)c * r + i];
  double ph = 0.0;
  for (int i = threadIdx.x; i < dy; i += blockDim.x) {
    const double rs = (double)f[i] - a.y[i];
    res[i] = rs;
    ph += rs * rs;
  }
  const double phi_b = 0.5 * block_sum(ph, red) * inv_nv;  // includes a barrier
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < dy; ++i) acc += (double)J[(size_t)i * r + j] * res[i];
    vg[j] = acc * inv_nv;  // g = J^T (f - y) / noise_var
  }
  if constexpr (sizeof(TJ) == 4) {
    form_h_f32(reinterpret_cast<const float *>(J), dy, r, inv_nv, Ls,
               reinterpret_cast<float *>(sm + lay.tail));
  } else {
    form_h_f64(reinterpret_cast<const double *>(J), dy, r, inv_nv, Ls, sm + lay.tail);
    if (dy == 0) {
      for (int e = threadIdx.x; e < tri(r); e += blockDim.x) Ls[e] = 0.0;
      __syncthreads();
      for (int i = threadIdx.x; i < r; i += blockDim.x) Ls[tri(i) + i] = 1.0;
      __syncthreads();
    }
  }
  cta_cholesky(Ls, inv, r);
  double ld = 0.0;
  for (int i = threadIdx.x; i < r; i += blockDim.x) ld += log(Ls[tri(i) + i]);
  const double hld_b = block_sum(ld, red);

  if (!G) {
    const int lsz = tri(r);
    for (int e = threadIdx.x; e < lsz; e += blockDim.x) Lg[e] = Ls[e];
  }
  double *gout = mode == 0 ? a.g : a.g_c;
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    gout[(size_t)c * r + i] = vg[i];
    if (mode == 0) a.mr[(size_t)c * r + i] = vb[i];
  }
  if (threadIdx.x == 0) {
    (mode == 0 ? a.phi : a.phi_c)[c] = phi_b;
    (mode == 0 ? a.hld : a.hld_c)[c] = hld_b;
  }
}

// ---------------------------------------------------------------------------
// Accept: log rho_{0,r}(b -> a) with the candidate factor, log rho_r^(1)
// (eq:da_dino_trr_1), the test log u <= min(0, log rho) (Alg. 1 line 6) and
// the state update.  Warp per chain like the proposal; an accepted chain
// takes the candidate factor by flipping its slot index.

__device__ __forceinline__ void accept_tail(const ReducedArgs &a, int c, double lr) {
  // lane-0 bookkeeping shared by the warp and CTA variants; returns via a.acc
  const uint32_t chain = (uint32_t)(a.id_base + (uint64_t)c);
  const double log_u = log(word_to_uniform(philox_block(a.seed, STREAM_U, a.step, chain, 0).x));
  const bool finite = isfinite(lr);
  const bool accept = finite && log_u <= fmin(0.0, lr);
  a.log_rho[c] = lr;
  a.log_u[c] = log_u;
  a.acc[c] = accept ? 1 : 0;
  if (accept) {
    a.acc_count[c] += 1;
    atomicAdd(&a.counters[0], 1ull);
    a.phi[c] = a.phi_c[c];
    a.hld[c] = a.hld_c[c];
    a.cur[c] ^= 1;
  }
  if (!finite) atomicAdd(&a.counters[1], 1ull);
  atomicAdd(a.sum_alpha, finite ? exp(fmin(0.0, lr)) : 0.0);
}

template <int S>
__global__ void __launch_bounds__(32 * kPropWarps) k_accept_warp(ReducedArgs a) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c = blockIdx.x * kPropWarps + w;
  if (c >= a.C) return;  // whole warp
  const int r = a.r;
  const double *L = a.L + (size_t)(1 - a.cur[c]) * a.L_slot + (size_t)c * l_stride(r);
  double va[S], vb[S], vg[S], vv[S], vp[S], vq[S], invd[S];
  const double s_ = a.s, cs = sqrt(1.0 - s_ * s_);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int i = 32 * s + lane;
    const bool in = i < r;
    va[s] = in ? a.mr[(size_t)c * r + i] : 0.0;
    vb[s] = in ? a.b[(size_t)c * r + i] : 0.0;
    vg[s] = in ? a.g_c[(size_t)c * r + i] : 0.0;
    vv[s] = vb[s] + vg[s];
    invd[s] = in ? 1.0 / L[tri(i) + i] : 0.0;
  }
  warp_lower_solve<S>(L, r, invd, vv);
  warp_upper_solve<S>(L, r, invd, vv);  // vv = (I+H_b)^-1 (b + g_b)
  warp_upper_matvec<S>(L, r, vb, vp);   // p = L^T b
  warp_lower_matvec<S>(L, r, vp, vq);   // q = (I+H_b) b
  double t1 = 0.0, t2 = 0.0, nm = 0.0;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int i = 32 * s + lane;
    if (i < r) {
      const double wv = vq[s] - vb[s] - vg[s];       // w = H_b b - g_b
      const double mh = (va[s] - s_ * vb[s]) / cs;   // mhat for b -> a
      t1 += wv * (vb[s] - vv[s]);
      t2 += mh * wv;
      nm += mh * mh;
      vp[s] = mh;
    } else {
      vp[s] = 0.0;
    }
  }
  t1 = warp_sum(t1);
  t2 = warp_sum(t2);
  nm = warp_sum(nm);
  warp_upper_matvec<S>(L, r, vp, vq);  // q = L^T mhat
  double t3 = 0.0;
#pragma unroll
  for (int s = 0; s < S; ++s) t3 += vq[s] * vq[s];
  t3 = warp_sum(t3) - nm;
  const double lq_rev = -a.dt / 8.0 * t1 + sqrt(a.dt) / 2.0 * t2 + a.hld_c[c] - 0.5 * t3;
  const double lr = a.phi[c] - a.phi_c[c] + lq_rev - a.lq_fwd[c];
  __syncwarp();
  int accept = 0;
  if (lane == 0) {
    accept_tail(a, c, lr);
    accept = a.acc[c];
  }
  accept = __shfl_sync(kFull, accept, 0);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int i = 32 * s + lane;
    if (i < r) {
      a.coef[(size_t)c * r + i] = vb[s] - s_ * va[s];
      if (accept) {
        a.mr[(size_t)c * r + i] = vb[s];
        a.g[(size_t)c * r + i] = vg[s];
      }
    }
  }
}

// CTA variant for r beyond the register-resident warp kernel (factor in global memory).
__global__ void __launch_bounds__(kThreads) k_accept_cta(ReducedArgs a) {
  extern __shared__ __align__(16) double sm[];
  const int c = blockIdx.x, r = a.r;
  const Layout lay(r, 0, l_stride(r), true);
  const double *Ls = a.L + (size_t)(1 - a.cur[c]) * a.L_slot + (size_t)c * l_stride(r);
  double *inv = sm + lay.inv;
  double *va = sm + lay.v0, *vb = va + r, *vg = vb + r, *vv = vg + r, *vp = vv + r, *vq = vp + r;
  double *red = sm + lay.red;
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    va[i] = a.mr[(size_t)c * r + i];
    vb[i] = a.b[(size_t)c * r + i];
    vg[i] = a.g_c[(size_t)c * r + i];
    vv[i] = vb[i] + vg[i];
    inv[i] = 1.0 / Ls[tri(i) + i];
  }
  __syncthreads();
  cta_lower_solve(Ls, inv, r, vv);
  cta_upper_solve(Ls, inv, r, vv);
  const double phi_a = a.phi[c];  // read before thread 0 may overwrite it
  const double lq_rev = log_rho0(Ls, r, vb, vg, vv, va, a.hld_c[c], a.s, a.dt, vp, vq, red);
  const double lr = phi_a - a.phi_c[c] + lq_rev - a.lq_fwd[c];
  int *flag = reinterpret_cast<int *>(sm + lay.flag);
  if (threadIdx.x == 0) {
    accept_tail(a, c, lr);
    *flag = a.acc[c];
  }
  __syncthreads();
  const int accept = *flag;
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    a.coef[(size_t)c * r + i] = vb[i] - a.s * va[i];
    if (accept) {
      a.mr[(size_t)c * r + i] = vb[i];
      a.g[(size_t)c * r + i] = vg[i];
    }
  }
}

}  // namespace

bool uses_global_factor(int r, int d_y) {
  const Layout lay(r, d_y, l_stride(r));
  const size_t jc = (size_t)kJChunkF * ((r + kHT - 1) / kHT * kHT) * sizeof(float);
  return r > kMaxRSmem || lay.tail * sizeof(double) + jc > kSmemLimit;
}

size_t propose_smem_bytes(int r) {
  const bool G = uses_global_factor(r, 0);
  const Layout lay(r, 0, l_stride(r), G);
  return lay.tail * sizeof(double);
}

size_t geometry_smem_bytes(int r, int d_y, int jf_f32) {
  const bool G = uses_global_factor(r, d_y);
  const Layout lay(r, d_y, l_stride(r), G);
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
  if (uses_global_factor(a.r, 0)) {
    cudaError_t e = cudaFuncSetAttribute(k_propose<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_propose<true><<<a.C, kThreads, smem, st>>>(a);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_propose<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_propose<false><<<a.C, kThreads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

template <typename TJ, bool G>
static cudaError_t launch_geometry_t(const ReducedArgs &a, int mode, size_t smem,
                                     cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_geometry<TJ, G>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_geometry<TJ, G><<<a.C, kThreads, smem, st>>>(a, mode);
  return cudaGetLastError();
}

cudaError_t launch_accept(const ReducedArgs &a, cudaStream_t st) {
  if (a.r <= 32 * 7) {
    const int grid = (a.C + kPropWarps - 1) / kPropWarps;
    if (a.r <= 32 * 2)
      k_accept_warp<2><<<grid, 32 * kPropWarps, 0, st>>>(a);
    else
      k_accept_warp<7><<<grid, 32 * kPropWarps, 0, st>>>(a);
    return cudaGetLastError();
  }
  const Layout lay(a.r, 0, l_stride(a.r), true);
  const size_t smem = lay.tail * sizeof(double);
  cudaError_t e =
      cudaFuncSetAttribute(k_accept_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_accept_cta<<<a.C, kThreads, smem, st>>>(a);
  return cudaGetLastError();
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
