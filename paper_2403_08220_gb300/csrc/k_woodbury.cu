// Per-chain kernels of the surrogate mMALA step when d_y < r (Woodbury form).
//
// With K = J / sigma (d_y x r, sigma^2 = noise_var), eps = (f - y) / sigma,
// H = K^T K, g = K^T eps and M = I_{d_y} + K K^T = R R^T (lower Cholesky
// factor), the push-through and Woodbury identities give (exact in real
// arithmetic):
//   log det(I_r + H) = log det M,           (I + H)^-1 K^T = K^T M^-1,
//   (I + H)^-1 (x + g) = x - K^T M^-1 u,     u = K x - eps,
//   w = H x - g = K^T u,   w^T (I + H)^-1 w = |u|^2 - |R^-1 u|^2,
//   mhat^T w = (K mhat)^T u,   mhat^T H mhat = |K mhat|^2,
// and the perturbation noise (I + H)^-1 (xi1 + K^T xi2) = xi1 + K^T M^-1 (xi2 - K xi1).
// The proposal from x (eq:reduced_space_sampling with that noise) is then
//   mu      = s x + (1 - s) K^T v,                  v = M^-1 u,
//   m_r^dag = s x + sqrt(1-s^2) xi1 + K^T M^-1 y,   y = (1-s) u + sqrt(1-s^2) (xi2 - K xi1),
// with K mhat = K xi1 + (y - M^-1 y) / sqrt(1-s^2) for the forward move, and
// log rho_{0,r} (Sec. 5.4) needs only d_y-vectors: the d_y x d_y matrix M is
// the only one factored.
//
// State per chain: J at the current point (Js) and a factor slot holding the
// packed factor of M bordered by u^T (its row d_y is R^-1 u), 1 / R_ii, u, v
// and t1 = |u|^2 - |R^-1 u|^2, double-buffered like the r-sized path's slots.
//
//   k_wb_propose   the proposal and log rho_{0,r}(m_r, m_r^dag) from the state;
//   k_wb_geometry  at m_r^dag: misfit, K m_r^dag and K m_r, M and its bordered
//                  factor, log rho_{0,r}(m_r^dag, m_r), log rho_r^(1)
//                  (eq:da_dino_trr_1), the accept test and the state update
//                  (mode 1); mode 0 makes m_r^dag the state;
//   k_rowprod      K m_r^dag and K m_r for k_wb_geometry, when the Gram
//                  matrices K K^T come from the tensor cores (k_tc_gram):
//                  the geometry kernel then reads both instead of its own
//                  pass over J.
// The tensor-core path (FP32 J) computes in double-float arithmetic on the
// FP32 pipe, the FP64 path in FP64.
#include "chol.cuh"

namespace dino {
namespace {

constexpr int kWbThreads = 128;
constexpr int kWbPreThreads = 256;  // geometry with the Gram matrix and K b, K a formed beforehand
constexpr int kWbMinBlocks = 4;     // CTAs per SM the register budget is sized for

// Slot offsets (8-byte elements).
struct WbSlot {
  size_t R, inv, u, v, t1;
  __host__ __device__ explicit WbSlot(int dy) {
    R = 0;
    inv = tri_size(dy + 1);
    u = inv + dy + 1;
    v = u + dy;
    t1 = v + dy;
  }
};

// Shared-memory layout in 8-byte elements:
//   Ms[tri(dy+1)] inv[dy+1] | r-vectors: vb va be ae | dy-vectors: Kb Ka u sv eE zE vE
//   | red[kRed] flag lu | staging of J (FP64 geometry only)
// On the tensor-core path J is staged inside Ms, which holds nothing until
// the Gram tiles are written (wb_stage_fits).
struct WbLayout {
  size_t Ms, inv, vb, va, be, ae, Kb, Ka, u, sv, eE, zE, vE, red, flag, lu, tail;
  __host__ __device__ WbLayout(int r, int dy) {
    Ms = 0;
    inv = (tri_size(dy + 1) + 1) & ~(size_t)1;
    vb = inv + dy + 1;
    va = vb + r;
    be = va + r;
    ae = be + r;
    Kb = ae + r;
    Ka = Kb + dy;
    u = Ka + dy;
    sv = u + dy;
    eE = sv + dy;
    zE = eE + dy;
    vE = zE + dy;
    red = vE + dy;
    flag = red + kRed;
    lu = flag + 1;  // log u of the accept test
    tail = (lu + 1 + 1) & ~(size_t)1;
  }
};

template <typename TJ>
__host__ __device__ size_t wb_stage_bytes(int r, int dy);

// y1 = (K x1) and, when `two`, y2 = (K x2) as doubles: warp per row of J,
// lanes along the row (coalesced), the row sums combined by shuffles.
template <class A, typename TJ>
__device__ void rows_times(const TJ *J, int dy, int r, double inv_sigma, const typename A::T *x1,
                           const typename A::T *x2, bool two, double *y1, double *y2) {
  using E = typename A::T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < dy; i += nw) {
    const TJ *Ji = J + (size_t)i * r;
    typename A::Acc a1 = A::begin(E{}), a2 = A::begin(E{});
#pragma unroll 4
    for (int k = lane; k < r; k += 32) {
      const E jk = A::from_j(Ji[k]);
      A::sub(a1, jk, A::neg(x1[k]));
      if (two) A::sub(a2, jk, A::neg(x2[k]));
    }
    const E s1 = warp_sum_elt<A>(A::end(a1));
    const E s2 = warp_sum_elt<A>(A::end(a2));
    if (lane == 0) {
      y1[i] = A::to(s1) * inv_sigma;
      if (two) y2[i] = A::to(s2) * inv_sigma;
    }
  }
  __syncthreads();
}

constexpr int kWbKc = 16;          // J columns per staged chunk (tensor-core path)
constexpr int kWbLd = kWbKc + 4;   // padded row length (floats) of a staged chunk

// Entry of M = I + G / noise_var in double-float from the FP32 Gram value x:
// x (nh + nl) with (nh, nl) = 1 / noise_var as a double-float pair, and 1
// added on the diagonal.
__device__ __forceinline__ float2 gram_entry(float x, float nh, float nl, bool diag) {
  const float ph = __fmul_rn(x, nh);
  float e = __fmaf_rn(x, nh, -ph);
  e = __fmaf_rn(x, nl, e);
  float h, l;
  fast_two_sum(ph, e, h, l);
  if (diag) {
    float s1, q1;
    two_sum(1.0f, h, s1, q1);
    fast_two_sum(s1, __fadd_rn(q1, l), h, l);
  }
  return make_float2(h, l);
}

// y = K x (= J x / sigma) from the chain's FP32 J with 16-byte rows (r a
// multiple of 4), x as float pairs in shared memory: eight lanes per row,
// four rows per warp and blockDim / 8 rows per pass, lane q taking the column
// quads q, q + 8, ... straight from global memory; the eight double-float
// partial sums of a row meet in a three-level butterfly.  Every lane runs the
// same passes (rows past the end compute row d_y - 1 and store nothing).
__device__ void rows_times_quads(const float *J, int dy, int r, double inv_sigma,
                                 const float2 *x, double *y) {
  const int q = threadIdx.x & 7, groups = blockDim.x >> 3, nq = r / 4;
  const int passes = (dy + groups - 1) / groups;
  for (int ps = 0; ps < passes; ++ps) {
    const int row = ps * groups + (threadIdx.x >> 3), rr = min(row, dy - 1);
    const float4 *J4 = reinterpret_cast<const float4 *>(J + (size_t)rr * r);
    DF::Acc acc = DF::begin(float2{});
    for (int k = q; k < nq; k += 8) {
      const float4 j = J4[k];
      const float2 *xk = x + 4 * k;
      DF::sub_f(acc, j.x, DF::neg(xk[0]));
      DF::sub_f(acc, j.y, DF::neg(xk[1]));
      DF::sub_f(acc, j.z, DF::neg(xk[2]));
      DF::sub_f(acc, j.w, DF::neg(xk[3]));
    }
    float2 v = DF::end(acc);
#pragma unroll
    for (int o = 4; o; o >>= 1) v = DF::add(v, shfl_xor_elt(v, o));
    if (q == 0 && row < dy) y[row] = DF::to(v) * inv_sigma;
  }
}

// Shared bytes of the two staging buffers of wb_gram_rows.
__host__ __device__ inline size_t wb_stage2_bytes(int dy) {
  return 2 * (size_t)((dy + kHT - 1) / kHT * kHT) * kWbLd * sizeof(float);
}

// The two FP32 staging buffers fit in the factor's region when
// 2 ceil4(d_y) kWbLd floats <= tri(d_y + 1) doubles (from d_y of about 36 up).
__host__ __device__ inline bool wb_stage_fits(int dy) {
  return wb_stage2_bytes(dy) <= ((tri_size(dy + 1) + 1) & ~(size_t)1) * sizeof(double);
}

// A ring of four staging buffers (three chunks of J in flight) for the
// row-products-only passes, when it fits in the factor's region.
__host__ __device__ inline bool wb_ring4_fits(int dy) {
  return 2 * wb_stage2_bytes(dy) <= ((tri_size(dy + 1) + 1) & ~(size_t)1) * sizeof(double);
}

template <typename TJ>
__host__ __device__ size_t wb_stage_bytes(int r, int dy) {
  if (sizeof(TJ) == 4) return wb_stage_fits(dy) ? 0 : wb_stage2_bytes(dy);
  return (size_t)kJChunk * dy * sizeof(double);
}

// M = I + J J^T / noise_var (double-float entries, FP32 register tiles) and,
// from the same pass over J, Kb = (J b) / sigma and Ka = (J a) / sigma
// (double-float dot products, a thread per row, or two per row taking
// alternate columns when there are threads for it).  J (dy x r, row-major FP32)
// streams through a ring of kDepth shared buffers in chunks of kWbKc columns
// by asynchronous copies, kDepth - 1 chunks in flight while one is used;
// rows are kept in natural order (padded to kWbLd floats) and read as float4
// along the reduction index.
// kGram = false: only the row products (no Gram tiles, Ms untouched).
template <class A, bool kGram = true, int kDepth = 2>
__device__ void wb_gram_rows(const float *J, int dy, int r, double inv_nv, double inv_sigma,
                             float2 *Ms, float *stage, const float2 *be, const float2 *ae,
                             bool two, double *Kb, double *Ka) {
  const int tid = threadIdx.x, T = blockDim.x;
  const bool split = 2 * dy <= T;  // two threads per row of the row products
  const int nt = (dy + kHT - 1) / kHT, dyp = nt * kHT;
  const int ntiles = nt * (nt + 1) / 2;
  const int nch = (r + kWbKc - 1) / kWbKc;
  const bool vec = (r % 4) == 0;  // 16-byte aligned rows
  const size_t bstride = (size_t)dyp * kWbLd;  // floats between consecutive buffers
  for (int e = tid; e < (dyp - dy) * kWbLd; e += T)  // padding rows stay zero
#pragma unroll
    for (int q = 0; q < kDepth; ++q) stage[q * bstride + (size_t)dy * kWbLd + e] = 0.0f;
  auto issue = [&](int ch) {
    float *dst = stage + (ch % kDepth) * bstride;
    const int k0 = ch * kWbKc;
    if (vec) {
      for (int e = tid; e < dy * (kWbKc / 4); e += T) {
        const int j = e / (kWbKc / 4), k = 4 * (e % (kWbKc / 4));
        const int left = r - (k0 + k);
        const int bytes = left >= 4 ? 16 : (left > 0 ? 4 * left : 0);
        const float *src = J + (size_t)j * r + (left > 0 ? k0 + k : 0);
        cp_async16(dst + (size_t)j * kWbLd + k, src, bytes);
      }
    } else {
      for (int e = tid; e < dy * kWbKc; e += T) {
        const int j = e / kWbKc, k = e % kWbKc;
        const bool in = k0 + k < r;
        cp_async4(dst + (size_t)j * kWbLd + k, J + (size_t)j * r + (in ? k0 + k : 0), in ? 4 : 0);
      }
    }
    cp_async_commit();
  };

  int ti[kHMaxTiles], tj[kHMaxTiles];
  float acc[kHMaxTiles][kHT][kHT];
#pragma unroll
  for (int s = 0; s < kHMaxTiles; ++s) {
    const int tt = tid + s * T;
    if (tt < ntiles) {
      tri_pos(tt, ti[s], tj[s]);
    } else {
      ti[s] = -1;
      tj[s] = 0;
    }
#pragma unroll
    for (int p = 0; p < kHT; ++p)
#pragma unroll
      for (int q = 0; q < kHT; ++q) acc[s][p][q] = 0.0f;
  }
  typename A::Acc kb[2] = {A::begin(float2{}), A::begin(float2{})};
  typename A::Acc ka[2] = {A::begin(float2{}), A::begin(float2{})};

  // one commit group per chunk (empty past the end), so that waiting until
  // kDepth - 1 groups are pending completes chunk ch
  for (int ch = 0; ch < kDepth - 1; ++ch) {
    if (ch < nch) issue(ch);
    else cp_async_commit();
  }
  for (int ch = 0; ch < nch; ++ch) {
    // refills the buffer of chunk ch - 1, released by the barrier ending its use
    if (ch + kDepth - 1 < nch) issue(ch + kDepth - 1);
    else cp_async_commit();
    cp_async_wait<kDepth - 1>();
    __syncthreads();
    const float *x = stage + (ch % kDepth) * bstride;
    const int k0 = ch * kWbKc;
#pragma unroll
    for (int kk = 0; kk < kWbKc; kk += 4) {
#pragma unroll
      for (int s = 0; s < kHMaxTiles; ++s) {
        if (!kGram || ti[s] < 0) continue;
        float4 xa[kHT], ya[kHT];
#pragma unroll
        for (int p = 0; p < kHT; ++p) {
          xa[p] = *reinterpret_cast<const float4 *>(x + (size_t)(kHT * ti[s] + p) * kWbLd + kk);
          ya[p] = *reinterpret_cast<const float4 *>(x + (size_t)(kHT * tj[s] + p) * kWbLd + kk);
        }
#pragma unroll
        for (int p = 0; p < kHT; ++p)
#pragma unroll
          for (int q = 0; q < kHT; ++q) {
            float v = acc[s][p][q];
            v = fmaf(xa[p].x, ya[q].x, v);
            v = fmaf(xa[p].y, ya[q].y, v);
            v = fmaf(xa[p].z, ya[q].z, v);
            v = fmaf(xa[p].w, ya[q].w, v);
            acc[s][p][q] = v;
          }
      }
    }
    if (split) {  // row tid >> 1, columns of parity tid & 1 of the chunk
      const int j = tid >> 1;
      if (j < dy) {
        const float *row = x + (size_t)j * kWbLd;
        const int kn = min(kWbKc, r - k0);
        for (int k = tid & 1; k < kn; k += 2) {
          const float2 jk = A::from_j(row[k]);
          A::sub(kb[0], jk, A::neg(be[k0 + k]));
          if (two) A::sub(ka[0], jk, A::neg(ae[k0 + k]));
        }
      }
    } else {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = tid + h * T;
        if (j < dy) {
          const float *row = x + (size_t)j * kWbLd;
          const int kn = min(kWbKc, r - k0);
          for (int k = 0; k < kn; ++k) {
            const float2 jk = A::from_j(row[k]);
            A::sub(kb[h], jk, A::neg(be[k0 + k]));
            if (two) A::sub(ka[h], jk, A::neg(ae[k0 + k]));
          }
        }
      }
    }
    __syncthreads();
  }
  if (split) {  // the two halves of each row meet in adjacent lanes
    const float2 b0 = A::end(kb[0]), b1 = shfl_xor_elt(b0, 1);
    const float2 a0 = A::end(ka[0]), a1 = shfl_xor_elt(a0, 1);
    const int j = tid >> 1;
    if (j < dy && (tid & 1) == 0) {
      Kb[j] = A::to(A::add(b0, b1)) * inv_sigma;
      if (two) Ka[j] = A::to(A::add(a0, a1)) * inv_sigma;
    }
  } else {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = tid + h * T;
      if (j < dy) {
        Kb[j] = A::to(A::end(kb[h])) * inv_sigma;
        if (two) Ka[j] = A::to(A::end(ka[h])) * inv_sigma;
      }
    }
  }
  const float nh = __double2float_rn(inv_nv), nl = __double2float_rn(inv_nv - (double)nh);
#pragma unroll
  for (int s = 0; s < kHMaxTiles; ++s) {
    if (!kGram || ti[s] < 0) continue;
#pragma unroll
    for (int p = 0; p < kHT; ++p)
#pragma unroll
      for (int q = 0; q < kHT; ++q) {
        const int i = kHT * ti[s] + p, j = kHT * tj[s] + q;
        if (i < dy && j <= i) Ms[tri(i) + j] = gram_entry(acc[s][p][q], nh, nl, i == j);
      }
  }
  __syncthreads();
}

template <typename TJ, class A>
__device__ void wb_store_factor(double *Lg, const typename A::T *Ms, const typename A::T *inv,
                                const double *u, const double *v, double t1, int dy) {
  using E = typename A::T;
  const WbSlot sl(dy);
  E *G = reinterpret_cast<E *>(Lg);
  for (size_t e = threadIdx.x; e < tri_size(dy + 1); e += blockDim.x) G[sl.R + e] = Ms[e];
  for (int i = threadIdx.x; i <= dy; i += blockDim.x) G[sl.inv + i] = inv[i];
  for (int i = threadIdx.x; i < dy; i += blockDim.x) {
    Lg[sl.u + i] = u[i];
    Lg[sl.v + i] = v[i];
  }
  if (threadIdx.x == 0) Lg[sl.t1] = t1;
}

// One CTA of NT threads per chain at the point b (see the file comment).
// kPre: the Gram matrix J J^T and K b, K a come formed (the tensor-core
// path); this instantiation is kept lean in registers so that NT = 256
// threads (64 registers each) fit four CTAs on an SM.
template <typename TJ, bool kPre, int NT>
__global__ void __launch_bounds__(NT, kWbMinBlocks) k_wb_geometry(ReducedArgs a, int mode) {
  using A = std::conditional_t<sizeof(TJ) == 4, DF, F64>;
  using E = typename A::T;
  static_assert(sizeof(E) == sizeof(double), "one factor element per double of the slot");
  extern __shared__ __align__(16) double sm[];
  const int c = blockIdx.x, r = a.r, dy = a.d_y;
  const WbLayout lay(r, dy);
  const WbSlot sl(dy);
  const size_t ldW = wb_slot_stride(dy);
  const int slot = mode == 0 ? a.cur[c] : 1 - a.cur[c];
  double *Lg = a.L + (size_t)slot * a.L_slot + (size_t)c * ldW;
  E *Ms = reinterpret_cast<E *>(sm + lay.Ms);
  E *inv = reinterpret_cast<E *>(sm + lay.inv);
  double *vb = sm + lay.vb, *va = sm + lay.va;
  E *be = reinterpret_cast<E *>(sm + lay.be), *ae = reinterpret_cast<E *>(sm + lay.ae);
  double *Kb = sm + lay.Kb, *Ka = sm + lay.Ka, *u = sm + lay.u, *sv = sm + lay.sv;
  E *vE = reinterpret_cast<E *>(sm + lay.vE);
  double *red = sm + lay.red;
  int *flag = reinterpret_cast<int *>(sm + lay.flag);
  double *log_u_s = sm + lay.lu;
  const TJ *J = reinterpret_cast<const TJ *>(a.J) + (size_t)c * dy * r;
  const TJ *f = reinterpret_cast<const TJ *>(a.f) + (size_t)c * dy;
  const double inv_nv = a.inv_nv, inv_sigma = a.inv_sigma;
  // log u, off the accept test's critical path (read after several barriers)
  if (mode == 1 && threadIdx.x == blockDim.x - 1) *log_u_s = draw_log_u(a, c);
  // kPre: this chain's Gram matrix (d_y x ldg FP32) streams into the top of
  // the factor's region by 16-byte asynchronous copies while the state loads
  // and the misfit below proceed
  float *gstage = nullptr;
  if constexpr (kPre) {
    const int gbytes = dy * a.ldg * 4;
    gstage = reinterpret_cast<float *>(reinterpret_cast<char *>(sm + lay.Ms) +
                                       (lay.inv * sizeof(double) - gbytes));
    const char *src = reinterpret_cast<const char *>(a.G + (size_t)c * dy * a.ldg);
    for (int o = threadIdx.x * 16; o < gbytes; o += blockDim.x * 16)
      cp_async16(reinterpret_cast<char *>(gstage) + o, src + o, 16);
    cp_async_commit();
  }

  for (int k = threadIdx.x; k < r; k += blockDim.x) {
    vb[k] = a.b[(size_t)c * r + k];
    va[k] = mode == 1 ? a.mr[(size_t)c * r + k] : 0.0;
    if (!kPre && !a.Kb_pre) {  // operands of this kernel's own K b, K a pass
      be[k] = A::from(vb[k]);
      ae[k] = A::from(va[k]);
    }
  }
  double ph = 0.0;
  for (int i = threadIdx.x; i < dy; i += blockDim.x) {
    const double rs = (double)f[i] - a.y[i];
    sv[i] = rs;  // f - y, until the factor's row replaces it
    ph += rs * rs;
  }
  const double phi_b = 0.5 * block_sum(ph, red) * inv_nv;  // includes a barrier
  if constexpr (sizeof(TJ) == 4) {  // M, K b and K a from one pass over J
    float *stage = wb_stage_fits(dy) ? reinterpret_cast<float *>(sm + lay.Ms)
                                     : reinterpret_cast<float *>(sm + lay.tail);
    if (kPre || a.G) {  // Gram matrix formed on the tensor cores: K b, K a only, then M from G
      if (kPre || a.Kb_pre) {  // ... and K b, K a too (the Jacobian GEMM's epilogue)
        for (int i = threadIdx.x; i < dy; i += blockDim.x) {
          Kb[i] = a.Kb_pre[(size_t)c * dy + i];
          if (mode == 1) Ka[i] = a.Ka_pre[(size_t)c * dy + i];
        }
      } else if (wb_ring4_fits(dy)) {
        wb_gram_rows<A, false, 4>(reinterpret_cast<const float *>(J), dy, r, inv_nv, inv_sigma,
                                  reinterpret_cast<float2 *>(Ms), stage,
                                  reinterpret_cast<const float2 *>(be),
                                  reinterpret_cast<const float2 *>(ae), mode == 1, Kb, Ka);
      } else {
        wb_gram_rows<A, false>(reinterpret_cast<const float *>(J), dy, r, inv_nv, inv_sigma,
                               reinterpret_cast<float2 *>(Ms), stage,
                               reinterpret_cast<const float2 *>(be),
                               reinterpret_cast<const float2 *>(ae), mode == 1, Kb, Ka);
      }
      const float nh = __double2float_rn(inv_nv), nl = __double2float_rn(inv_nv - (double)nh);
      constexpr int kLoads = 8;
      const int ntri = tri(dy);
      if constexpr (kPre) {
        // M in place from the staged G, bottom-up in chunks of kLoads
        // entries per thread: a chunk's entries are all read before any is
        // written, and its writes end below the staged rows of the chunks
        // after it (wb_pre_stage_fits)
        cp_async_wait<0>();
        __syncthreads();
        // the same number of passes in every thread (barriers inside)
        for (int e00 = 0; e00 < ntri; e00 += kLoads * blockDim.x) {
          const int e0 = e00 + threadIdx.x;
          float x[kLoads];
          int dg = 0;
#pragma unroll
          for (int q = 0; q < kLoads; ++q) {
            const int e = e0 + q * blockDim.x;
            x[q] = 0.0f;
            if (e < ntri) {
              int i, j;
              tri_pos(e, i, j);
              x[q] = gstage[(size_t)i * a.ldg + j];
              dg |= (i == j) << q;
            }
          }
          __syncthreads();
#pragma unroll
          for (int q = 0; q < kLoads; ++q) {
            const int e = e0 + q * blockDim.x;
            if (e < ntri) reinterpret_cast<float2 *>(Ms)[e] = gram_entry(x[q], nh, nl, (dg >> q) & 1);
          }
          __syncthreads();
        }
      }
      // otherwise from global memory: the packed lower triangle in order,
      // kLoads independent loads in flight per thread
      const float *Gc = a.G + (size_t)c * dy * a.ldg;
      for (int e0 = threadIdx.x; e0 < (kPre ? 0 : ntri); e0 += kLoads * blockDim.x) {
        float x[kLoads];
        int ii[kLoads], jj[kLoads];
#pragma unroll
        for (int q = 0; q < kLoads; ++q) {
          const int e = e0 + q * blockDim.x;
          ii[q] = jj[q] = 0;
          x[q] = 0.0f;
          if (e < ntri) {
            tri_pos(e, ii[q], jj[q]);
            x[q] = Gc[(size_t)ii[q] * a.ldg + jj[q]];
          }
        }
#pragma unroll
        for (int q = 0; q < kLoads; ++q) {
          const int e = e0 + q * blockDim.x;
          if (e < ntri) reinterpret_cast<float2 *>(Ms)[e] = gram_entry(x[q], nh, nl, ii[q] == jj[q]);
        }
      }
      __syncthreads();
    } else if constexpr (!kPre) {
      wb_gram_rows<A>(reinterpret_cast<const float *>(J), dy, r, inv_nv, inv_sigma,
                      reinterpret_cast<float2 *>(Ms), stage,
                      reinterpret_cast<const float2 *>(be), reinterpret_cast<const float2 *>(ae),
                      mode == 1, Kb, Ka);
    }
  } else {
    rows_times<A, TJ>(J, dy, r, inv_sigma, be, ae, mode == 1, Kb, Ka);  // K b, K a
    form_gram_f64<true>(reinterpret_cast<const double *>(J), r, dy, r, inv_nv,
                        reinterpret_cast<double *>(Ms), sm + lay.tail);
  }
  double uu = 0.0;
  for (int i = threadIdx.x; i < dy; i += blockDim.x) {
    u[i] = Kb[i] - sv[i] * inv_sigma;  // u = K b - eps
    uu += u[i] * u[i];
  }
  // bordered row u^T with pivot 1 + |u|^2 (the last pivot stays >= 1: |R^-1 u| <= |u|)
  uu = block_sum(uu, red);
  for (int i = threadIdx.x; i < dy; i += blockDim.x) Ms[tri(dy) + i] = A::from(u[i]);
  if (threadIdx.x == 0) Ms[tri(dy) + dy] = A::from(1.0 + uu);
  __syncthreads();
  cta_cholesky_panels<A>(Ms, inv, dy + 1);
  double ld = 0.0, ss = 0.0;
  for (int i = threadIdx.x; i < dy; i += blockDim.x) {
    ld += log(A::to(Ms[tri(i) + i]));
    sv[i] = A::to(Ms[tri(dy) + i]);  // R^-1 u
    ss += sv[i] * sv[i];
  }
  const double hld_b = block_sum(ld, red);
  const double t1 = uu - block_sum(ss, red);  // w^T (I+H)^-1 w at b

  // v = M^-1 u = R^-T (R^-1 u), needed by the next proposal from b
  auto solve_v = [&]() {
    for (int i = threadIdx.x; i < dy; i += blockDim.x) vE[i] = A::from(sv[i]);
    __syncthreads();
    cta_upper_solve_t<A>(Ms, inv, dy, vE);
    double *vv = Ka;  // K a is no longer needed
    for (int i = threadIdx.x; i < dy; i += blockDim.x) vv[i] = A::to(vE[i]);
    __syncthreads();
    return vv;
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
    const double *vv = solve_v();
    wb_store_factor<TJ, A>(Lg, Ms, inv, u, vv, t1, dy);
    take_state();
    if (threadIdx.x == 0) {
      a.phi[c] = phi_b;
      a.hld[c] = hld_b;
    }
    return;
  }
  const double s = a.s, inv_cs = a.inv_cs;
  double t2 = 0.0, t3 = 0.0, unused = 0.0;
  for (int i = threadIdx.x; i < dy; i += blockDim.x) {
    const double km = (Ka[i] - s * Kb[i]) * inv_cs;  // K mhat for b -> a
    t2 += km * u[i];
    t3 += km * km;
  }
  block_sum3(t2, t3, unused, red);
  double lr = 0.0;
  if (threadIdx.x == 0) {
    const double lq_rev = -a.dt / 8.0 * t1 + a.sqrt_dt / 2.0 * t2 + hld_b - 0.5 * t3;
    lr = a.phi[c] - phi_b + lq_rev - a.lq_fwd[c];
    *flag = accept_decide(lr, *log_u_s) ? 1 : 0;
  }
  __syncthreads();
  const bool accept = *flag != 0;
  if (threadIdx.x == 0) accept_record(a, c, lr, *log_u_s, accept, phi_b, hld_b);
  for (int k = threadIdx.x; k < r; k += blockDim.x) a.coef[(size_t)c * r + k] = vb[k] - s * va[k];
  if (accept) {
    const double *vv = solve_v();
    wb_store_factor<TJ, A>(Lg, Ms, inv, u, vv, t1, dy);
    if (!a.da) take_state();  // delayed acceptance: the second stage commits
  }
}

// One CTA per chain at the state x = m_r (see the file comment).
template <typename TJ, int NT>
__global__ void __launch_bounds__(NT, kWbMinBlocks) k_wb_propose(ReducedArgs a) {
  using A = std::conditional_t<sizeof(TJ) == 4, DF, F64>;
  using E = typename A::T;
  extern __shared__ __align__(16) double sm[];
  const int c = blockIdx.x, r = a.r, dy = a.d_y;
  const WbLayout lay(r, dy);
  const WbSlot sl(dy);
  const double *Lg = a.L + (size_t)a.cur[c] * a.L_slot + (size_t)c * wb_slot_stride(dy);
  const E *G = reinterpret_cast<const E *>(Lg);
  E *Ms = reinterpret_cast<E *>(sm + lay.Ms);
  E *inv = reinterpret_cast<E *>(sm + lay.inv);
  double *xa = sm + lay.vb, *xi1 = sm + lay.va;
  E *x1E = reinterpret_cast<E *>(sm + lay.be);
  double *Kxi = sm + lay.Kb, *xi2 = sm + lay.Ka, *u = sm + lay.u, *yv = sm + lay.sv;
  E *zE = reinterpret_cast<E *>(sm + lay.zE), *vE = reinterpret_cast<E *>(sm + lay.vE);
  double *red = sm + lay.red;
  const TJ *J = reinterpret_cast<const TJ *>(a.Js) + (size_t)c * dy * r;
  const double inv_sigma = a.inv_sigma;
  const double s = a.s, cs = a.cs;

  for (int i = threadIdx.x; i < dy; i += blockDim.x) {
    inv[i] = G[sl.inv + i];
    u[i] = Lg[sl.u + i];
    vE[i] = A::from((1.0 - s) * Lg[sl.v + i]);
  }
  const uint32_t chain = (uint32_t)(a.id_base + (uint64_t)c);
  for (int k = threadIdx.x; k < r; k += blockDim.x) xa[k] = a.mr[(size_t)c * r + k];
  // Box-Muller in FP32 on the tensor-core path (its precision bars are far
  // above FP32's; an FP32 normal is an exact double-float pair (x, 0), so no
  // FP64 conversion is needed), in FP64 on the FP64 path (FP64 parity with
  // the oracle)
  auto normals4 = [&](uint4 w, double n4[4], E e4[4]) {
    if constexpr (sizeof(TJ) == 4) {
      float f4[4];
      normals4_f32(w, f4);
      for (int q = 0; q < 4; ++q) {
        n4[q] = f4[q];
        e4[q] = A::from_j(f4[q]);
      }
    } else {
      normals4_f64(w, n4);
      for (int q = 0; q < 4; ++q) e4[q] = A::from(n4[q]);
    }
  };
  // caller-supplied normals (FP64) instead of Philox
  auto ext4 = [&](const double *x, int n, int blk, double n4[4], E e4[4]) {
    for (int q = 0; q < 4; ++q) {
      n4[q] = 4 * blk + q < n ? x[(size_t)c * n + 4 * blk + q] : 0.0;
      e4[q] = A::from(n4[q]);
    }
  };
  for (int blk = threadIdx.x; blk < (r + 3) / 4; blk += blockDim.x) {
    double n4[4];
    E e4[4];
    if (a.ext_xi)
      ext4(a.ext_xi, r, blk, n4, e4);
    else
      normals4(philox_block(a.seed, STREAM_XI, a.step, chain, blk), n4, e4);
    for (int q = 0; q < 4; ++q)
      if (4 * blk + q < r) {
        xi1[4 * blk + q] = n4[q];
        x1E[4 * blk + q] = e4[q];
      }
  }
  for (int blk = threadIdx.x; blk < (dy + 3) / 4; blk += blockDim.x) {
    double n4[4];
    E e4[4];
    if (a.ext_xi2)
      ext4(a.ext_xi2, dy, blk, n4, e4);
    else
      normals4(philox_block(a.seed, STREAM_XI2, a.step, chain, blk), n4, e4);
    for (int q = 0; q < 4; ++q)
      if (4 * blk + q < dy) xi2[4 * blk + q] = n4[q];
  }
  __syncthreads();
  if constexpr (sizeof(TJ) == 4) {  // K xi1: by row quads, else J staged through the factor region
    if ((r & 3) == 0 && (reinterpret_cast<uintptr_t>(J) & 15) == 0) {
      rows_times_quads(reinterpret_cast<const float *>(J), dy, r, inv_sigma,
                       reinterpret_cast<const float2 *>(x1E), Kxi);
      __syncthreads();
    } else if (wb_ring4_fits(dy)) {
      wb_gram_rows<A, false, 4>(reinterpret_cast<const float *>(J), dy, r, 0.0, inv_sigma,
                                nullptr, reinterpret_cast<float *>(sm + lay.Ms),
                                reinterpret_cast<const float2 *>(x1E), nullptr, false, Kxi, Kxi);
    } else if (wb_stage_fits(dy)) {
      wb_gram_rows<A, false>(reinterpret_cast<const float *>(J), dy, r, 0.0, inv_sigma, nullptr,
                             reinterpret_cast<float *>(sm + lay.Ms),
                             reinterpret_cast<const float2 *>(x1E), nullptr, false, Kxi, Kxi);
    } else {
      rows_times<A, TJ>(J, dy, r, inv_sigma, x1E, x1E, false, Kxi, Kxi);
    }
  } else {
    rows_times<A, TJ>(J, dy, r, inv_sigma, x1E, x1E, false, Kxi, Kxi);  // K xi1
  }
  {  // the factor by 16-byte asynchronous copies (slots start on 16 bytes), all in flight
    const size_t ne = tri_size(dy), npair = ne / 2;
    for (size_t q = threadIdx.x; q < npair; q += blockDim.x)
      cp_async16(Ms + 2 * q, G + sl.R + 2 * q, 16);
    cp_async_commit();
    if (threadIdx.x == 0 && (ne & 1)) Ms[ne - 1] = G[sl.R + ne - 1];
    cp_async_wait<0>();
  }
  for (int i = threadIdx.x; i < dy; i += blockDim.x) {
    yv[i] = (1.0 - s) * u[i] + cs * (xi2[i] - Kxi[i]);
    zE[i] = A::from(yv[i]);
  }
  __syncthreads();
  cta_lower_solve_t<A>(Ms, inv, dy, zE);
  cta_upper_solve_t<A>(Ms, inv, dy, zE);  // z = M^-1 y
  // K^T z and K^T ((1-s) v): thread per column of J (coalesced across threads)
  for (int k = threadIdx.x; k < r; k += blockDim.x) {
    typename A::Acc az = A::begin(E{}), av = A::begin(E{});
#pragma unroll 8
    for (int i = 0; i < dy; ++i) {
      const E jk = A::from_j(J[(size_t)i * r + k]);
      A::sub(az, jk, A::neg(zE[i]));
      A::sub(av, jk, A::neg(vE[i]));
    }
    const double bk = s * xa[k] + cs * xi1[k] + A::to(A::end(az)) * inv_sigma;
    const double mk = s * xa[k] + A::to(A::end(av)) * inv_sigma;
    a.mu[(size_t)c * r + k] = mk;
    a.b[(size_t)c * r + k] = bk;
    if constexpr (sizeof(TJ) == 4)
      if (a.b_df) a.b_df[(size_t)c * r + k] = A::from(bk);
    if (a.b_bf16) split_bf16_store(bk, a.b_bf16 + (size_t)c * a.b_ld + k, a.b_plane, a.b_slices);
  }
  double t2 = 0.0, t3 = 0.0, unused = 0.0;
  const double inv_cs = a.inv_cs;
  for (int i = threadIdx.x; i < dy; i += blockDim.x) {
    const double km = Kxi[i] + (yv[i] - A::to(zE[i])) * inv_cs;  // K mhat
    t2 += km * u[i];
    t3 += km * km;
  }
  block_sum3(t2, t3, unused, red);
  if (threadIdx.x == 0)
    a.lq_fwd[c] = -a.dt / 8.0 * Lg[sl.t1] + a.sqrt_dt / 2.0 * t2 + a.hld[c] - 0.5 * t3;
}

// K b and K a from the FP32 Jacobian: eight lanes per row (c, i), four rows
// per warp, and the eight double-float partial sums of a row combined by a
// three-level butterfly of double-float additions.  kVec (r a multiple of
// 4, so that rows of J and of b, a start on 16 bytes): lane q takes the
// column quads q, q + 8, ... (one 16-byte load of J and two of each vector
// per quad; a warp's load of J covers four rows' 128-byte segments); else
// lane q takes the columns q, q + 8, ...
constexpr int kRowLanes = 8;

template <bool kVec>
__global__ void k_rowprod(int rows, int r, int dy, const float *__restrict__ J,
                          const float2 *__restrict__ b, const float2 *__restrict__ a,
                          double kscale, double *__restrict__ Kb, double *__restrict__ Ka) {
  const int q = threadIdx.x & (kRowLanes - 1);
  const int groups = (gridDim.x * blockDim.x) / kRowLanes;
  // every lane runs the same number of iterations (rows past the end compute
  // row rows - 1 and store nothing), so the butterfly's shuffles see full warps
  const int iters = (rows + groups - 1) / groups;
  int row = (blockIdx.x * blockDim.x + threadIdx.x) / kRowLanes;
  for (int it = 0; it < iters; ++it, row += groups) {
    const int rr = min(row, rows - 1), c = rr / dy;
    const float *Jr = J + (size_t)rr * r;
    const float2 *br = b + (size_t)c * r;
    const float2 *ar = a ? a + (size_t)c * r : nullptr;
    DF::Acc kb = DF::begin(float2{}), ka = DF::begin(float2{});
    if constexpr (kVec) {
      const int nq = r / 4;
      for (int k = q; k < nq; k += kRowLanes) {
        const float4 jq = reinterpret_cast<const float4 *>(Jr)[k];
        const float4 b0 = reinterpret_cast<const float4 *>(br)[2 * k];
        const float4 b1 = reinterpret_cast<const float4 *>(br)[2 * k + 1];
        DF::sub_f(kb, jq.x, float2{-b0.x, -b0.y});
        DF::sub_f(kb, jq.y, float2{-b0.z, -b0.w});
        DF::sub_f(kb, jq.z, float2{-b1.x, -b1.y});
        DF::sub_f(kb, jq.w, float2{-b1.z, -b1.w});
        if (ar) {
          const float4 a0 = reinterpret_cast<const float4 *>(ar)[2 * k];
          const float4 a1 = reinterpret_cast<const float4 *>(ar)[2 * k + 1];
          DF::sub_f(ka, jq.x, float2{-a0.x, -a0.y});
          DF::sub_f(ka, jq.y, float2{-a0.z, -a0.w});
          DF::sub_f(ka, jq.z, float2{-a1.x, -a1.y});
          DF::sub_f(ka, jq.w, float2{-a1.z, -a1.w});
        }
      }
    } else {
#pragma unroll 5
      for (int k = q; k < r; k += kRowLanes) {
        const float jk = Jr[k];
        DF::sub_f(kb, jk, DF::neg(br[k]));
        if (ar) DF::sub_f(ka, jk, DF::neg(ar[k]));
      }
    }
    float2 vb = DF::end(kb), va = DF::end(ka);
#pragma unroll
    for (int o = kRowLanes / 2; o; o >>= 1) {
      vb = DF::add(vb, shfl_xor_elt(vb, o));
      if (ar) va = DF::add(va, shfl_xor_elt(va, o));
    }
    if (q == 0 && row < rows) {
      Kb[row] = DF::to(vb) * kscale;
      if (ar) Ka[row] = DF::to(va) * kscale;
    }
  }
}

__global__ void k_to_df(size_t n, const double *__restrict__ src, float2 *dst1, float2 *dst2) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const float2 x = DF::from(src[e]);
    if (dst1) dst1[e] = x;
    if (dst2) dst2[e] = x;
  }
}

template <typename TJ>
size_t wb_geometry_smem(int r, int dy) {
  return WbLayout(r, dy).tail * sizeof(double) + wb_stage_bytes<TJ>(r, dy);
}

template <typename TJ, bool kPre, int NT>
cudaError_t launch_wb_geometry_k(const ReducedArgs &a, int mode, cudaStream_t st) {
  const size_t smem = wb_geometry_smem<TJ>(a.r, a.d_y);
  cudaError_t e = cudaFuncSetAttribute(k_wb_geometry<TJ, kPre, NT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  ReducedArgs b = a;
  b.derive();
  k_wb_geometry<TJ, kPre, NT><<<a.C, NT, smem, st>>>(b, mode);
  return cudaGetLastError();
}

// The in-place conversion of the staged Gram matrix (kPre) is safe when, at
// every chunk boundary E (entries of 8 per thread of kWbPreThreads), the
// double-float writes below it (bytes [0, 8E)) end at or below the staged
// FP32 entry E, the first one not yet read.
bool wb_pre_stage_fits(int dy, int ldg) {
  const size_t region = WbLayout(1, dy).inv * sizeof(double);
  const size_t gbytes = (size_t)dy * ldg * 4;
  if (gbytes > region || gbytes % 16) return false;
  const size_t S = region - gbytes;
  const long ntri = (long)dy * (dy + 1) / 2, step = 8L * kWbPreThreads;
  for (long E = step; E < ntri; E += step) {
    long i = 0;
    while ((i + 1) * (i + 2) / 2 <= E) ++i;
    const long j = E - i * (i + 1) / 2;
    if ((size_t)(8 * E) > S + 4 * (size_t)(ldg * i + j)) return false;
  }
  return true;
}

template <typename TJ>
cudaError_t launch_wb_geometry_t(const ReducedArgs &a, int mode, cudaStream_t st) {
  if constexpr (sizeof(TJ) == 4)
    if (a.G && a.Kb_pre && wb_pre_stage_fits(a.d_y, a.ldg))
      return launch_wb_geometry_k<TJ, true, kWbPreThreads>(a, mode, st);
  return launch_wb_geometry_k<TJ, false, kWbThreads>(a, mode, st);
}

template <typename TJ>
cudaError_t launch_wb_propose_t(const ReducedArgs &a, cudaStream_t st) {
  const size_t smem = WbLayout(a.r, a.d_y).tail * sizeof(double);
  // the double-float path at 256 threads (64 registers, 32 warps per SM)
  constexpr int NT = sizeof(TJ) == 4 ? kWbPreThreads : kWbThreads;
  cudaError_t e = cudaFuncSetAttribute(k_wb_propose<TJ, NT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  ReducedArgs b = a;
  b.derive();
  k_wb_propose<TJ, NT><<<a.C, NT, smem, st>>>(b);
  return cudaGetLastError();
}

}  // namespace

size_t wb_smem_bytes(int r, int d_y, int jf_f32) {
  return jf_f32 ? wb_geometry_smem<float>(r, d_y) : wb_geometry_smem<double>(r, d_y);
}

cudaError_t launch_wb_geometry(const ReducedArgs &a, int mode, cudaStream_t st) {
  return a.jf_f32 ? launch_wb_geometry_t<float>(a, mode, st)
                  : launch_wb_geometry_t<double>(a, mode, st);
}

cudaError_t launch_wb_propose(const ReducedArgs &a, cudaStream_t st) {
  return a.jf_f32 ? launch_wb_propose_t<float>(a, st) : launch_wb_propose_t<double>(a, st);
}

cudaError_t launch_rowprod(int rows, int r, int d_y, const float *J, const float2 *b,
                           const float2 *a, double kscale, double *Kb, double *Ka,
                           cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  if (d_y < 1 || r < 1) return cudaErrorInvalidValue;
  const int grid = std::min((rows + 31) / 32, 152 * 16);  // 32 rows per 256-thread block
  const bool vec = r % 4 == 0 && ((uintptr_t)J & 15) == 0 && ((uintptr_t)b & 15) == 0 &&
                   ((uintptr_t)a & 15) == 0;
  if (vec)
    k_rowprod<true><<<grid, 256, 0, st>>>(rows, r, d_y, J, b, a, kscale, Kb, Ka);
  else
    k_rowprod<false><<<grid, 256, 0, st>>>(rows, r, d_y, J, b, a, kscale, Kb, Ka);
  return cudaGetLastError();
}

cudaError_t launch_to_df(size_t n, const double *src, float2 *dst1, float2 *dst2,
                         cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int grid = (int)std::min<size_t>((n + 255) / 256, 152 * 8);
  k_to_df<<<grid, 256, 0, st>>>(n, src, dst1, dst2);
  return cudaGetLastError();
}

}  // namespace dino
