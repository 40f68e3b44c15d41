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
#include <type_traits>

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
constexpr int kRed = 104;      // reduction scratch (doubles): block_sum3 [0, 99), Cholesky counters [100, 103)

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

// Three sums over the CTA at once; `red` holds >= kRed doubles.
__device__ void block_sum3(double &x, double &y, double &z, double *red) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    x += __shfl_xor_sync(kFull, x, o);
    y += __shfl_xor_sync(kFull, y, o);
    z += __shfl_xor_sync(kFull, z, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    red[warp] = x;
    red[32 + warp] = y;
    red[64 + warp] = z;
  }
  __syncthreads();
  if (warp == 0) {
    const bool in = lane < (int)(blockDim.x >> 5);
    double a = in ? red[lane] : 0.0, b = in ? red[32 + lane] : 0.0, c = in ? red[64 + lane] : 0.0;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      a += __shfl_xor_sync(kFull, a, o);
      b += __shfl_xor_sync(kFull, b, o);
      c += __shfl_xor_sync(kFull, c, o);
    }
    if (lane == 0) {
      red[96] = a;
      red[97] = b;
      red[98] = c;
    }
  }
  __syncthreads();
  x = red[96];
  y = red[97];
  z = red[98];
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

// Element arithmetic of the Cholesky factorisation and of the products with
// its factor.  F64: native FP64.  DF: double-float pairs (value = h + l with
// |l| <= ulp(h) / 2, a 48-bit significand) on the FP32 pipe, which GB300 runs
// at 64 times the FP64 rate: products are split exactly with an FMA, sums with
// Knuth's two-sum, and a dot product is accumulated as in the compensated
// Dot2 of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci.
// Comput. 26 (2005)), whose result is as accurate as if computed in twice the
// working precision.  Intrinsics with explicit rounding keep the compiler
// from contracting the error-free transformations.
struct F64 {
  using T = double;
  using Acc = double;
  __device__ static T from(double x) { return x; }
  __device__ static T from_j(double x) { return x; }
  __device__ static double to(T x) { return x; }
  __device__ static Acc begin(T a) { return a; }
  __device__ static void sub(Acc &a, T x, T y) { a -= x * y; }  // a <- a - x y
  __device__ static T end(Acc a) { return a; }
  __device__ static T mul(T a, T b) { return a * b; }
  __device__ static T neg(T a) { return -a; }
  // pivot d = sqrt(x) and id = 1 / d: y = x^(-1/2) from an FP32 estimate
  // refined by two Newton-Raphson steps on 1/y^2 - x = 0 (y <- y (3 - x y^2) / 2)
  __device__ static void pivot(T x, T &d, T &id) {
    double y = (double)rsqrtf((float)x);
    y = y * (1.5 - 0.5 * x * y * y);
    y = y * (1.5 - 0.5 * x * y * y);
    id = y;
    d = x * y;
  }
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly, given |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

struct DF {
  using T = float2;  // (h, l)
  struct Acc {
    float s, c;
  };
  __device__ static T from(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
  }
  __device__ static T from_j(float x) { return make_float2(x, 0.0f); }
  __device__ static double to(T x) { return (double)x.x + (double)x.y; }
  __device__ static Acc begin(T a) { return {a.x, a.y}; }
  // a <- a - x y: the high product p and its rounding error e are exact up
  // to the dropped l*l term; -p enters the running sum by two-sum, whose
  // error joins e in the compensation c.
  __device__ static void sub(Acc &a, T x, T y) {
    const float p = __fmul_rn(x.x, y.x);
    float e = __fmaf_rn(x.x, y.x, -p);
    e = __fmaf_rn(x.x, y.y, e);
    e = __fmaf_rn(x.y, y.x, e);
    float s, q;
    two_sum(a.s, -p, s, q);
    a.s = s;
    a.c = __fadd_rn(a.c, __fsub_rn(q, e));
  }
  __device__ static T end(Acc a) {
    float h, l;
    two_sum(a.s, a.c, h, l);
    return make_float2(h, l);
  }
  __device__ static T mul(T a, T b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    float h, l;
    fast_two_sum(p, e, h, l);
    return make_float2(h, l);
  }
  __device__ static T neg(T a) { return make_float2(-a.x, -a.y); }
  // The same pivot on the FP32 pipe: each Newton step y <- y + y (1 - x y^2) / 2
  // takes the residual 1 - x y^2 exactly (double-float product, two-sum
  // against 1) and the small correction in FP32.  From the FP32 estimate
  // (relative error ~2^-22) the first step reaches ~2^-43, the second the
  // double-float precision.  x <= 0 gives NaN, as in FP64.
  __device__ static void newton_rsqrt(T x, T &y) {
    const T y2 = mul(y, y);
    const T xy2 = mul(x, y2);
    float s, q;
    two_sum(1.0f, -xy2.x, s, q);
    const float res = __fadd_rn(s, __fsub_rn(q, xy2.y));
    const float c = __fmul_rn(__fmul_rn(0.5f, y.x), res);
    float h, l;
    two_sum(y.x, c, h, l);
    fast_two_sum(h, __fadd_rn(l, y.y), y.x, y.y);
  }
  __device__ static void pivot(T x, T &d, T &id) {
    T y = make_float2(rsqrtf(x.x), 0.0f);
    newton_rsqrt(x, y);
    newton_rsqrt(x, y);
    id = y;
    d = mul(x, y);
  }
};

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

// Position (ii, jj) of packed index e in a lower triangle.
__device__ __forceinline__ void tri_pos(int e, int &ii, int &jj) {
  ii = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while (tri(ii + 1) <= e) ++ii;
  while (tri(ii) > e) --ii;
  jj = e - tri(ii);
}

// Lane-to-lane copy of a factor element.
__device__ __forceinline__ double shfl_elt(double x, int src) {
  return __shfl_sync(kFull, x, src);
}
__device__ __forceinline__ float2 shfl_elt(float2 x, int src) {
  return make_float2(__shfl_sync(kFull, x.x, src), __shfl_sync(kFull, x.y, src));
}

// Factor the 8 x 8 diagonal block at kb (size nb) by one warp, in registers:
// lane i < nb holds row i of the block.  When pk >= 0 the block first takes
// the rank-8 update from the panel at pk (final by then).  At step q, c[k]
// holds L(i, q + k): the pivot (A::pivot, computed by every lane from the
// broadcast diagonal entry), the scaling of column q, its store, the rank-1
// update of the columns to its right (L(q + k, q) by shuffle from lane q + k),
// then a shift of c by one column.  Lanes compute every column and keep
// theirs by selects, so the independent updates interleave; the q loop stays
// rolled to keep its code small.  inv[k] = 1 / L_kk.
template <class A>
__device__ __noinline__ void warp_factor_diag(typename A::T *Ls, typename A::T *inv, int kb,
                                              int nb, int pk, int lane) {
  using E = typename A::T;
  E c[kNB];
  const bool in = lane < nb;
  const int ri = kb + (in ? lane : nb - 1);  // lanes >= nb shadow the last row
#pragma unroll
  for (int j = 0; j < kNB; ++j) c[j] = j < nb ? Ls[tri(ri) + kb + min(j, lane)] : E{};
  if (pk >= 0) {
    E xr[kNB];
#pragma unroll
    for (int p = 0; p < kNB; ++p) xr[p] = Ls[tri(ri) + pk + p];
#pragma unroll
    for (int j = 0; j < kNB; ++j) {
      if (j < nb) {
        const E *lj = Ls + tri(kb + j) + pk;
        typename A::Acc acc = A::begin(c[j]);
#pragma unroll
        for (int p = 0; p < kNB; ++p) A::sub(acc, xr[p], lj[p]);
        const E u = A::end(acc);
        c[j] = j <= lane ? u : c[j];
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kNB; ++j) c[j] = (in && j <= lane) ? c[j] : E{};
#pragma unroll 1
  for (int q = 0; q < nb; ++q) {
    E d, id;
    A::pivot(shfl_elt(c[0], q), d, id);
    const E sc = A::mul(c[0], id);
    c[0] = lane == q ? d : (lane > q ? sc : c[0]);
    if (lane == 0) inv[kb + q] = id;
    if (in && lane >= q) Ls[tri(kb + lane) + kb + q] = c[0];
#pragma unroll
    for (int k = 1; k < kNB; ++k) {
      const E l = shfl_elt(c[0], q + k);
      typename A::Acc acc = A::begin(c[k]);
      A::sub(acc, c[0], l);
      const E u = A::end(acc);
      c[k] = lane >= q + k ? u : c[k];
    }
#pragma unroll
    for (int k = 0; k + 1 < kNB; ++k) c[k] = c[k + 1];
    c[kNB - 1] = E{};
  }
  __syncwarp();
}

// Row i of the panel at kb (width nb): when pk >= 0 its entries first take
// the rank-8 update from the panel at pk, then L[i, kb:kb+nb] <- L[i, kb:kb+nb] L_bb^-T
// against the factored diagonal block.
template <class A>
__device__ __noinline__ void panel_row(typename A::T *Ls, const typename A::T *inv, int kb,
                                       int nb, int pk, int i) {
  using E = typename A::T;
  E *row = Ls + tri(i);
  typename A::Acc acc[kNB];
#pragma unroll
  for (int q = 0; q < kNB; ++q) acc[q] = A::begin(q < nb ? row[kb + q] : E{});
  if (pk >= 0) {
#pragma unroll
    for (int p = 0; p < kNB; ++p) {
      const E x = row[pk + p];
#pragma unroll
      for (int q = 0; q < kNB; ++q)
        if (q < nb) A::sub(acc[q], x, Ls[tri(kb + q) + pk + p]);
    }
  }
  E x[kNB];
#pragma unroll
  for (int q = 0; q < kNB; ++q) {
    if (q < nb) {
      const E *lq = Ls + tri(kb + q) + kb;
#pragma unroll
      for (int p = 0; p < q; ++p) A::sub(acc[q], x[p], lq[p]);
      x[q] = A::mul(A::end(acc[q]), inv[kb + q]);
    }
  }
#pragma unroll
  for (int q = 0; q < kNB; ++q)
    if (q < nb) row[kb + q] = x[q];
}

// Rank-nb update from the panel at kb of the entries (i, j), j0 <= j <= i < r
// and j < j1: the triangle below j0 when j1 >= r, or a column strip.
// Threads t0, t0 + T, ... share the entries evenly; each thread works on two
// entries at a time so that two independent FMA chains hide the FP64 latency.
struct StripPos {
  int ii, jj;
};

// Rows ii < w of the strip are the triangle's (length ii + 1), the rows below
// have length w: the walk crosses triangle rows one by one and the
// rectangular part by one division.
__device__ __forceinline__ void strip_advance(StripPos &p, int step, int w) {
  p.jj += step;
  while (p.ii < w) {
    if (p.jj <= p.ii) return;
    p.jj -= p.ii + 1;
    ++p.ii;
  }
  if (p.jj >= w) {
    p.ii += p.jj / w;
    p.jj %= w;
  }
}

__device__ __forceinline__ int strip_entries(int r, int j0, int j1) {
  const int n = r - j0, w = min(j1, r) - j0;
  return w * (w + 1) / 2 + (n - w) * w;
}

// Entries [e0, e1) of the enumeration (clipped to the strip).
template <class A>
__device__ __noinline__ void trailing_update(typename A::T *Ls, int r, int kb, int nb, int j0,
                                                int j1, int e0, int e1, int t0, int T) {
  using E = typename A::T;
  const int w = min(j1, r) - j0;  // strip width (w == n: whole triangle)
  e1 = min(e1, strip_entries(r, j0, j1));
  if (e0 + t0 >= e1) return;
  StripPos p;
  {
    const int tw = w * (w + 1) / 2, e = e0 + t0;
    if (e < tw) {
      tri_pos(e, p.ii, p.jj);
    } else {
      p.ii = w + (e - tw) / w;
      p.jj = (e - tw) % w;
    }
  }
  for (int e = e0 + t0; e < e1; e += 2 * T) {
    StripPos q = p;
    const bool two = e + T < e1;
    if (two) strip_advance(q, T, w);
    const int i1 = j0 + p.ii, c1 = j0 + p.jj;
    const int i2 = j0 + q.ii, c2 = j0 + q.jj;
    const E *li1 = Ls + tri(i1) + kb, *lj1 = Ls + tri(c1) + kb;
    const E *li2 = Ls + tri(i2) + kb, *lj2 = Ls + tri(c2) + kb;
    E *a1 = Ls + tri(i1) + c1;
    E *a2 = Ls + tri(i2) + c2;
    // without a second entry q == p: the second chain recomputes the first
    // entry from valid addresses and is not stored (no selects in the loop)
    typename A::Acc acc1 = A::begin(*a1), acc2 = A::begin(*a2);
    if (nb == kNB) {
      E x1[kNB], y1[kNB], x2[kNB], y2[kNB];
#pragma unroll
      for (int k = 0; k < kNB; ++k) {
        x1[k] = li1[k];
        y1[k] = lj1[k];
        x2[k] = li2[k];
        y2[k] = lj2[k];
      }
#pragma unroll
      for (int k = 0; k < kNB; ++k) {
        A::sub(acc1, x1[k], y1[k]);
        A::sub(acc2, x2[k], y2[k]);
      }
    } else {
      for (int k = 0; k < nb; ++k) A::sub(acc1, li1[k], lj1[k]);
      if (two)
        for (int k = 0; k < nb; ++k) A::sub(acc2, li2[k], lj2[k]);
    }
    *a1 = A::end(acc1);
    if (two) *a2 = A::end(acc2);
    p = q;
    strip_advance(p, two ? T : 0, w);
  }
}

// In-place right-looking Cholesky of the packed matrix in 8-column panels.
// After the first panel, step kb (the panel at kb final) factors the next
// panel nk = kb + 8 in two phases separated by CTA barriers:
//   (A) all threads: panel nk's columns take panel kb's rank-8 update;
//   (B) warp 0 factors the diagonal block of nk and raises a flag; all warps
//       take work from shared counters: once the flag is up, rows of panel
//       nk (one per lane, solved against the block), otherwise chunks of
//       kChunk entries of the trailing triangle right of nk (panel kb's
//       update); a warp with nothing left but rows waits for the flag
//       (bounded: on timeout bit 8 of `err` is raised).
// The counters and the flag alternate between two sets by step parity, so
// that the set of the next step is cleared while this one is in use.  Per
// element this is the same sequence of fused multiply-adds as the
// column-at-a-time algorithm.  A non-positive pivot produces NaN, which the
// caller turns into a reject.
constexpr int kChunk = 128;                // trailing-update entries per warp grab
constexpr uint32_t kFlagSpins = 1u << 22;  // polls of the diagonal-block flag

// `ctr` is six ints of shared memory.
template <class A>
__device__ void cta_cholesky(typename A::T *Ls, typename A::T *inv, int r, int *ctr, int *err) {
  const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < 6) ctr[tid] = 0;
  if (warp == 0) warp_factor_diag<A>(Ls, inv, 0, min(kNB, r), -1, lane);
  __syncthreads();
  for (int i = min(kNB, r) + tid; i < r; i += T) panel_row<A>(Ls, inv, 0, min(kNB, r), -1, i);
  __syncthreads();
  int step = 0;
  for (int kb = 0; kb + kNB < r; kb += kNB, ++step) {
    const int nk = kb + kNB, nb2 = min(kNB, r - nk), j0 = nk + nb2;
    const int rows = r - j0, full = rows > 0 ? strip_entries(r, j0, r) : 0;
    int *c3 = ctr + 3 * (step & 1);
    trailing_update<A>(Ls, r, kb, kNB, nk, j0, 0, 1 << 30, tid, T);  // (A)
    if (tid == 0) {
      int *o = ctr + 3 * ((step + 1) & 1);
      o[0] = o[1] = o[2] = 0;
    }
    __syncthreads();
    if (warp == 0) {  // (B)
      warp_factor_diag<A>(Ls, inv, nk, nb2, -1, lane);
      __threadfence_block();
      if (lane == 0) atomicExch(&c3[2], 1);
    }
    uint32_t spins = 0;
    for (;;) {
      int job = 0, base = 0;  // 0 done, 1 rows, 2 trailing chunk, 3 wait
      if (lane == 0) {
        const bool ready = atomicAdd(&c3[2], 0) != 0;
        if (ready && rows > 0) {
          base = atomicAdd(&c3[1], 32);
          if (base < rows) job = 1;
        }
        if (job == 0) {
          base = atomicAdd(&c3[0], 1) * kChunk;
          if (base < full) job = 2;
        }
        if (job == 0 && !ready && rows > 0) job = 3;
      }
      job = __shfl_sync(kFull, job, 0);
      base = __shfl_sync(kFull, base, 0);
      if (job == 0) break;
      if (job == 1) {
        __syncwarp();
        __threadfence_block();
        if (base + lane < rows) panel_row<A>(Ls, inv, nk, nb2, -1, j0 + base + lane);
      } else if (job == 2) {
        trailing_update<A>(Ls, r, kb, kNB, j0, r, base, base + kChunk, lane, 32);
      } else {
        if (++spins > kFlagSpins) {
          if (lane == 0) atomicOr(err, 8);
          break;
        }
        __nanosleep(32);
      }
    }
    __syncthreads();
  }
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
    normals4_f64(philox_block(a.seed, STREAM_XI, a.step, chain, blk), n4);
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
  const double *L = a.L + (size_t)a.cur[c] * a.L_slot + (size_t)c * slot_stride(r);
  const double *tv = L + tri(r), *pv = L + tri(r + 1);
  const uint32_t chain = (uint32_t)(a.id_base + (uint64_t)c);
  for (int blk = lane; blk < (r + 3) / 4; blk += 32) {
    double n4[4];
    normals4_f64(philox_block(a.seed, STREAM_XI, a.step, chain, blk), n4);
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

// The same from an FP32 J into double-float entries: each thread
// accumulates up to kHMaxTiles 4 x 4 tiles of J^T J in FP32 registers over
// all d_y rows (chunks of kJChunkF rows staged in shared memory, padded to a
// multiple of 4 columns), then writes I + H once, the product with
// 1 / noise_var taken exactly as a double-float.  Large r takes several
// rounds of tiles.
__device__ void form_h_f32(const float *J, int dy, int r, double inv_nv, float2 *Ls,
                           float *Jc) {
  const int nt = (r + kHT - 1) / kHT, rp = nt * kHT;
  const int ntiles = nt * (nt + 1) / 2;
  if (dy == 0) {
    for (int e = threadIdx.x; e < tri(r); e += blockDim.x) Ls[e] = make_float2(0.0f, 0.0f);
    __syncthreads();
    for (int i = threadIdx.x; i < r; i += blockDim.x) Ls[tri(i) + i] = make_float2(1.0f, 0.0f);
    __syncthreads();
    return;
  }
  const float nh = __double2float_rn(inv_nv), nl = __double2float_rn(inv_nv - (double)nh);
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
          if (i < r && j <= i) {
            const float x = acc[s][p][q], ph = __fmul_rn(x, nh);
            float e = __fmaf_rn(x, nh, -ph);
            e = __fmaf_rn(x, nl, e);
            float h, l;
            fast_two_sum(ph, e, h, l);
            if (i == j) {
              float s1, q1;
              two_sum(1.0f, h, s1, q1);
              fast_two_sum(s1, __fadd_rn(q1, l), h, l);
            }
            Ls[tri(i) + j] = make_float2(h, l);
          }
        }
    }
  }
  __syncthreads();
}

// The accept test log u <= min(0, log rho) (Algorithm 1; NaN rejects), the
// counters, and the scalar state of an accepted chain.  Thread 0 only.
__device__ bool accept_test(const ReducedArgs &a, int c, double lr, double phi_b, double hld_b) {
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
    a.phi[c] = phi_b;
    a.hld[c] = hld_b;
    a.cur[c] ^= 1;
  }
  if (!finite) atomicAdd(&a.counters[1], 1ull);
  atomicAdd(a.sum_alpha, finite ? exp(fmin(0.0, lr)) : 0.0);
  return accept;
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
template <typename TJ, bool G>
__global__ void __launch_bounds__(kThreads) k_geometry(ReducedArgs a, int mode) {
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
    form_h_f32(reinterpret_cast<const float *>(J), dy, r, inv_nv, reinterpret_cast<float2 *>(Ls),
               reinterpret_cast<float *>(sm + lay.tail));
  } else {
    double *Ld = reinterpret_cast<double *>(Ls);
    form_h_f64(reinterpret_cast<const double *>(J), dy, r, inv_nv, Ld, sm + lay.tail);
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
  cta_cholesky<A>(Ls, inv, r + 1, reinterpret_cast<int *>(red + 100), a.err);
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
      a.mr[(size_t)c * r + i] = vb[i];
      a.g[(size_t)c * r + i] = vg[i];
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

template <typename TJ, bool G>
static cudaError_t launch_geometry_t(const ReducedArgs &a, int mode, size_t smem,
                                     cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_geometry<TJ, G>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_geometry<TJ, G><<<a.C, kThreads, smem, st>>>(a, mode);
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
