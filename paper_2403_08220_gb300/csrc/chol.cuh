// Device code shared by the per-chain reduced-space kernels: reductions,
// the element arithmetic (native FP64 or double-float pairs on the FP32
// pipe), the blocked packed Cholesky factorisation, triangular solves, the
// Gram-matrix products from an FP32 or FP64 Jacobian, and the accept test.
// Included by one translation unit per kernel family; every definition has
// internal linkage.
#pragma once
#include <type_traits>

#include "dino_internal.h"
#include "philox.cuh"

namespace dino {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kJChunk = 16;    // rows of an FP64 matrix staged per pass when forming a Gram matrix
constexpr int kJChunkF = 32;   // rows of an FP32 matrix staged per pass
constexpr int kNB = 8;         // Cholesky panel width
constexpr int kHT = 4;         // FP32 register tile edge of the Gram products
constexpr int kHMaxTiles = 3;  // tiles per thread: ceil(52*53/2 / 512) for n <= 208
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
  __device__ static T add(T a, T b) { return a + b; }
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
  __device__ static T add(T a, T b) {
    float s, e;
    two_sum(a.x, b.x, s, e);
    float h, l;
    fast_two_sum(s, __fadd_rn(e, __fadd_rn(a.y, b.y)), h, l);
    return make_float2(h, l);
  }
  __device__ static T neg(T a) { return make_float2(-a.x, -a.y); }
  // The same pivot on the FP32 pipe: the Newton step y <- y + y (1 - x y^2) / 2
  // takes the residual 1 - x y^2 exactly (double-float product, two-sum
  // against 1) and the small correction in FP32, so from an estimate with
  // relative error e it reaches about 1.5 e^2.  x <= 0 gives NaN, as in FP64.
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
    // FP32 estimate, one FP32 Newton step (relative error ~2^-23), then one
    // double-float step (~2^-45)
    float y0 = rsqrtf(x.x);
    y0 = y0 * (1.5f - 0.5f * x.x * y0 * y0);
    T y = make_float2(y0, 0.0f);
    newton_rsqrt(x, y);
    id = y;
    d = mul(x, y);
  }
};

// Lane-to-lane copies of a factor element.
__device__ __forceinline__ double shfl_elt(double x, int src) {
  return __shfl_sync(kFull, x, src);
}
__device__ __forceinline__ float2 shfl_elt(float2 x, int src) {
  return make_float2(__shfl_sync(kFull, x.x, src), __shfl_sync(kFull, x.y, src));
}
__device__ __forceinline__ double shfl_xor_elt(double x, int m) {
  return __shfl_xor_sync(kFull, x, m);
}
__device__ __forceinline__ float2 shfl_xor_elt(float2 x, int m) {
  return make_float2(__shfl_xor_sync(kFull, x.x, m), __shfl_xor_sync(kFull, x.y, m));
}

// Warp sum of a factor element (every lane gets it).
template <class A>
__device__ __forceinline__ typename A::T warp_sum_elt(typename A::T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = A::add(v, shfl_xor_elt(v, o));
  return v;
}

// x <- L^-1 x over the leading n rows of a packed lower factor (x in shared
// memory): 32-row diagonal blocks are solved by warp 0 with shuffles (every
// lane computes, selects keep its own), the rows below each block are
// updated by the whole CTA.
template <class A>
__device__ void cta_lower_solve_t(const typename A::T *Ls, const typename A::T *inv, int n,
                                  typename A::T *x) {
  using E = typename A::T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int jb = 0; jb < n; jb += 32) {
    const int nb = min(32, n - jb);
    if (warp == 0) {
      E xl = lane < nb ? x[jb + lane] : E{};
      const int row = jb + min(lane, nb - 1);
      for (int k = 0; k < nb; ++k) {
        const E yk = A::mul(shfl_elt(xl, k), inv[jb + k]);
        const E l = Ls[tri(row) + jb + min(k, row - jb)];
        typename A::Acc acc = A::begin(xl);
        A::sub(acc, l, yk);
        const E u = A::end(acc);
        xl = lane == k ? yk : ((lane > k && lane < nb) ? u : xl);
      }
      if (lane < nb) x[jb + lane] = xl;
    }
    __syncthreads();
    for (int i = jb + nb + threadIdx.x; i < n; i += blockDim.x) {
      const E *row = Ls + tri(i) + jb;
      typename A::Acc acc = A::begin(x[i]);
      for (int k = 0; k < nb; ++k) A::sub(acc, row[k], x[jb + k]);
      x[i] = A::end(acc);
    }
    __syncthreads();
  }
}

// x <- L^-T x (back substitution on the upper factor L^T), same scheme.
template <class A>
__device__ void cta_upper_solve_t(const typename A::T *Ls, const typename A::T *inv, int n,
                                  typename A::T *x) {
  using E = typename A::T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int jb = ((n - 1) / 32) * 32; jb >= 0; jb -= 32) {
    const int nb = min(32, n - jb);
    if (warp == 0) {
      E xl = lane < nb ? x[jb + lane] : E{};
      const int col = jb + min(lane, nb - 1);
      for (int k = nb - 1; k >= 0; --k) {
        const E yk = A::mul(shfl_elt(xl, k), inv[jb + k]);
        const E l = Ls[tri(jb + k) + min(col, jb + k)];
        typename A::Acc acc = A::begin(xl);
        A::sub(acc, l, yk);
        const E u = A::end(acc);
        xl = lane == k ? yk : (lane < k ? u : xl);
      }
      if (lane < nb) x[jb + lane] = xl;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < jb; i += blockDim.x) {
      typename A::Acc acc = A::begin(x[i]);
      for (int k = 0; k < nb; ++k) A::sub(acc, Ls[tri(jb + k) + i], x[jb + k]);
      x[i] = A::end(acc);
    }
    __syncthreads();
  }
}

// Position (ii, jj) of packed index e in a lower triangle.
__device__ __forceinline__ void tri_pos(int e, int &ii, int &jj) {
  ii = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while (tri(ii + 1) <= e) ++ii;
  while (tri(ii) > e) --ii;
  jj = e - tri(ii);
}


// Factor the 8 x 8 diagonal block at kb (size nb) by one warp, in registers.
// Every lane holds the whole lower block and factors it (column q: the pivot
// A::pivot, the scaling of column q, the rank-1 update of the columns to its
// right), so no value crosses lanes and the dependent chain per column is
// only pivot -> scale -> next diagonal update; the off-diagonal updates of
// the unrolled loop overlap it.  Rows and columns >= nb are padded with the
// identity, which leaves the rows < nb unchanged and is never stored.  The
// arithmetic per entry is the column-at-a-time sequence.  After a warp
// barrier (the block is read by all lanes and overwritten in place) lanes
// share the stores: entry e of the block by lane e mod 32, inv[k] = 1 / L_kk.
template <class A>
__device__ __noinline__ void warp_factor_diag(typename A::T *Ls, typename A::T *inv, int kb,
                                              int nb, int lane) {
  using E = typename A::T;
  E c[kNB][kNB];
#pragma unroll
  for (int i = 0; i < kNB; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j)
      c[i][j] = i < nb ? Ls[tri(kb + i) + kb + j] : (i == j ? A::from_j(1.0f) : E{});
#pragma unroll
  for (int q = 0; q < kNB; ++q) {
    E d, id;
    A::pivot(c[q][q], d, id);
    c[q][q] = d;
    if (lane == 0 && q < nb) inv[kb + q] = id;
#pragma unroll
    for (int i = q + 1; i < kNB; ++i) c[i][q] = A::mul(c[i][q], id);
#pragma unroll
    for (int k = q + 1; k < kNB; ++k)
#pragma unroll
      for (int i = k; i < kNB; ++i) {
        typename A::Acc acc = A::begin(c[i][k]);
        A::sub(acc, c[i][q], c[k][q]);
        c[i][k] = A::end(acc);
      }
  }
  __syncwarp();  // every lane's loads of the block precede any lane's stores
#pragma unroll
  for (int i = 0; i < kNB; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j)
      if (lane == (tri(i) + j) % 32 && i < nb) Ls[tri(kb + i) + kb + j] = c[i][j];
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
    if (w == kNB) {  // a full panel strip: shifts instead of a runtime division
      static_assert(kNB == 8, "strip width is a power of two");
      p.ii += p.jj >> 3;
      p.jj &= kNB - 1;
    } else {
      p.ii += p.jj / w;
      p.jj %= w;
    }
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

// `ctr` is six ints of shared memory; a warp gives up waiting for the flag
// after `max_spins` polls.
template <class A>
__device__ void cta_cholesky(typename A::T *Ls, typename A::T *inv, int r, int *ctr, int *err,
                             uint32_t max_spins) {
  const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < 6) ctr[tid] = 0;
  if (warp == 0) warp_factor_diag<A>(Ls, inv, 0, min(kNB, r), lane);
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
      warp_factor_diag<A>(Ls, inv, nk, nb2, lane);
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
        if (++spins > max_spins) {
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

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}


// Gram products.  X(k, i), k < m (reduction), i < n: element X[k * ldx + i]
// (kRedContig = false: X^T X of a row-major m x n matrix, the r-sized path's
// J^T J) or X[i * ldx + k] (kRedContig = true: the Gram matrix X X^T of a
// row-major n x m matrix, the Woodbury path's J J^T).  Staging reads run along
// the contiguous index.  Out: I + (sum_k X(k, i) X(k, j)) / noise_var into the
// packed lower matrix Ls (i, j < n).

// From an FP64 X: chunks of kJChunk reduction rows, FP64 products
// accumulated in shared memory.
template <bool kRedContig>
__device__ void form_gram_f64(const double *X, int m, int n, int ldx, double inv_nv, double *Ls,
                              double *Jc) {
  const int lsz = tri(n);
  for (int i0 = 0; i0 < m; i0 += kJChunk) {
    const int nr = min(kJChunk, m - i0);
    // unrolled so that each thread has several independent loads in flight
    if (kRedContig) {
#pragma unroll 8
      for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
        const int i = e / nr, k = e % nr;
        Jc[k * n + i] = X[(size_t)i * ldx + i0 + k];
      }
    } else {
#pragma unroll 8
      for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
        const int k = e / n, i = e % n;
        Jc[e] = X[(size_t)(i0 + k) * ldx + i];
      }
    }
    __syncthreads();
    if ((int)threadIdx.x < lsz) {
      int ii, jj;
      tri_pos(threadIdx.x, ii, jj);
      for (int e = threadIdx.x; e < lsz; e += blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < nr; ++k) acc += Jc[k * n + ii] * Jc[k * n + jj];
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

// From an FP32 X into double-float entries: each thread accumulates up to
// kHMaxTiles 4 x 4 tiles in FP32 registers (chunks of kJChunkF reduction rows
// staged in shared memory, padded to a multiple of 4 columns); every
// kGramFlush rows the FP32 tile sums are added exactly into double-float sums
// held in Ls (each entry owned by one thread) and restart from zero, so the
// FP32 rounding error grows with kGramFlush rather than with m.  At the end
// each entry is multiplied by 1 / noise_var as a double-float and 1 is added
// on the diagonal.  Large n takes several rounds of tiles.
constexpr int kGramFlush = 2 * kJChunkF;

template <bool kRedContig>
__device__ void form_gram_f32(const float *X, int m, int n, int ldx, double inv_nv, float2 *Ls,
                              float *Jc) {
  const int r = n, dy = m;
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
    bool first = true;
    for (int i0 = 0; i0 < dy; i0 += kJChunkF) {
      const int nr = min(kJChunkF, dy - i0);
      // unrolled so that each thread has several independent loads in flight
      if (kRedContig) {
#pragma unroll 8
        for (int e = threadIdx.x; e < nr * rp; e += blockDim.x) {
          const int j = e / nr, k = e % nr;
          Jc[k * rp + j] = j < r ? X[(size_t)j * ldx + i0 + k] : 0.0f;
        }
      } else {
#pragma unroll 8
        for (int e = threadIdx.x; e < nr * rp; e += blockDim.x) {
          const int k = e / rp, j = e % rp;
          Jc[e] = j < r ? X[(size_t)(i0 + k) * ldx + j] : 0.0f;
        }
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
      if ((i0 + nr) % kGramFlush == 0 || i0 + nr >= dy) {
#pragma unroll
        for (int s = 0; s < kHMaxTiles; ++s) {
          if (ti[s] < 0) continue;
#pragma unroll
          for (int p = 0; p < kHT; ++p)
#pragma unroll
            for (int q = 0; q < kHT; ++q) {
              const int i = kHT * ti[s] + p, j = kHT * tj[s] + q;
              if (i < r && j <= i) {
                float2 *e = Ls + tri(i) + j;
                const float2 x = make_float2(acc[s][p][q], 0.0f);
                *e = first ? x : DF::add(*e, x);
              }
              acc[s][p][q] = 0.0f;
            }
        }
        first = false;
      }
    }
    // scale by 1 / noise_var and add the identity (the entries this thread owns)
#pragma unroll
    for (int s = 0; s < kHMaxTiles; ++s) {
      if (ti[s] < 0) continue;
#pragma unroll
      for (int p = 0; p < kHT; ++p)
#pragma unroll
        for (int q = 0; q < kHT; ++q) {
          const int i = kHT * ti[s] + p, j = kHT * tj[s] + q;
          if (i < r && j <= i) {
            float2 v = DF::mul(Ls[tri(i) + j], make_float2(nh, nl));
            if (i == j) v = DF::add(make_float2(1.0f, 0.0f), v);
            Ls[tri(i) + j] = v;
          }
        }
    }
  }
  __syncthreads();
}

// The accept test log u <= min(0, log rho) (Algorithm 1; NaN rejects), the
// counters ([0] accepts, [1] non-finite rejects, [2] first-stage accepts),
// and the scalar state of an accepted chain, or with delayed acceptance its
// staging for the second stage.  Thread 0 only.
__device__ bool accept_test(const ReducedArgs &a, int c, double lr, double phi_b, double hld_b) {
  const uint32_t chain = (uint32_t)(a.id_base + (uint64_t)c);
  const double log_u =
      a.ext_log_u ? a.ext_log_u[c]
                  : log(word_to_uniform(philox_block(a.seed, STREAM_U, a.step, chain, 0).x));
  const bool finite = isfinite(lr);
  const bool accept = finite && log_u <= fmin(0.0, lr);
  a.log_rho[c] = lr;
  a.log_u[c] = log_u;
  a.acc[c] = accept ? 1 : 0;
  if (accept) {
    atomicAdd(&a.counters[2], 1ull);  // first-stage accepts
    if (a.da) {  // delayed acceptance: staged for the second stage
      a.phi_st[c] = phi_b;
      a.hld_st[c] = hld_b;
    } else {
      a.acc_count[c] += 1;
      atomicAdd(&a.counters[0], 1ull);
      a.phi[c] = phi_b;
      a.hld[c] = hld_b;
      a.cur[c] ^= 1;
    }
  }
  if (!finite) atomicAdd(&a.counters[1], 1ull);
  atomicAdd(a.sum_alpha, finite ? exp(fmin(0.0, lr)) : 0.0);
  return accept;
}

}  // namespace
}  // namespace dino
