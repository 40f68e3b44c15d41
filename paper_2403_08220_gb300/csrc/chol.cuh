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
constexpr int kRed = 104;      // reduction scratch (doubles): block_sum3 uses [0, 99)

__device__ __forceinline__ int tri(int i) { return i * (i + 1) / 2; }

// Asynchronous copies global -> shared (cp.async, 16 or 4 bytes; bytes
// beyond src_bytes are zero-filled), their commit groups and waits on the
// thread's own groups.
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// 16-byte asynchronous copy global -> shared; bytes beyond `src_bytes` (0..16)
// are zero-filled.  Both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
               "r"(src_bytes)
               : "memory");
}
// 4-byte variant (src_bytes 0 or 4).
__device__ __forceinline__ void cp_async4(void *dst, const void *src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(dst)), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
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
  // the same for an FP32 x (a pair whose low part is 0: that term vanishes)
  __device__ static void sub_f(Acc &a, float x, T y) {
    const float p = __fmul_rn(x, y.x);
    float e = __fmaf_rn(x, y.x, -p);
    e = __fmaf_rn(x, y.y, e);
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
  // The same pivot on the FP32 pipe: an FP32 estimate y of x^(-1/2), one
  // FP32 Newton step (relative error ~2^-24), then one Newton step
  // y <- y + y (1 - x y^2) / 2 whose residual is formed from exact pieces:
  // y^2 = p + e and x.h p = hp + herr exactly, 1 - hp is exact (hp is within
  // a factor 2 of 1), so r = 1 - x y^2 is accurate to ~2^-47 absolute and
  // from an estimate with relative error e the step reaches about 1.5 e^2
  // (~2^-45 from e ~ 2^-23).  The correction y r / 2 needs only FP32
  // precision.  x <= 0 gives NaN, as in FP64.
  __device__ static void pivot(T x, T &d, T &id) {
    float y = rsqrtf(x.x);
    y = y * (1.5f - 0.5f * x.x * y * y);
    const float p = __fmul_rn(y, y);
    const float e = __fmaf_rn(y, y, -p);
    const float hp = __fmul_rn(x.x, p);
    const float herr = __fmaf_rn(x.x, p, -hp);
    float r = __fsub_rn(__fsub_rn(1.0f, hp), herr);
    r = __fmaf_rn(-x.x, e, r);
    r = __fmaf_rn(-x.y, p, r);
    const float c = __fmul_rn(__fmul_rn(0.5f, y), r);
    fast_two_sum(y, c, id.x, id.y);
    d = mul(x, id);
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
// memory): 32-row diagonal blocks are solved by warp 0 with shuffles, the
// rows below each block are updated by the whole CTA.  In a block, lane i
// carries its running value scaled by 1 / L_ii, so that step k of the
// dependent chain is one broadcast and one multiply-subtract with
// L_ik / L_ii (formed off the chain): y_k is lane k's value as it stands.
template <class A>
__device__ void cta_lower_solve_t(const typename A::T *Ls, const typename A::T *inv, int n,
                                  typename A::T *x) {
  using E = typename A::T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int jb = 0; jb < n; jb += 32) {
    const int nb = min(32, n - jb);
    if (warp == 0) {
      const int row = jb + min(lane, nb - 1);
      const E il = inv[row];
      E xl = lane < nb ? A::mul(x[jb + lane], il) : E{};
      for (int k = 0; k < nb; ++k) {
        const E yk = shfl_elt(xl, k);
        const E l = A::mul(Ls[tri(row) + jb + min(k, row - jb)], il);
        typename A::Acc acc = A::begin(xl);
        A::sub(acc, l, yk);
        const E u = A::end(acc);
        xl = (lane > k && lane < nb) ? u : xl;
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

// x <- L^-T x (back substitution on the upper factor L^T), same scheme
// (lane i scaled by 1 / L_ii, coefficients L_ki / L_ii).
template <class A>
__device__ void cta_upper_solve_t(const typename A::T *Ls, const typename A::T *inv, int n,
                                  typename A::T *x) {
  using E = typename A::T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int jb = ((n - 1) / 32) * 32; jb >= 0; jb -= 32) {
    const int nb = min(32, n - jb);
    if (warp == 0) {
      const int col = jb + min(lane, nb - 1);
      const E il = inv[col];
      E xl = lane < nb ? A::mul(x[jb + lane], il) : E{};
      for (int k = nb - 1; k >= 0; --k) {
        const E yk = shfl_elt(xl, k);
        const E l = A::mul(Ls[tri(jb + k) + min(col, jb + k)], il);
        typename A::Acc acc = A::begin(xl);
        A::sub(acc, l, yk);
        const E u = A::end(acc);
        xl = lane < k ? u : xl;
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
// Lane 4 i + s holds the entries (i, s) and (i, s + 4) of the lower block;
// rows and columns >= nb are padded with the identity, which leaves the rows
// < nb unchanged and is never stored.  Column q: every lane takes the pivot
// A::pivot of the broadcast diagonal entry, the owners of column q scale it,
// and each entry (i, k), q < k <= i, takes the rank-1 update with the scaled
// values of rows i and k fetched by shuffles.  The arithmetic per entry is the
// column-at-a-time sequence; inv[k] = 1 / L_kk, and lsc (packed, 8 x 8)
// receives the strictly lower block scaled by row, L_ij / L_ii.
template <class A>
__device__ __noinline__ void warp_factor_diag(typename A::T *Ls, typename A::T *inv, int kb,
                                              int nb, int lane, typename A::T *lsc) {
  using E = typename A::T;
  const int i = lane >> 2, s = lane & 3;
  const E one = A::from_j(1.0f);
  E c0 = E{}, c1 = E{};  // (i, s) and (i, s + 4)
  E id_i = one;          // 1 / L_ii of this lane's row
  if (s <= i) c0 = i < nb ? Ls[tri(kb + i) + kb + s] : (i == s ? one : E{});
  if (s + 4 <= i) c1 = i < nb ? Ls[tri(kb + i) + kb + s + 4] : (i == s + 4 ? one : E{});
#pragma unroll
  for (int q = 0; q < kNB; ++q) {
    const int sq = q & 3;
    E &own = q < 4 ? c0 : c1;  // this lane's entry in column q, if any
    E d, id;
    A::pivot(shfl_elt(own, 4 * q + sq), d, id);
    if (lane == 0 && q < nb) inv[kb + q] = id;
    if (i == q) id_i = id;
    if (s == sq && i > q) own = A::mul(own, id);
    if (s == sq && i == q) own = d;
    if (q == kNB - 1) break;  // nothing right of the last column
    const E ciq = shfl_elt(own, 4 * i + sq);  // L_iq
    if (q < 3) {                              // entries (i, s) with s > q exist
      const E csq = shfl_elt(own, 4 * s + sq);  // L_sq
      if (s > q && s <= i) {
        typename A::Acc acc = A::begin(c0);
        A::sub(acc, ciq, csq);
        c0 = A::end(acc);
      }
    }
    const E cs4q = shfl_elt(own, 4 * (s + 4) + sq);  // L_{s+4,q}
    if (s + 4 > q && s + 4 <= i) {
      typename A::Acc acc = A::begin(c1);
      A::sub(acc, ciq, cs4q);
      c1 = A::end(acc);
    }
  }
  if (i < nb && s <= i) Ls[tri(kb + i) + kb + s] = c0;
  if (i < nb && s + 4 <= i) Ls[tri(kb + i) + kb + s + 4] = c1;
  // the rows of the block scaled by their inverse pivots, L_ij / L_ii (j < i),
  // for the row solves
  if (s < i) lsc[tri(i) + s] = A::mul(c0, id_i);
  if (s + 4 < i) lsc[tri(i) + s + 4] = A::mul(c1, id_i);
  __syncwarp();
}

// Row i of the panel at kb (width nb): L[i, kb:kb+nb] <- L[i, kb:kb+nb] L_bb^-T,
// by forward substitution with the row-scaled block lsc (L_qp / L_qq):
// x_q = b_q / L_qq - sum_{p<q} x_p (L_qp / L_qq), so that each step of the
// dependent chain is one multiply-subtract.
template <class A>
__device__ __noinline__ void panel_row(typename A::T *Ls, const typename A::T *inv,
                                       const typename A::T *lsc, int kb, int nb, int i) {
  using E = typename A::T;
  E *row = Ls + tri(i);
  E x[kNB];
#pragma unroll
  for (int q = 0; q < kNB; ++q)
    if (q < nb) x[q] = A::mul(row[kb + q], inv[kb + q]);
#pragma unroll
  for (int q = 1; q < kNB; ++q) {
    if (q < nb) {
      typename A::Acc acc = A::begin(x[q]);
#pragma unroll
      for (int p = 0; p < q; ++p) A::sub(acc, x[p], lsc[tri(q) + p]);
      x[q] = A::end(acc);
    }
  }
#pragma unroll
  for (int q = 0; q < kNB; ++q)
    if (q < nb) row[kb + q] = x[q];
}

// Trailing update of a right-looking Cholesky step: every entry (i, j) with
// c0 <= j <= i < n takes the rank-8 update from the factored panel at kb,
// A_ij -= sum_{k < 8} L_{i,kb+k} L_{j,kb+k}.  The columns are cut into blocks
// of 32; per block the work items, which warps take from the shared counter
// *next (one atomic per item), are
//   the block's diagonal triangle (rows and columns in the block) in three
//   items, its 8 x 8 corner and two halves of the rest, entries enumerated in
//   packed order, one entry per lane at a time with both panel rows read
//   from shared memory;
//   chunks of kColRows rows below the triangle, where each lane owns one
//   column j (its panel values L_{j,kb..} in registers) and the rows are read
//   as warp-wide broadcasts, two rows at a time so that every lane runs two
//   independent accumulations; every lane has work in every row.
// Every entry is written by one lane and only panel columns are read, so the
// items need no synchronisation.  The first item (the corner of the first
// block) is the 8 x 8 diagonal block of the next panel at c0; with
// `factor_next` the warp that takes it factors that block right after, a
// short serial path that the other warps' items overlap.
constexpr int kColRows = 16;

template <class A>
__device__ void trailing_cols(typename A::T *Ls, typename A::T *inv, typename A::T *lsc, int n,
                              int kb, int c0, int *next, bool factor_next) {
  using E = typename A::T;
  const int lane = threadIdx.x & 31;
  const int nblk = (n - c0 + 31) / 32;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(next, 1);
    item = __shfl_sync(kFull, item, 0);
    int b = 0, jb = c0, q = item;
    for (; b < nblk; ++b, jb += 32) {
      const int chunks = 3 + (max(0, n - jb - 32) + kColRows - 1) / kColRows;
      if (q < chunks) break;
      q -= chunks;
    }
    if (b == nblk) return;
    if (q < 3) {  // the diagonal triangle: its 8 x 8 corner, then two halves of the rest
      const int m = min(32, n - jb), ne = m * (m + 1) / 2, nc = min(ne, tri(kNB));
      const int half = (ne - nc + 1) / 2;
      const int e0 = q == 0 ? 0 : nc + (q - 1) * half;
      const int e1 = q == 0 ? nc : min(ne, nc + q * half);
      for (int e = e0 + lane; e < e1; e += 32) {
        int ii, jj;
        tri_pos(e, ii, jj);
        const E *x = Ls + tri(jb + ii) + kb, *y = Ls + tri(jb + jj) + kb;
        E *p = Ls + tri(jb + ii) + jb + jj;
        typename A::Acc acc = A::begin(*p);
#pragma unroll
        for (int k = 0; k < kNB; ++k) A::sub(acc, x[k], y[k]);
        *p = A::end(acc);
      }
      if (factor_next && item == 0) {  // the next panel's diagonal block is final
        __syncwarp();
        warp_factor_diag<A>(Ls, inv, c0, min(kNB, n - c0), lane, lsc);
      }
      continue;
    }
    const int j = jb + lane;  // < jb + 32 <= every row of the chunk
    E yj[kNB];
#pragma unroll
    for (int k = 0; k < kNB; ++k) yj[k] = Ls[tri(j) + kb + k];
    const int i0 = jb + 32 + (q - 3) * kColRows, i1 = min(n, i0 + kColRows);
    for (int i = i0; i < i1; i += 2) {
      const bool two = i + 1 < i1;
      const int ib = two ? i + 1 : i;
      const E *xa = Ls + tri(i) + kb;
      const E *xb = Ls + tri(ib) + kb;
      E *pa = Ls + tri(i) + j;
      E *pb = Ls + tri(ib) + j;
      typename A::Acc acc1 = A::begin(*pa), acc2 = A::begin(*pb);
#pragma unroll
      for (int k = 0; k < kNB; ++k) {
        A::sub(acc1, xa[k], yj[k]);
        A::sub(acc2, xb[k], yj[k]);
      }
      *pa = A::end(acc1);
      if (two) *pb = A::end(acc2);
    }
  }
}

// In-place right-looking Cholesky of the packed n x n matrix in 8-column
// panels.  The first diagonal block is factored by one warp (in registers);
// then per panel kb, with a CTA barrier after each phase:
//   every thread takes rows below the factored diagonal block and solves
//   them against it;
//   the warps apply the panel's rank-8 update to the columns right of it
//   (work items from a shared counter), and the warp that updates the next
//   panel's diagonal block factors it as soon as it is final, while the
//   others carry on with the update.
// Row assignment rotates with the panel and the CTA, so that the CTAs
// resident on an SM load its schedulers evenly.  Per element this is the
// column-at-a-time sequence of fused multiply-adds.  A non-positive pivot
// produces NaN, which the caller turns into a reject.  No thread waits on
// another beyond the barriers.
template <class A>
__device__ void cta_cholesky_panels(typename A::T *Ls, typename A::T *inv, int n) {
  __shared__ int next_item;
  __shared__ typename A::T lsc[kNB * (kNB + 1) / 2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (warp == blockIdx.x % nw) warp_factor_diag<A>(Ls, inv, 0, min(kNB, n), lane, lsc);
  __syncthreads();
  for (int kb = 0; kb < n; kb += kNB) {
    const int nb = min(kNB, n - kb), j1 = kb + nb;
    const int rot = (kb / kNB + blockIdx.x) % nw;
    if (threadIdx.x == 0) next_item = 0;
    const int t = (threadIdx.x + 32 * rot) % blockDim.x;
    for (int i = j1 + t; i < n; i += blockDim.x) panel_row<A>(Ls, inv, lsc, kb, nb, i);
    __syncthreads();
    if (j1 < n) {
      trailing_cols<A>(Ls, inv, lsc, n, kb, j1, &next_item, true);
      __syncthreads();
    }
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
  const bool vec16 = !kRedContig && (ldx & 3) == 0 && ((uintptr_t)X & 15) == 0;
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
      } else if (vec16) {  // 16-byte rows: asynchronous 16-byte copies, all in flight at once
        const int q4 = rp / 4;
        for (int e = threadIdx.x; e < nr * q4; e += blockDim.x) {
          const int k = e / q4, j = 4 * (e - k * q4);
          const int left = r - j;
          const int bytes = left >= 4 ? 16 : (left > 0 ? 4 * left : 0);
          cp_async16(Jc + k * rp + j, X + (size_t)(i0 + k) * ldx + (left > 0 ? j : 0), bytes);
        }
        cp_async_commit();
        cp_async_wait<0>();
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

// log u of the accept test: caller-supplied, or from the chain's Philox
// stream STREAM_U at this step.
__device__ double draw_log_u(const ReducedArgs &a, int c) {
  const uint32_t chain = (uint32_t)(a.id_base + (uint64_t)c);
  return a.ext_log_u ? a.ext_log_u[c]
                     : log(word_to_uniform(philox_block(a.seed, STREAM_U, a.step, chain, 0).x));
}

// The accept test log u <= min(0, log rho) (Algorithm 1; NaN rejects).
__device__ __forceinline__ bool accept_decide(double lr, double log_u) {
  return isfinite(lr) && log_u <= fmin(0.0, lr);
}

// The record of the test: log rho, log u, the decision, the counters ([0]
// accepts, [1] non-finite rejects, [2] first-stage accepts), the sum of the
// acceptance probabilities, and the scalar state of an accepted chain, or
// with delayed acceptance its staging for the second stage.  One thread.
__device__ void accept_record(const ReducedArgs &a, int c, double lr, double log_u, bool accept,
                              double phi_b, double hld_b) {
  const bool finite = isfinite(lr);
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
}

// Both at once (thread 0).
__device__ bool accept_test(const ReducedArgs &a, int c, double lr, double phi_b, double hld_b) {
  const double log_u = draw_log_u(a, c);
  const bool accept = accept_decide(lr, log_u);
  accept_record(a, c, lr, log_u, accept, phi_b, hld_b);
  return accept;
}

}  // namespace
}  // namespace dino
