// Tensor-core GEMMs on sm_103a (tcgen05): the reduced MLP and its Jacobian,
// the complement projections, and the per-chain Gram matrices (k_tc_gram).
//
//   D[M x N] = sum_{(i,j): i + j < nslice} A_i B_j^T,   FP32 accumulation in TMEM,
//
// where X ~= X_0 + X_1 + ... are bf16 "slice planes" of an FP32 value
// (X_0 = bf16(X), X_1 = bf16(X - X_0), ...).  nslice = 1 is the plain BF16
// product, 2 the three-product "bf16x3" scheme, 3 six products (FP32-level).
//
// A persistent CTA (one per SM) computes 128 x BN output tiles in turn (cta_group::1, M = 128):
//   warp 0     TMA producer: 3D tiled loads (k, row, slice) of 128 x 64 A and
//              BN x 64 B boxes, 128-byte swizzle, into a ring of stages (one
//              stage per slice pair, or per k-block with every slice of A
//              and B when two such stages fit);
//   warp 1     allocates TMEM (two accumulator buffers) and issues tcgen05.mma
//              (K = 16 per instruction, four per 64-wide stage) into the buffer of
//              the current tile; tcgen05.commit frees each stage and, per tile,
//              hands the buffer to the epilogue;
//   warps 2-5  epilogue: tcgen05.ld of their 32 TMEM lanes, fused bias /
//              activation / derivative / per-chain scaling, bf16 re-slicing,
//              the complement's coefficient and field updates, stores of
//              whole 128-byte row segments through swizzled staging tiles
//              (bulk tensor stores, cp.async.bulk.tensor, where the epilogue
//              stages only its output), overlapping the next tile's MMAs;
//              then release the buffer.
// Work items are output tiles, or (tile, K chunk) pairs when a projection of
// a small pool splits K (FP32 partials, reduced by k_coef_finish).
// Every mbarrier wait is bounded; on timeout the CTA raises a device error
// flag, lets its copies and MMAs drain (bounded), frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "dino_internal.h"

namespace dino {
namespace {

constexpr int kBlockM = 128;
constexpr int kBlockK = 64;  // 128 bytes of bf16: one swizzle row
constexpr int kThreads = 192;
constexpr uint32_t kSpinLimit = 1u << 24;
constexpr int kMaxStages = 4;
constexpr int kStageTiles = 4 * 32 * 128;  // epilogue staging: 32 rows x 128 B per warp
constexpr int kStageTilesTma = 2 * kStageTiles;  // two such tiles per warp (bulk stores)

struct TcParams {
  int M, N, K, BN, nkb, npairs, stages;
  int pair_a[6], pair_b[6];
  int epi, ldo, act, out_slices, lds, group;
  int ldob;  // TC_EPI_STORE_F32 with out_bf: row pitch of the bf16 slice planes
  // split K: work item = (tile, K chunk of kb_per k-blocks); with ksplit > 1
  // every item stores its FP32 partial sums to ws + chunk * M * N (pitch N)
  int ksplit, kb_per;
  float *ws;
  int grouped;  // one stage per k-block carrying every slice (see the kernel)
  int nslice;
  size_t out_plane;
  float *outf;
  const float *bias;
  __nv_bfloat16 *out_bf;
  float *der;
  const float *scale;
  const double *coef;
  int ldc;
  double cs, sc;
  const int *acc;
  float *m;
  const float *Mf;
  int ldm;
  // bulk tensor stores of the epilogue's 128-byte segments (tmO: FP32 output,
  // tmS: bf16 slice planes); the staging region is stg_bytes (two tiles per
  // epilogue warp with tma, else one)
  int tma, stg_bytes;
  uint32_t tmem_cols;
  int *err;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; gives up early when another role has aborted.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    if (mbar_try(bar, parity)) return true;
    if (abort_flag && *abort_flag) return false;
    if (it > 32) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *tm, int c0, int c1,
                                            int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// Bulk tensor stores of the epilogue (shared -> global, 128-byte swizzle):
// the issuing lane commits each store as a bulk group and, before a staging
// tile is written again, waits until the stores that read it are done.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *tm, uint32_t src, int c0, int c1) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];"
               ::"l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(src)
               : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *tm, uint32_t src, int c0, int c1,
                                             int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
          reinterpret_cast<uint64_t>(tm)),
      "r"(c0), "r"(c1), "r"(c2), "r"(src)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), descriptor version 1 (bits 46-47).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: D f32, A and B bf16, both K-major.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Wider TMEM reads for the coalesced epilogue: lane i gets 32 (64) consecutive
// columns of TMEM lane (taddr lane + i); the wait is inside the same asm
// statement, so no use of the values can be scheduled before it.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "{\n tcgen05.ld.sync.aligned.32x32b.x32.b32 {"
      "%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31"
      "}, [%32];\n tcgen05.wait::ld.sync.aligned;\n}\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float v[64]) {
  uint32_t r[64];
  asm volatile(
      "{\n tcgen05.ld.sync.aligned.32x32b.x64.b32 {"
      "%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
      "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
      "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63"
      "}, [%64];\n tcgen05.wait::ld.sync.aligned;\n}\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
        "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
        "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
        "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// Coalesced row stores through a per-warp staging tile.  Lane i holds 128
// bytes (w[0..31]) of output row i of a 32-row block whose first byte is at
// dst + i * ld_bytes (16-byte aligned); rows >= nrows are not stored.  The
// lanes write their rows into `stg` (32 x 128 bytes, 16-byte chunks XOR-
// swizzled by row, so both phases take the minimum four wavefronts per
// instruction), then read it back so that each store instruction writes four
// whole 128-byte row segments instead of 32 scattered 16-byte pieces.
__device__ __forceinline__ void store_rows_coalesced(uint4 *stg, const uint32_t w[32], char *dst,
                                                     size_t ld_bytes, int nrows, int lane) {
#pragma unroll
  for (int c = 0; c < 8; ++c)
    stg[lane * 8 + (c ^ (lane & 7))] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int r = q * 4 + (lane >> 3), c = lane & 7;
    const uint4 x = stg[r * 8 + (c ^ (r & 7))];
    if (r < nrows) *reinterpret_cast<uint4 *>(dst + (size_t)r * ld_bytes + c * 16) = x;
  }
  __syncwarp();
}

// The same 32 x 128-byte segment by one bulk tensor store: the lanes write
// their rows into one of the warp's two staging tiles in the map's 128-byte
// swizzle (chunk c of row r at c ^ (r & 7)), lane 0 stores the tile at
// (x, y[, z]) of the map (rows past the tensor's end are not written) and
// commits it.  Before a tile is written again, lane 0 waits until at most
// one bulk group (the other tile's) is still reading shared memory.
__device__ __forceinline__ void store_rows_tma(uint4 *stg2, int &buf, const uint32_t w[32],
                                               const CUtensorMap *tm, bool three_d, int x, int y,
                                               int z, int nrows, int lane) {
  uint4 *stg = stg2 + buf * 256;
  if (lane == 0) bulk_wait_read1();
  __syncwarp();
#pragma unroll
  for (int c = 0; c < 8; ++c)
    stg[lane * 8 + (c ^ (lane & 7))] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  if (lane == 0 && nrows > 0) {  // a warp whose rows all lie past the end stores nothing
    if (three_d)
      tma_store_3d(tm, smem_u32(stg), x, y, z);
    else
      tma_store_2d(tm, smem_u32(stg), x, y);
    bulk_commit();
  }
  buf ^= 1;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float &a, float &b) {
  // bf16 of a and b (low half a), leaving the remainders a - bf16(a), b - bf16(b):
  // one paired round-to-nearest conversion; a bf16 widens to FP32 exactly by
  // moving its bits to the upper half of the word
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const uint32_t u =
      (uint32_t)__bfloat16_as_ushort(h.x) | ((uint32_t)__bfloat16_as_ushort(h.y) << 16);
  a -= __uint_as_float(u << 16);
  b -= __uint_as_float(u & 0xffff0000u);
  return u;
}

__device__ __forceinline__ float act_fn(int kind, float z) {
  if (kind == 1) return tanhf(z);
  if (kind == 2) return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
  return z;
}
__device__ __forceinline__ float act_deriv(int kind, float z) {
  if (kind == 1) {
    const float t = tanhf(z);
    return 1.0f - t * t;
  }
  if (kind == 2)
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
           z * __expf(-0.5f * z * z) * 0.39894228040143267794f;
  return 1.0f;
}

__device__ __forceinline__ void store_slices(float x, __nv_bfloat16 *dst, size_t plane,
                                             int nslice) {
  float rem = x;
  for (int s = 0; s < nslice; ++s) {
    const __nv_bfloat16 h = __float2bfloat16_rn(rem);
    dst[s * plane] = h;
    rem -= __bfloat162float(h);
  }
}

// Persistent: each CTA walks the output tiles t = blockIdx.x, + gridDim.x, ...
// (N tiles of one M block adjacent, so that concurrent CTAs share A in L2).
// The TMA producer and the MMA issuer run one stage ring across tiles; the
// MMA issuer accumulates tile j into TMEM buffer j & 1 while the epilogue
// warps drain the other buffer (acc_full / acc_empty mbarriers).
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const __grid_constant__ CUtensorMap tmO, const __grid_constant__ CUtensorMap tmS,
              const TcParams p) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  // 1024-byte aligned stage ring, then barriers
  const uint32_t raw = smem_u32(smraw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char *gbase = smraw + (base - raw);
  const uint32_t a_bytes = kBlockM * kBlockK * 2, b_bytes = (uint32_t)p.BN * kBlockK * 2;
  // grouped: a stage holds every slice of A and B of one k-block (A_0 .. A_{s-1},
  // B_0 .. B_{s-1}) and feeds all slice pairs; otherwise one pair per stage
  const uint32_t stage_bytes = p.grouped ? (a_bytes + b_bytes) * (uint32_t)p.nslice
                                         : a_bytes + b_bytes;
  // after the ring: one or two 4 KB epilogue staging tiles per epilogue warp
  // (1024-byte aligned, as the bulk stores' swizzle needs), then the barriers
  uint4 *stg_all = reinterpret_cast<uint4 *>(gbase + p.stages * stage_bytes);
  uint64_t *bars = reinterpret_cast<uint64_t *>(gbase + p.stages * stage_bytes + p.stg_bytes);
  // bars[0..S) full, [S..2S) empty, [2S, 2S+2) acc_full, [2S+2, 2S+4) acc_empty, [2S+4] drain
  const int S = p.stages;
  volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 2 * S + 5);
  volatile int *consumed = abort_flag + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * S + 6);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntn = (p.N + p.BN - 1) / p.BN;
  const int ntiles = ((p.M + kBlockM - 1) / kBlockM) * ntn;
  const int nitems = ntiles * p.ksplit;
  // item t: tile t / ksplit, k-blocks [kb0, kb0 + nk) of chunk t % ksplit
  auto item_k = [&](int t, int &kb0, int &nk) {
    kb0 = (t % p.ksplit) * p.kb_per;
    nk = min(p.kb_per, p.nkb - kb0);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&bars[s]), 1);
      mbar_init(smem_u32(&bars[S + s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bars[2 * S + b]), 1);
      mbar_init(smem_u32(&bars[2 * S + 2 + b]), 4);  // one arrive per epilogue warp
    }
    mbar_init(smem_u32(&bars[2 * S + 4]), 1);
    *abort_flag = 0;
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int g = 0;  // stage iterations issued, across tiles
      bool ok = true;
      for (int t = blockIdx.x; t < nitems && ok; t += gridDim.x) {
        const int tile = t / p.ksplit;
        const int m0 = (tile / ntn) * kBlockM, n0 = (tile % ntn) * p.BN;
        int kb0, nk;
        item_k(t, kb0, nk);
        const int n_iter = p.grouped ? nk : p.npairs * nk;
        for (int it = 0; it < n_iter; ++it, ++g) {
          const int s = g % S;
          const uint32_t ph = (uint32_t)(g / S) & 1u;
          if (!mbar_wait(smem_u32(&bars[S + s]), ph ^ 1u, abort_flag)) {
            *abort_flag = 1;
            atomicOr(p.err, 1);
            ok = false;
            break;
          }
          const uint32_t full = smem_u32(&bars[s]);
          mbar_expect_tx(full, stage_bytes);
          const uint32_t sa = base + s * stage_bytes;
          if (p.grouped) {
            const int kb = kb0 + it;
            for (int sl = 0; sl < p.nslice; ++sl)
              tma_load_3d(sa + sl * a_bytes, &tmA, kb * kBlockK, m0, sl, full);
            for (int sl = 0; sl < p.nslice; ++sl)
              tma_load_3d(sa + p.nslice * a_bytes + sl * b_bytes, &tmB, kb * kBlockK, n0, sl,
                          full);
          } else {
            const int pr = it / nk, kb = kb0 + it % nk;
            tma_load_3d(sa, &tmA, kb * kBlockK, m0, p.pair_a[pr], full);
            tma_load_3d(sa + a_bytes, &tmB, kb * kBlockK, n0, p.pair_b[pr], full);
          }
        }
      }
      if (*abort_flag) {
        // let the copies already issued land before the CTA's memory goes away
        for (int i = *consumed; i < g; ++i)
          mbar_wait(smem_u32(&bars[i % S]), (uint32_t)(i / S) & 1u, nullptr);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kBlockM, p.BN);
      bool ok = true;
      int g = 0, j = 0;
      for (int t = blockIdx.x; t < nitems && ok; t += gridDim.x, ++j) {
        const int b = j & 1;
        if (!mbar_wait(smem_u32(&bars[2 * S + 2 + b]), (((uint32_t)j >> 1) & 1u) ^ 1u,
                       abort_flag)) {
          *abort_flag = 1;
          atomicOr(p.err, 2);
          ok = false;
          break;
        }
        fence_after();
        const uint32_t tacc = tmem + (uint32_t)(b * p.BN);
        int kb0, nk;
        item_k(t, kb0, nk);
        const int n_iter = p.grouped ? nk : p.npairs * nk;
        for (int it = 0; it < n_iter; ++it, ++g) {
          const int s = g % S;
          const uint32_t ph = (uint32_t)(g / S) & 1u;
          if (!mbar_wait(smem_u32(&bars[s]), ph, abort_flag)) {
            *abort_flag = 1;
            atomicOr(p.err, 2);
            ok = false;
            break;
          }
          *consumed = g + 1;
          fence_after();
          const uint32_t sa = base + s * stage_bytes;
          if (p.grouped) {
            for (int pr = 0; pr < p.npairs; ++pr) {
              const uint64_t ad = smem_desc_sw128(sa + p.pair_a[pr] * a_bytes);
              const uint64_t bd =
                  smem_desc_sw128(sa + p.nslice * a_bytes + p.pair_b[pr] * b_bytes);
#pragma unroll
              for (int k = 0; k < kBlockK / 16; ++k)
                mma_bf16(tacc, ad + 2 * k, bd + 2 * k, idesc,
                         (it > 0 || pr > 0 || k > 0) ? 1u : 0u);
            }
          } else {
            const uint64_t ad = smem_desc_sw128(sa), bd = smem_desc_sw128(sa + a_bytes);
#pragma unroll
            for (int k = 0; k < kBlockK / 16; ++k)
              mma_bf16(tacc, ad + 2 * k, bd + 2 * k, idesc, (it > 0 || k > 0) ? 1u : 0u);
          }
          mma_commit(smem_u32(&bars[S + s]));
        }
        if (ok) mma_commit(smem_u32(&bars[2 * S + b]));
      }
      if (!ok) {  // drain the MMAs already issued
        mma_commit(smem_u32(&bars[2 * S + 4]));
        mbar_wait(smem_u32(&bars[2 * S + 4]), 0, nullptr);
      }
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31
    const int quarter = warp & 3;
    int sbuf = 0;  // staging tile of the next bulk store
    int j = 0;
    for (int t = blockIdx.x; t < nitems; t += gridDim.x, ++j) {
      const int b = j & 1;
      const int tile = t / p.ksplit;
      const int m0 = (tile / ntn) * kBlockM, n0 = (tile % ntn) * p.BN;
      // a K chunk of a split product stores FP32 partial sums (pitch N)
      const bool split = p.ksplit > 1;
      const int epi = split ? (int)TC_EPI_STORE_F32 : p.epi;
      float *outf = split ? p.ws + (size_t)(t % p.ksplit) * p.M * p.N : p.outf;
      const int ldo = split ? p.N : p.ldo;
      __nv_bfloat16 *const out_bf = split ? nullptr : p.out_bf;
      const int row = m0 + quarter * 32 + lane;
      // one lane waits, the warp follows its verdict (tcgen05.ld is warp-collective)
      int okl = 0;
      if (lane == 0)
        okl = mbar_wait(smem_u32(&bars[2 * S + b]), ((uint32_t)j >> 1) & 1u, abort_flag) ? 1 : 0;
      if (__shfl_sync(0xffffffffu, okl, 0) == 0) {
        if (lane == 0) {
          *abort_flag = 1;
          atomicOr(p.err, 4);
        }
        break;
      }
      fence_after();
      const uint32_t tacc = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * p.BN);
      const int nvalid = min(p.BN, p.N - n0);
      const int row0 = m0 + quarter * 32, nrows = min(32, p.M - row0);
      uint4 *stg = stg_all + quarter * (p.stg_bytes / 64);
      int c0 = 0;  // columns [0, c0) done by the coalesced groups below
      if (epi == TC_EPI_FIELD_T) {
        // lanes are consecutive field nodes of one chain per column: each
        // column's loads and stores are 128 contiguous bytes per warp
        for (; c0 < nvalid; c0 += 16) {
          float v[16];
          tmem_ld16(tacc + (uint32_t)c0, v);
          if (row < p.M) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int ch = n0 + c0 + j;
              if (c0 + j < nvalid && p.acc[ch]) {
                const size_t o = (size_t)ch * p.ldm + row;
                p.m[o] = (float)(p.sc * (double)p.m[o] + p.cs * (double)p.Mf[o]) + v[j];
              }
            }
          }
        }
      } else if (epi == TC_EPI_STORE_F32 && out_bf) {
        // FP32 values and their bf16 slices: 64 columns = two 128-byte FP32
        // halves and one 128-byte segment per slice
        if ((ldo & 3) == 0 && (p.ldob & 7) == 0) {
          for (; c0 + 64 <= nvalid; c0 += 64) {
            float v[64];
            tmem_ld64(tacc + (uint32_t)c0, v);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              uint32_t w[32];
#pragma unroll
              for (int j = 0; j < 32; ++j) w[j] = __float_as_uint(v[32 * h + j]);
              if (p.tma)
                store_rows_tma(stg, sbuf, w, &tmO, false, n0 + c0 + 32 * h, row0, 0, nrows,
                               lane);
              else
                store_rows_coalesced(
                    stg, w, reinterpret_cast<char *>(outf + (size_t)row0 * ldo + n0 + c0 + 32 * h),
                    (size_t)ldo * 4, nrows, lane);
            }
            for (int sl = 0; sl < p.out_slices; ++sl) {
              uint32_t w[32];
#pragma unroll
              for (int j = 0; j < 32; ++j) w[j] = pack_bf16x2(v[2 * j], v[2 * j + 1]);
              if (p.tma)
                store_rows_tma(stg, sbuf, w, &tmS, true, n0 + c0, row0, sl, nrows, lane);
              else
                store_rows_coalesced(
                    stg, w,
                    reinterpret_cast<char *>(out_bf + (size_t)row0 * p.ldob + n0 + c0 +
                                             (size_t)sl * p.out_plane),
                    (size_t)p.ldob * 2, nrows, lane);
            }
          }
        }
      } else if ((epi == TC_EPI_STORE_F32 || epi == TC_EPI_BIAS_F32) && (ldo & 3) == 0 &&
                 (reinterpret_cast<uintptr_t>(outf) & 15) == 0) {
        // 32 FP32 columns = 128 bytes per row
        for (; c0 + 32 <= nvalid; c0 += 32) {
          float v[32];
          tmem_ld32(tacc + (uint32_t)c0, v);
          uint32_t w[32];
#pragma unroll
          for (int j = 0; j < 32; ++j)
            w[j] = __float_as_uint(epi == TC_EPI_BIAS_F32 ? v[j] + p.bias[n0 + c0 + j] : v[j]);
          store_rows_coalesced(stg, w, reinterpret_cast<char *>(outf + (size_t)row0 * ldo + n0 + c0),
                               (size_t)ldo * 4, nrows, lane);
        }
      } else if ((epi == TC_EPI_SCALE_GROUP && (p.lds & 3) == 0) ||
                 (epi == TC_EPI_BIAS_ACT && (p.N & 3) == 0) || epi == TC_EPI_COEF) {
        // 64 columns = 128 bytes per row and bf16 slice (the derivative: two
        // 128-byte FP32 halves)
        if ((ldo & 7) == 0) {
          for (; c0 + 64 <= nvalid; c0 += 64) {
            float v[64];
            tmem_ld64(tacc + (uint32_t)c0, v);
            if (epi == TC_EPI_COEF) {
              if (row < p.M) {
                const double *cf = p.coef + (size_t)row * p.ldc + n0 + c0;
#pragma unroll
                for (int j = 0; j < 64; ++j) v[j] = (float)(cf[j] - p.cs * (double)v[j]);
              }
            } else if (epi == TC_EPI_SCALE_GROUP) {
              if (row < p.M) {
                const float4 *sc = reinterpret_cast<const float4 *>(
                    p.scale + (size_t)(row / p.group) * p.lds + n0 + c0);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                  const float4 t = sc[q];
                  v[4 * q] *= t.x;
                  v[4 * q + 1] *= t.y;
                  v[4 * q + 2] *= t.z;
                  v[4 * q + 3] *= t.w;
                }
              }
            } else {
#pragma unroll
              for (int j = 0; j < 64; ++j) v[j] += p.bias[n0 + c0 + j];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                uint32_t w[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) w[j] = __float_as_uint(act_deriv(p.act, v[32 * h + j]));
                if (p.tma)  // tmO maps the derivative here
                  store_rows_tma(stg, sbuf, w, &tmO, false, n0 + c0 + 32 * h, row0, 0, nrows,
                                 lane);
                else
                  store_rows_coalesced(
                      stg, w,
                      reinterpret_cast<char *>(p.der + (size_t)row0 * p.N + n0 + c0 + 32 * h),
                      (size_t)p.N * 4, nrows, lane);
              }
#pragma unroll
              for (int j = 0; j < 64; ++j) v[j] = act_fn(p.act, v[j]);
            }
            for (int sl = 0; sl < p.out_slices; ++sl) {
              uint32_t w[32];
#pragma unroll
              for (int j = 0; j < 32; ++j) w[j] = pack_bf16x2(v[2 * j], v[2 * j + 1]);
              if (p.tma)
                store_rows_tma(stg, sbuf, w, &tmS, true, n0 + c0, row0, sl, nrows, lane);
              else
                store_rows_coalesced(
                    stg, w,
                    reinterpret_cast<char *>(out_bf + (size_t)row0 * ldo + n0 + c0 +
                                             (size_t)sl * p.out_plane),
                    (size_t)ldo * 2, nrows, lane);
            }
          }
        }
      }
      for (; c0 < nvalid; c0 += 16) {
        float v[16];
        tmem_ld16(tacc + (uint32_t)c0, v);
        if (row >= p.M) continue;
        const int ncols = min(16, nvalid - c0);
        const int col0 = n0 + c0;
        if (epi == TC_EPI_STORE_F32 || epi == TC_EPI_BIAS_F32) {
          if (epi == TC_EPI_BIAS_F32)
            for (int j = 0; j < ncols; ++j) v[j] += p.bias[col0 + j];
          // a ragged last group of 4, 8 or 12 columns (N = 200 leaves 8) in
          // 16-byte stores as well: one per 4 FP32 values, one per 8 bf16s
          float *o = outf + (size_t)row * ldo + col0;
          if ((ncols & 3) == 0 && (ldo & 3) == 0 && (reinterpret_cast<uintptr_t>(outf) & 15) == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (4 * q < ncols)
                reinterpret_cast<float4 *>(o)[q] =
                    make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
          } else {
            for (int j = 0; j < ncols; ++j) o[j] = v[j];
          }
          if (epi == TC_EPI_STORE_F32 && out_bf) {
            __nv_bfloat16 *ob = out_bf + (size_t)row * p.ldob + col0;
            if ((ncols & 7) == 0 && (p.ldob & 7) == 0 && (p.out_plane & 7) == 0 &&
                (reinterpret_cast<uintptr_t>(out_bf) & 15) == 0) {
              for (int sl = 0; sl < p.out_slices; ++sl) {
                uint32_t h[8];  // pack_bf16x2 leaves the remainders in v
#pragma unroll
                for (int j = 0; j < 8; ++j) h[j] = pack_bf16x2(v[2 * j], v[2 * j + 1]);
                uint4 *os = reinterpret_cast<uint4 *>(ob + (size_t)sl * p.out_plane);
                os[0] = make_uint4(h[0], h[1], h[2], h[3]);
                if (ncols == 16) os[1] = make_uint4(h[4], h[5], h[6], h[7]);
              }
            } else {
              for (int j = 0; j < ncols; ++j)
                store_slices(v[j], ob + j, p.out_plane, p.out_slices);
            }
          }
        } else {
          float x[16];
          if (epi == TC_EPI_BIAS_ACT) {
            float *d = p.der + (size_t)row * p.N + col0;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const float z = v[j] + (j < ncols ? p.bias[col0 + j] : 0.0f);
              x[j] = act_fn(p.act, z);
              v[j] = act_deriv(p.act, z);
            }
            if (ncols == 16 && (p.N & 3) == 0) {
#pragma unroll
              for (int q = 0; q < 4; ++q)
                reinterpret_cast<float4 *>(d)[q] =
                    make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            } else {
              for (int j = 0; j < ncols; ++j) d[j] = v[j];
            }
          } else if (epi == TC_EPI_COEF) {
            const double *cf = p.coef + (size_t)row * p.ldc + col0;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              x[j] = j < ncols ? (float)(cf[j] - p.cs * (double)v[j]) : 0.0f;
          } else {
            const float *sc = p.scale + (size_t)(row / p.group) * p.lds + col0;
            if (ncols == 16 && (p.lds & 3) == 0) {
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const float4 t = reinterpret_cast<const float4 *>(sc)[q];
                x[4 * q] = v[4 * q] * t.x;
                x[4 * q + 1] = v[4 * q + 1] * t.y;
                x[4 * q + 2] = v[4 * q + 2] * t.z;
                x[4 * q + 3] = v[4 * q + 3] * t.w;
              }
            } else {
              for (int j = 0; j < 16; ++j) x[j] = j < ncols ? v[j] * sc[j] : 0.0f;
            }
          }
          // x ~= sum of bf16 slices; 16-byte stores of 8 values per slice
          __nv_bfloat16 *o = out_bf + (size_t)row * ldo + col0;
          const bool vec = ncols == 16 && (ldo & 7) == 0;
          for (int sl = 0; sl < p.out_slices; ++sl) {
            uint32_t h[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) h[j] = pack_bf16x2(x[2 * j], x[2 * j + 1]);
            __nv_bfloat16 *os = o + sl * p.out_plane;
            if (vec) {
              reinterpret_cast<uint4 *>(os)[0] = make_uint4(h[0], h[1], h[2], h[3]);
              reinterpret_cast<uint4 *>(os)[1] = make_uint4(h[4], h[5], h[6], h[7]);
            } else {
              for (int j = 0; j < ncols; ++j)
                os[j] = __ushort_as_bfloat16((unsigned short)(h[j >> 1] >> (16 * (j & 1))));
            }
          }
        }
      }
      // buffer b drained: hand it back to the MMA issuer
      fence_before();
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bars[2 * S + 2 + b]))
                     : "memory");
    }
    // the bulk stores have read their staging tiles and written global memory
    if (p.tma && lane == 0) bulk_wait_all();
    __syncwarp();
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(p.tmem_cols)
                 : "memory");
  }
}

// Per-group Gram matrices G_c = J_c J_c^T (persistent, one CTA per SM, groups
// c = blockIdx.x, + gridDim.x, ...).  A stage holds one 64-wide k-block of
// all slices of the 128 rows starting at row c g (the rows past the group
// belong to the next group or are zero-filled past the end, and are never
// stored); both MMA operands are views of the same staged tile, B its first
// BN = ceil16(g) rows.  Roles and bounded waits as in k_tc_gemm; the
// epilogue writes rows i < g, columns j < g.
struct GramParams {
  int C, g, K, BN, nkb, nslice, npairs, stages;
  int pair_a[6], pair_b[6];
  float *out;
  int ldo;
  uint32_t tmem_cols;
  int *err;
};

__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gram(const __grid_constant__ CUtensorMap tmJ, const GramParams p) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  const uint32_t raw = smem_u32(smraw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char *gbase = smraw + (base - raw);
  const uint32_t tile_bytes = kBlockM * kBlockK * 2;  // one slice of the stage
  const uint32_t stage_bytes = tile_bytes * (uint32_t)p.nslice;
  uint4 *stg_all = reinterpret_cast<uint4 *>(gbase + p.stages * stage_bytes);
  uint64_t *bars = reinterpret_cast<uint64_t *>(gbase + p.stages * stage_bytes + kStageTiles);
  const int S = p.stages;
  volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 2 * S + 5);
  volatile int *consumed = abort_flag + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * S + 6);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&bars[s]), 1);
      mbar_init(smem_u32(&bars[S + s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bars[2 * S + b]), 1);
      mbar_init(smem_u32(&bars[2 * S + 2 + b]), 4);
    }
    mbar_init(smem_u32(&bars[2 * S + 4]), 1);
    *abort_flag = 0;
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int g = 0;
      bool ok = true;
      for (int c = blockIdx.x; c < p.C && ok; c += gridDim.x) {
        for (int kb = 0; kb < p.nkb; ++kb, ++g) {
          const int s = g % S;
          const uint32_t ph = (uint32_t)(g / S) & 1u;
          if (!mbar_wait(smem_u32(&bars[S + s]), ph ^ 1u, abort_flag)) {
            *abort_flag = 1;
            atomicOr(p.err, 1);
            ok = false;
            break;
          }
          const uint32_t full = smem_u32(&bars[s]);
          mbar_expect_tx(full, stage_bytes);
          const uint32_t sa = base + s * stage_bytes;
          for (int sl = 0; sl < p.nslice; ++sl)
            tma_load_3d(sa + sl * tile_bytes, &tmJ, kb * kBlockK, c * p.g, sl, full);
        }
      }
      if (*abort_flag) {
        for (int i = *consumed; i < g; ++i)
          mbar_wait(smem_u32(&bars[i % S]), (uint32_t)(i / S) & 1u, nullptr);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kBlockM, p.BN);
      bool ok = true;
      int g = 0, j = 0;
      for (int c = blockIdx.x; c < p.C && ok; c += gridDim.x, ++j) {
        const int b = j & 1;
        if (!mbar_wait(smem_u32(&bars[2 * S + 2 + b]), (((uint32_t)j >> 1) & 1u) ^ 1u,
                       abort_flag)) {
          *abort_flag = 1;
          atomicOr(p.err, 2);
          ok = false;
          break;
        }
        fence_after();
        const uint32_t tacc = tmem + (uint32_t)(b * p.BN);
        for (int kb = 0; kb < p.nkb; ++kb, ++g) {
          const int s = g % S;
          const uint32_t ph = (uint32_t)(g / S) & 1u;
          if (!mbar_wait(smem_u32(&bars[s]), ph, abort_flag)) {
            *abort_flag = 1;
            atomicOr(p.err, 2);
            ok = false;
            break;
          }
          *consumed = g + 1;
          fence_after();
          const uint32_t sa = base + s * stage_bytes;
          for (int pr = 0; pr < p.npairs; ++pr) {
            const uint64_t ad = smem_desc_sw128(sa + p.pair_a[pr] * tile_bytes);
            const uint64_t bd = smem_desc_sw128(sa + p.pair_b[pr] * tile_bytes);
#pragma unroll
            for (int k = 0; k < kBlockK / 16; ++k)
              mma_bf16(tacc, ad + 2 * k, bd + 2 * k, idesc, (kb > 0 || pr > 0 || k > 0) ? 1u : 0u);
          }
          mma_commit(smem_u32(&bars[S + s]));
        }
        if (ok) mma_commit(smem_u32(&bars[2 * S + b]));
      }
      if (!ok) {
        mma_commit(smem_u32(&bars[2 * S + 4]));
        mbar_wait(smem_u32(&bars[2 * S + 4]), 0, nullptr);
      }
    }
  } else {
    const int quarter = warp & 3;
    const int i0 = quarter * 32, nrows = min(32, p.g - i0);  // rows of this warp in the group
    uint4 *stg = stg_all + quarter * 256;
    int j = 0;
    for (int c = blockIdx.x; c < p.C; c += gridDim.x, ++j) {
      const int b = j & 1;
      int okl = 0;
      if (lane == 0)
        okl = mbar_wait(smem_u32(&bars[2 * S + b]), ((uint32_t)j >> 1) & 1u, abort_flag) ? 1 : 0;
      if (__shfl_sync(0xffffffffu, okl, 0) == 0) {
        if (lane == 0) {
          *abort_flag = 1;
          atomicOr(p.err, 4);
        }
        break;
      }
      fence_after();
      const uint32_t tacc = tmem + ((uint32_t)(i0) << 16) + (uint32_t)(b * p.BN);
      float *orow = p.out + ((size_t)c * p.g + i0) * p.ldo;
      int c0 = 0;
      if ((p.ldo & 3) == 0) {
        for (; c0 + 32 <= p.g; c0 += 32) {
          float v[32];
          tmem_ld32(tacc + (uint32_t)c0, v);
          uint32_t w[32];
#pragma unroll
          for (int q = 0; q < 32; ++q) w[q] = __float_as_uint(v[q]);
          store_rows_coalesced(stg, w, reinterpret_cast<char *>(orow + c0), (size_t)p.ldo * 4,
                               nrows, lane);
        }
      }
      for (; c0 < p.g; c0 += 16) {
        float v[16];
        tmem_ld16(tacc + (uint32_t)c0, v);
        if (lane < nrows)
          for (int q = 0; q < 16 && c0 + q < p.g; ++q) orow[(size_t)lane * p.ldo + c0 + q] = v[q];
      }
      fence_before();
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bars[2 * S + 2 + b]))
                     : "memory");
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(p.tmem_cols)
                 : "memory");
  }
}

// Split-K finish of TC_EPI_COEF: out slices = coef - cs * (sum of the K
// chunks' FP32 partials), in chunk order.
__global__ void k_coef_finish(uint32_t total, int N, int ksplit, const float *__restrict__ ws,
                              const double *__restrict__ coef, int ldc, double cs,
                              __nv_bfloat16 *__restrict__ out, int ldo, size_t plane,
                              int nslice) {
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += gridDim.x * blockDim.x) {
    const uint32_t row = e / (uint32_t)N, col = e - row * (uint32_t)N;
    float acc = 0.0f;
    for (int k = 0; k < ksplit; ++k) acc += ws[(size_t)k * total + e];
    const float x = (float)(coef[(size_t)row * ldc + col] - cs * (double)acc);
    store_slices(x, out + (size_t)row * ldo + col, plane, nslice);
  }
}

__global__ void k_split_bf16(int rows, int cols, const double *__restrict__ src, int lds,
                             __nv_bfloat16 *__restrict__ dst, int ldd, size_t plane, int nslice) {
  const size_t total = (size_t)rows * cols;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / cols;
    const int j = (int)(e % cols);
    store_slices((float)src[i * lds + j], dst + i * ldd + j, plane, nslice);
  }
}

__global__ void k_jac_init_bf16(int C, int d_y, int w, const float *__restrict__ WL,
                                const float *__restrict__ der, int ldd,
                                __nv_bfloat16 *__restrict__ P, int ldp, size_t plane,
                                int nslice) {
  // P = W_L .* der (per chain).  Work items are groups of 8 consecutive
  // columns of one row (c, i), enumerated row-major over all rows, so that
  // consecutive threads write consecutive 16-byte pieces and every thread
  // has the same share; float4 loads when the rows are 16-byte aligned.
  const int groups = (w + 7) / 8;
  const size_t items = (size_t)C * d_y * groups;
  const bool vload = (w & 3) == 0 && (ldd & 3) == 0;
  const bool vstore = (ldp & 7) == 0;
  // 32-bit index arithmetic (the launcher caps items below 2^32)
  const uint32_t nitems = (uint32_t)items, ug = (uint32_t)groups, udy = (uint32_t)d_y;
  for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < nitems;
       it += gridDim.x * blockDim.x) {
    const uint32_t urow = it / ug;
    const int g = (int)(it - urow * ug);
    const size_t row = urow;
    const int c = (int)(urow / udy), i = (int)(urow - (uint32_t)c * udy);
    const float *wr = WL + (size_t)i * w;
    const float *dr = der + (size_t)c * ldd;
    __nv_bfloat16 *o = P + row * ldp;
    const int k0 = 8 * g;
    float x[8];
    if (vload && k0 + 8 <= w) {
      const float4 w0 = *reinterpret_cast<const float4 *>(wr + k0);
      const float4 w1 = *reinterpret_cast<const float4 *>(wr + k0 + 4);
      const float4 d0 = *reinterpret_cast<const float4 *>(dr + k0);
      const float4 d1 = *reinterpret_cast<const float4 *>(dr + k0 + 4);
      x[0] = w0.x * d0.x; x[1] = w0.y * d0.y; x[2] = w0.z * d0.z; x[3] = w0.w * d0.w;
      x[4] = w1.x * d1.x; x[5] = w1.y * d1.y; x[6] = w1.z * d1.z; x[7] = w1.w * d1.w;
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) x[q] = k0 + q < w ? wr[k0 + q] * dr[k0 + q] : 0.0f;
    }
    const bool vec = vstore && k0 + 8 <= ldp;
    for (int sl = 0; sl < nslice; ++sl) {
      uint32_t h[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) h[q] = pack_bf16x2(x[2 * q], x[2 * q + 1]);
      __nv_bfloat16 *os = o + sl * plane + k0;
      if (vec) {
        *reinterpret_cast<uint4 *>(os) = make_uint4(h[0], h[1], h[2], h[3]);
      } else {
        for (int q = 0; q < 8 && k0 + q < w; ++q) {
          const uint32_t hw = h[q >> 1] >> (16 * (q & 1));
          os[q] = __ushort_as_bfloat16((unsigned short)(hw & 0xffffu));
        }
      }
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
  }
  return fn;
}

// 3D map over slice planes: dims (K, rows, slices), box (64, box_rows, 1).
bool make_map(CUtensorMap *tm, const __nv_bfloat16 *ptr, int K, int rows, int ld, size_t plane,
              int slices, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)slices};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)plane * 2};
  cuuint32_t box[3] = {(cuuint32_t)kBlockK, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)ptr, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2D map over an FP32 matrix for the epilogue's bulk stores: dims (cols,
// rows), box (32, 32): one 128-byte segment of 32 rows.
bool make_map_f32(CUtensorMap *tm, const float *ptr, int cols, int rows, int ld) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t es[2] = {1, 1};
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)ptr, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int *error_word() {
  static int *d = nullptr;
  if (!d && cudaMalloc(&d, sizeof(int)) == cudaSuccess) cudaMemset(d, 0, sizeof(int));
  return d;
}

}  // namespace

int tc_error_flag(bool reset) {
  int *d = error_word();
  if (!d) return 0;
  int h = 0;
  cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
  if (reset) cudaMemset(d, 0, sizeof(int));
  return h;
}

cudaError_t launch_tc_gemm(const TcGemmArgs &a, cudaStream_t st) {
  if (a.M <= 0 || a.N <= 0) return cudaSuccess;
  if (a.nslice < 1 || a.nslice > 3 || a.K <= 0 || (a.lda & 7) || (a.ldb & 7) ||
      (a.a_plane & 7) || (a.b_plane & 7) || ((uintptr_t)a.A & 15) || ((uintptr_t)a.B & 15))
    return cudaErrorInvalidValue;
  TcParams p{};
  p.M = a.M;
  p.N = a.N;
  p.K = a.K;
  // the complement's three-slice products (long K, many tiles): at most 128
  // columns, so that a stage with a k-block of every slice of A and B (at
  // most 96 KB) fits twice and each slice is loaded once per k-block
  const bool narrow = a.nslice == 3 && (a.epi == TC_EPI_COEF || a.epi == TC_EPI_FIELD_T);
  const int bn_max = narrow ? 128 : 256;
  const int ntiles = (a.N + bn_max - 1) / bn_max;
  p.BN = ((a.N + ntiles - 1) / ntiles + 15) / 16 * 16;
  p.nkb = (a.K + kBlockK - 1) / kBlockK;
  static const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
  p.npairs = a.nslice == 1 ? 1 : (a.nslice == 2 ? 3 : 6);
  for (int i = 0; i < 6; ++i) {
    p.pair_a[i] = pa[i];
    p.pair_b[i] = pb[i];
  }
  // group the slices of a k-block into one stage when two such stages fit
  // (the two-slice Jacobian products: each A and B tile loaded once per
  // k-block instead of once per slice pair)
  const int pair_bytes = kBlockM * kBlockK * 2 + p.BN * kBlockK * 2;
  p.nslice = a.nslice;
  p.grouped = a.nslice > 1 && 2 * pair_bytes * a.nslice <= 200 * 1024;
  const int stage_bytes = p.grouped ? pair_bytes * a.nslice : pair_bytes;
  p.stages = (200 * 1024) / stage_bytes;
  if (p.stages > kMaxStages) p.stages = kMaxStages;
  if (p.stages < 2) p.stages = 2;
  p.epi = a.epi;
  p.ldo = a.ldo;
  p.act = a.act;
  p.out_slices = a.out_slices;
  p.lds = a.lds;
  p.group = a.group > 0 ? a.group : 1;
  p.out_plane = a.out_plane;
  p.ldob = a.ldob;
  p.outf = a.outf;
  p.bias = a.bias;
  p.out_bf = a.out_bf;
  p.der = a.der;
  p.scale = a.scale;
  p.coef = a.coef;
  p.ldc = a.ldc;
  p.cs = a.cs;
  p.sc = a.sc;
  p.acc = a.acc;
  p.m = a.m;
  p.Mf = a.Mf;
  p.ldm = a.ldm;
  uint32_t cols = 32;  // two accumulator buffers of BN columns
  while (cols < 2u * (uint32_t)p.BN) cols <<= 1;
  p.tmem_cols = cols;
  p.err = error_word();
  if (!p.err) return cudaErrorMemoryAllocation;
  CUtensorMap tmA, tmB;
  if (!make_map(&tmA, a.A, a.K, a.M, a.lda, a.a_plane, a.nslice, kBlockM) ||
      !make_map(&tmB, a.B, a.K, a.N, a.ldb, a.b_plane, a.nslice, p.BN))
    return cudaErrorInvalidValue;
  int dev = 0, sms = 0;  // persistent grid: one CTA per SM (its shared memory allows one)
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return cudaErrorInvalidValue;
  const int total = ((a.M + kBlockM - 1) / kBlockM) * ntiles;
  // split K when the tiles fill fewer than two CTAs per SM (the projections
  // of small pools: M = chains, K = field nodes)
  p.ksplit = 1;
  p.kb_per = p.nkb;
  p.ws = nullptr;
  if (a.epi == TC_EPI_COEF && a.ws && total < 2 * sms &&
      (size_t)a.M * a.N < 0xffffffffull - 152ull * 32 * 256) {
    int ks = std::min({(2 * sms + total - 1) / total, 16, p.nkb});
    while (ks > 1 && (size_t)ks * a.M * a.N > a.ws_floats) --ks;
    if (ks > 1) {
      p.kb_per = (p.nkb + ks - 1) / ks;
      p.ksplit = (p.nkb + p.kb_per - 1) / p.kb_per;
      p.ws = a.ws;
    }
  }
  // bulk tensor stores for the epilogues that stage only their output's
  // 128-byte segments (FP32 with slices, scaled or coefficient slices), when
  // the maps encode and two staging tiles per warp fit
  CUtensorMap tmO, tmS;
  std::memset(&tmO, 0, sizeof(tmO));
  std::memset(&tmS, 0, sizeof(tmS));
  const size_t smem_base = 1024 + (size_t)p.stages * stage_bytes + (2 * p.stages + 8) * 8;
  p.tma = 0;
  p.stg_bytes = kStageTiles;
  if (p.ksplit == 1 && a.out_bf && smem_base + kStageTilesTma <= 227 * 1024) {
    if (a.epi == TC_EPI_STORE_F32 && a.outf)
      p.tma = make_map_f32(&tmO, a.outf, a.N, a.M, a.ldo) &&
              make_map(&tmS, a.out_bf, a.N, a.M, a.ldob, a.out_plane, a.out_slices, 32);
    else if (a.epi == TC_EPI_SCALE_GROUP || a.epi == TC_EPI_COEF)
      p.tma = make_map(&tmS, a.out_bf, a.N, a.M, a.ldo, a.out_plane, a.out_slices, 32);
    else if (a.epi == TC_EPI_BIAS_ACT && a.der)  // the derivative (pitch N) and the slices
      p.tma = make_map_f32(&tmO, a.der, a.N, a.M, a.N) &&
              make_map(&tmS, a.out_bf, a.N, a.M, a.ldo, a.out_plane, a.out_slices, 32);
    if (p.tma) p.stg_bytes = kStageTilesTma;
  }
  const size_t smem = smem_base + p.stg_bytes;
  cudaError_t e =
      cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_tc_gemm<<<std::min(total * p.ksplit, sms), kThreads, smem, st>>>(tmA, tmB, tmO, tmS, p);
  cudaError_t e2 = cudaGetLastError();
  if (e2 != cudaSuccess || p.ksplit == 1) return e2;
  const size_t n = (size_t)a.M * a.N;
  const int grid = (int)std::min<size_t>((n + 255) / 256, 152 * 32);
  k_coef_finish<<<grid, 256, 0, st>>>((uint32_t)n, a.N, p.ksplit, p.ws, a.coef, a.ldc, a.cs,
                                      a.out_bf, a.ldo, a.out_plane, a.out_slices);
  return cudaGetLastError();
}

cudaError_t launch_tc_gram(int C, int g, int K, const __nv_bfloat16 *J, int ldj, size_t plane,
                           int nslice, float *out, int ldo, cudaStream_t st) {
  if (C <= 0) return cudaSuccess;
  if (g < 1 || g > kBlockM || K <= 0 || nslice < 1 || nslice > 3 || (ldj & 7) || (plane & 7) ||
      ((uintptr_t)J & 15) || ldo < g || ((uintptr_t)out & 15))
    return cudaErrorInvalidValue;
  GramParams p{};
  p.C = C;
  p.g = g;
  p.K = K;
  p.BN = (g + 15) / 16 * 16;
  p.nkb = (K + kBlockK - 1) / kBlockK;
  p.nslice = nslice;
  static const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
  p.npairs = nslice == 1 ? 1 : (nslice == 2 ? 3 : 6);
  for (int i = 0; i < 6; ++i) {
    p.pair_a[i] = pa[i];
    p.pair_b[i] = pb[i];
  }
  const int stage_bytes = kBlockM * kBlockK * 2 * nslice;
  p.stages = std::max(2, std::min(kMaxStages, (200 * 1024) / stage_bytes));
  p.out = out;
  p.ldo = ldo;
  uint32_t cols = 32;
  while (cols < 2u * (uint32_t)p.BN) cols <<= 1;
  p.tmem_cols = cols;
  p.err = error_word();
  if (!p.err) return cudaErrorMemoryAllocation;
  CUtensorMap tm;
  if ((long long)C * g > 0x7fffffffLL ||
      !make_map(&tm, J, K, C * g, ldj, plane, nslice, kBlockM))
    return cudaErrorInvalidValue;
  const size_t smem = 1024 + (size_t)p.stages * stage_bytes + kStageTiles + (2 * p.stages + 8) * 8;
  cudaError_t e =
      cudaFuncSetAttribute(k_tc_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return cudaErrorInvalidValue;
  k_tc_gram<<<std::min(C, sms), kThreads, smem, st>>>(tm, p);
  return cudaGetLastError();
}

cudaError_t launch_split_bf16_f64(int rows, int cols, const double *src, int lds,
                                  __nv_bfloat16 *dst, int ldd, size_t plane, int nslice,
                                  cudaStream_t st) {
  const size_t n = (size_t)rows * cols;
  const int grid = (int)std::min<size_t>((n + 255) / 256, 152 * 32);
  k_split_bf16<<<grid > 0 ? grid : 1, 256, 0, st>>>(rows, cols, src, lds, dst, ldd, plane, nslice);
  return cudaGetLastError();
}

cudaError_t launch_jac_init_bf16(int C, int d_y, int w, const float *WL, const float *der,
                                 int ldd, __nv_bfloat16 *P, int ldp, size_t plane, int nslice,
                                 cudaStream_t st) {
  const size_t items = (size_t)C * d_y * ((w + 7) / 8);  // 8 columns per thread
  if (items >= 0xffffffffull - 152ull * 16 * 256) return cudaErrorInvalidValue;
  const int grid = (int)std::min<size_t>((items + 255) / 256, 152 * 16);
  k_jac_init_bf16<<<grid > 0 ? grid : 1, 256, 0, st>>>(C, d_y, w, WL, der, ldd, P, ldp, plane,
                                                       nslice);
  return cudaGetLastError();
}

}  // namespace dino
