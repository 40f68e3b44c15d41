// Internal interfaces between the host runtime (host.cpp) and the kernels.
// Every launcher issues exactly one kernel on the given stream.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstddef>
#include <cmath>
#include <cstdint>

namespace dino {

// Largest reduced dimension whose packed FP64 Cholesky factor the per-chain
// kernels keep in shared memory (r (r+1)/2 doubles plus work vectors); larger
// r works on a global (L2-resident) per-chain workspace.
constexpr int kMaxRSmem = 208;
constexpr int kMaxR = 1024;                 // largest reduced dimension supported
// Largest d_y of the Woodbury path (d_y < r): its (d_y+1)-square factor and
// vectors then fit one CTA's shared memory for every r <= kMaxR, in both
// precisions.  Larger d_y takes the r-sized path.
constexpr int kMaxWbDy = 192;
constexpr size_t kSmemLimit = 227 * 1024;   // opt-in shared memory per CTA

// Philox streams (counter word 3): reduced noise, accept uniform, complement
// prior draw, initial prior draw, observation-space noise of the
// perturbation map (d_y < r).
constexpr uint32_t STREAM_XI_ID = 0, STREAM_U_ID = 1, STREAM_Z_ID = 2, STREAM_INIT_ID = 3,
                   STREAM_XI2_ID = 4, STREAM_U2_ID = 5;

inline __host__ __device__ size_t tri_size(int r) { return (size_t)r * (r + 1) / 2; }
// Per-chain factor slot in global memory: the packed lower Cholesky factor
// of I + H bordered by the row (m_r + g)^T (r + 1 rows; row r holds
// L^-1 (m_r + g)), then p = L^T m_r (r doubles); rounded up to an even number
// of doubles so that every slot starts on 16 bytes.
inline __host__ __device__ size_t slot_stride(int r) {
  return (tri_size(r + 1) + r + 1) & ~(size_t)1;
}
// Per-chain factor slot of the Woodbury path (d_y < r): the packed factor of
// I + K K^T bordered by u^T (d_y + 1 rows), the d_y + 1 inverse pivots, u, v
// and the scalar t1, rounded up to an even number of doubles.
inline __host__ __device__ size_t wb_slot_stride(int d_y) {
  return (tri_size(d_y + 1) + (d_y + 1) + 2 * (size_t)d_y + 1 + 1) & ~(size_t)1;
}

// ---- per-chain reduced-space kernels (FP64) -----------------------------
struct ReducedArgs {
  int C = 0, r = 0, d_y = 0;
  double s = 0, dt = 0, noise_var = 1;
  // constants of every chain, set by derive() before a launch (the kernels
  // would otherwise each take FP64 divisions and square roots):
  // 1 / noise_var, its square root, c_s = sqrt(1 - s^2), 1 / c_s, sqrt(dt)
  double inv_nv = 1, inv_sigma = 1, cs = 1, inv_cs = 1, sqrt_dt = 0;
  void derive() {
    inv_nv = 1.0 / noise_var;
    inv_sigma = std::sqrt(inv_nv);
    cs = std::sqrt(1.0 - s * s);
    inv_cs = 1.0 / cs;
    sqrt_dt = std::sqrt(dt);
  }
  uint64_t seed = 0, id_base = 0;
  uint32_t step = 0;
  // chain state
  double *mr = nullptr, *g = nullptr, *phi = nullptr, *hld = nullptr, *L = nullptr;
  // proposal (written by propose, read by geometry)
  double *b = nullptr, *mu = nullptr, *lq_fwd = nullptr;
  // the factor slot is double-buffered: slot cur[c] holds the chain's
  // current one; an accepted proposal's slot is written into the other and
  // cur[c] flips.  L_slot = elements between the slots (C * slot_stride(r)).
  int *cur = nullptr;
  size_t L_slot = 0;
  // Woodbury path: J at each chain's current point (C x d_y x r, FP64 or FP32)
  void *Js = nullptr;
  // surrogate output at b: J (C x d_y x r) and f (C x d_y), FP64 or FP32
  const void *J = nullptr;
  const void *f = nullptr;
  // Woodbury path, FP32 J: the Gram matrices J J^T formed beforehand (C x
  // d_y x ldg), or nullptr to form them in the geometry kernel
  const float *G = nullptr;
  int ldg = 0;
  // Woodbury path with the tensor-core Gram: the proposal b and the state m_r
  // as double-float pairs (C x r), from which a warp-per-row kernel forms K b
  // and K a (C x d_y, already / sigma) into Kb_pre, Ka_pre right after the
  // Jacobian; nullptr to form them in the geometry kernel
  float2 *b_df = nullptr, *a_df = nullptr;
  const double *Kb_pre = nullptr, *Ka_pre = nullptr;
  int jf_f32 = 0;
  const double *y = nullptr;
  // accept outputs
  double *coef = nullptr, *log_rho = nullptr, *log_u = nullptr;
  int *acc = nullptr;
  unsigned long long *acc_count = nullptr;
  unsigned long long *counters = nullptr;  // [0] accepts, [1] nan rejects
  double *sum_alpha = nullptr;
  int *err = nullptr;  // set (bit 4) when a bounded device wait gives up
  // caller-supplied noise of this transition (nullptr: Philox): reduced
  // normals (C x r), observation-space normals of the perturbation map
  // (C x d_y) and the log of the accept uniform (C)
  const double *ext_xi = nullptr, *ext_xi2 = nullptr, *ext_log_u = nullptr;
  // delayed acceptance: the first stage only stages an accepted proposal
  // (its factor in the spare slot, Phi, half log det and, r-sized path, g in
  // the *_st buffers); the second stage (launch_da_decide) commits it
  int da = 0;
  double *phi_st = nullptr, *hld_st = nullptr, *g_st = nullptr;
  // tensor-core path: the proposal as bf16 slice planes (row pitch b_ld,
  // plane pitch b_plane elements); nullptr when unused
  __nv_bfloat16 *b_bf16 = nullptr;
  int b_slices = 0, b_ld = 0;
  size_t b_plane = 0;
};

// Woodbury path on the tensor path: Kb[row] = (sum_k J[row, k] b[c, k]) *
// kscale and Ka likewise with a (a may be nullptr), c = row / d_y, over the
// C d_y rows of the FP32 J (row pitch r); b, a as double-float pairs (C x r).
cudaError_t launch_rowprod(int rows, int r, int d_y, const float *J, const float2 *b,
                           const float2 *a, double kscale, double *Kb, double *Ka,
                           cudaStream_t st);
// dst1[i] = dst2[i] = src[i] as a double-float pair (either dst may be nullptr)
cudaError_t launch_to_df(size_t n, const double *src, float2 *dst1, float2 *dst2,
                         cudaStream_t st);
bool uses_global_factor(int r, int d_y);
size_t propose_smem_bytes(int r);
size_t geometry_smem_bytes(int r, int d_y, int jf_f32);
cudaError_t launch_propose(const ReducedArgs &a, cudaStream_t st);
// mode 0: initialise the state at b; mode 1: geometry at the proposal b,
// log-acceptance, accept test and state update
cudaError_t launch_geometry(const ReducedArgs &a, int mode, cudaStream_t st);
// The Woodbury path (d_y < r): the same two steps with the d_y x d_y factor
// of I + K K^T (K = J / sigma) and the perturbation noise map.
size_t wb_smem_bytes(int r, int d_y, int jf_f32);
cudaError_t launch_wb_propose(const ReducedArgs &a, cudaStream_t st);
cudaError_t launch_wb_geometry(const ReducedArgs &a, int mode, cudaStream_t st);
// The eigen map (d_y < r, d_y <= kMaxEigDy): the same two steps with the
// eigendecomposition of I + K K^T and the noise (I + H)^-1/2 xi.
constexpr int kMaxEigDy = 64;
size_t eig_slot_stride(int d_y);
size_t eig_smem_bytes(int r, int d_y);
cudaError_t launch_eig_propose(const ReducedArgs &a, cudaStream_t st);
cudaError_t launch_eig_geometry(const ReducedArgs &a, int mode, cudaStream_t st);

// ---- SIMT GEMMs: out = epilogue(A B^T), A: M x K (lda), B: N x K (ldb) ----
template <typename T>
cudaError_t gemm_store(int M, int N, int K, const T *A, int lda, const T *B, int ldb, T *out,
                       int ldo, cudaStream_t st);
// out = act(acc + bias[col]); der = act'(acc + bias[col])   (der may be null)
template <typename T>
cudaError_t gemm_bias_act(int M, int N, int K, const T *A, int lda, const T *B, int ldb,
                          const T *bias, int act, T *out, T *der, int ldo, cudaStream_t st);
// out = acc * scale[(row / group) * lds + col]
template <typename T>
cudaError_t gemm_scale_group(int M, int N, int K, const T *A, int lda, const T *B, int ldb,
                             const T *scale, int lds, int group, T *out, int ldo,
                             cudaStream_t st);
// complement coefficient: out[row, col] = coef[row * ldc + col] - c * acc.
template <typename T>
cudaError_t gemm_coef(int M, int N, int K, const T *A, int lda, const T *B, int ldb,
                      const double *coef, int ldc, double c, T *out, int ldo, cudaStream_t st);
// field update: if acc_flag[row]: m[row, col] = s m + c Mf[row, col] + acc
template <typename T>
cudaError_t gemm_field(int M, int N, int K, const T *A, int lda, const T *B, int ldb,
                       const int *acc_flag, double s, double c, T *m, const T *Mf, int ldm,
                       cudaStream_t st);

// ---- elementwise / per-chain helpers -------------------------------------
// Shared memory of the prior draw of one chain on an n x n grid (elements of `elem` bytes).
size_t prior_draw_smem_bytes(int n, int elem);
// Prior draw from the full KLE: out[c] = S^T (sqrt(Lambda) .* Z_c) S,
// Z_c from Philox stream `stream` at `step` for chain id_base + c.  With `ms`
// (FP32 only) the draw is also written as ms_slices bf16 slice planes
// (row pitch ldms, plane stride ms_plane) for the tensor-core projections.
// With ext_z (C x N doubles, nullptr for Philox) the normals Z_c are the
// caller's, indexed like the Philox ones.  With `only`, chains c with
// only[c] == 0 draw nothing (their rows keep earlier contents).
template <typename T>
cudaError_t launch_prior_draw(int C, int n, const T *sqrtlam, const T *S, uint64_t seed,
                              uint64_t id_base, uint32_t stream, uint32_t step, T *out,
                              int ldo, cudaStream_t st,
                              __nv_bfloat16 *ms = nullptr, int ldms = 0, size_t ms_plane = 0,
                              int ms_slices = 0, const double *ext_z = nullptr,
                              const int *only = nullptr);
// P[(c d_y + i) w + k] = WL[i w + k] * der[c ldd + k]
template <typename T>
cudaError_t launch_jac_init(int C, int d_y, int w, const T *WL, const T *der, int ldd, T *P,
                            cudaStream_t st);
// out[c] = W (broadcast of a d_y x r matrix to every chain)
template <typename T>
cudaError_t launch_broadcast(int C, size_t n, const T *src, T *out, cudaStream_t st);
cudaError_t launch_f64_to_f32(size_t n, const double *src, float *dst, cudaStream_t st);
// dst[c][i][j] = src[c][j][i]: C blocks of a x b (src) into b x a (dst), FP64 or FP32 (f32)
cudaError_t launch_batched_transpose(int C, int a, int b, const void *src, int f32, void *dst,
                                     cudaStream_t st);
// dst[i] = src[i]; src may be pageable host memory on a device that reads it
// coherently (cudaDevAttrPageableMemoryAccess)
cudaError_t launch_copy_f64(size_t n, const double *src, double *dst, cudaStream_t st);

// ---- delayed acceptance: the true-model stage (Algorithm 1) -------------
// xt = s mt + cs EtM + EtDc (C x r_t; EtM, EtDc FP64 or, with in_f32, FP32;
// either may be nullptr for 0), and with xb its nslice bf16 slice planes
// (row pitch ldx, plane stride plane).
cudaError_t launch_da_assemble(int C, int r_t, double s, double cs, const double *mt,
                               const void *EtM, const void *EtDc, int in_f32, double *xt,
                               __nv_bfloat16 *xb, int ldx, size_t plane, int nslice,
                               cudaStream_t st);
// phi_t[c] = |ft[c] - y|^2 / (2 noise_var) (ft FP64, or FP32 with f32)
cudaError_t launch_da_misfit(int C, int d_y, const void *ft, int f32, const double *y,
                             double noise_var, double *phi_t, cudaStream_t st);
struct DaArgs {
  int C = 0, r = 0, d_y = 0, r_t = 0;
  double noise_var = 1;
  uint64_t seed = 0, id_base = 0;
  uint32_t step = 0;
  int *acc = nullptr;                    // first-stage flags in, final flags out
  int *stage1 = nullptr;                 // copy of the first-stage flags
  double *mt = nullptr, *phi_t = nullptr;  // E_t m and Phi(m) of the chain state
  const double *xt = nullptr;            // E_t m^dagger
  const void *ft = nullptr;              // true map at m^dagger (C x d_y)
  int ft_f32 = 0;
  const double *y = nullptr;
  double *mr = nullptr, *phi = nullptr, *hld = nullptr, *g = nullptr;
  const double *b = nullptr, *phi_st = nullptr, *hld_st = nullptr, *g_st = nullptr;
  int *cur = nullptr;
  const void *J = nullptr;               // Woodbury path: J at b, copied into Js
  void *Js = nullptr;
  int j_f32 = 0;
  const float2 *b_df = nullptr;          // BF16 Woodbury path: b -> a_df
  float2 *a_df = nullptr;
  unsigned long long *acc_count = nullptr, *counters = nullptr;
  double *log_rho2 = nullptr, *log_u2 = nullptr;
  const double *ext_log_u2 = nullptr;
};
// Phi(m^dagger), log rho^(2) (eq:da_dino_trr_2), the second accept test and
// the commit of a chain that passes both stages; CTA per chain.
cudaError_t launch_da_decide(const DaArgs &a, cudaStream_t st);

// FP32 fused multiply-add throughput of the device: runs a kernel of
// independent FMA chains on every SM and returns its time and its flops
// (2 per FMA); the best of a few launches after a warm-up.
cudaError_t measure_fma_peak(cudaStream_t st, float *ms, double *flops);

// ---- chain diagnostics (Sec. 6.2) ----------------------------------------
// traj[(i n_c + k) max_s + j] = src[k ld_src + i] for k < n_c, i < d
cudaError_t launch_diag_record(int n_c, int d, const void *src, int src_f32, int ld_src,
                               double *traj, int max_s, int j, cudaStream_t st);
// per degree of freedom: chain means (d x n_c), ESS fraction, sum of squared jumps
cudaError_t launch_diag_ess(int d, int n_c, int n_s, const double *traj, int max_s, double *means,
                            double *ess, double *sqjump, cudaStream_t st);
// centred samples Xc (d x n_c n_s) and centred chain means Mc (d x n_c)
cudaError_t launch_diag_center(int d, int n_c, int n_s, const double *traj, int max_s,
                               const double *means, double *Xc, double *Mc, cudaStream_t st);
cudaError_t launch_diag_wv(int d, int n_c, int n_s, const double *Wr, const double *Br, double *W,
                           double *V, cudaStream_t st);
// one-sided Jacobi on the d columns of G (in place); Q (optional) gets the
// accumulated rotations, sig the column norms, *sweeps the sweeps taken
cudaError_t launch_jacobi(int d, double *G, double *Q, double *sig, int *sweeps, cudaStream_t st);
cudaError_t launch_sym_sqrt(int d, const double *Q, const double *lam, double *S, cudaStream_t st);
cudaError_t launch_small_mm(int d, const double *A, const double *B, double *C, cudaStream_t st);
cudaError_t launch_mpsrf_final(int d, const double *W, const double *V, const double *sig,
                               double *out, cudaStream_t st);
// out (n x r) = standard normals of Philox (seed, stream, step 0, chain i)
cudaError_t launch_normals(uint64_t seed, uint32_t stream, int n, int r, double *out,
                           cudaStream_t st);
// dst (cols x rows, FP64) = scale * src^T, src rows x cols (row pitch ld, FP64 or FP32)
cudaError_t launch_transpose(int rows, int cols, const void *src, int src_f32, int ld,
                             double scale, double *dst, cudaStream_t st);
constexpr uint32_t STREAM_DIS_ID = 6;  // Monte Carlo draws of the surrogate DIS

// ---- tcgen05 BF16 GEMM (sm_103a) -----------------------------------------
// Operands are bf16 "slice planes": X ~= sum_s X_s, plane s at X + s * plane.
// D = sum over slice pairs (i, j), i + j < nslice, of A_i B_j^T, FP32 accum.
// A: M x K (row pitch lda elements), B: N x K (row pitch ldb).
enum TcEpi : int {
  TC_EPI_STORE_F32 = 0,   // outf[row, col] = acc (and, with out_bf, its slices)
  TC_EPI_BIAS_F32 = 1,    // outf = acc + bias[col]
  TC_EPI_BIAS_ACT = 2,    // z = acc + bias; out slices = act(z); der = act'(z) (fp32)
  TC_EPI_SCALE_GROUP = 3,  // out slices = acc * scale[(row/group)*lds + col]
  TC_EPI_COEF = 4,         // out slices = coef[row*ldc + col] - cs * acc (coef FP64)
  TC_EPI_FIELD_T = 5       // rows are field nodes, columns chains: where acc[col],
                           // m[col*ldm + row] = (s m + cs Mf)[same] + acc
};
struct TcGemmArgs {
  int M = 0, N = 0, K = 0;
  const __nv_bfloat16 *A = nullptr;
  int lda = 0;
  size_t a_plane = 0;
  const __nv_bfloat16 *B = nullptr;
  int ldb = 0;
  size_t b_plane = 0;
  int nslice = 1;
  int epi = TC_EPI_STORE_F32;
  float *outf = nullptr;
  int ldo = 0;
  const float *bias = nullptr;
  int act = 0;
  __nv_bfloat16 *out_bf = nullptr;  // slice planes of the output
  int ldob = 0;                      // their row pitch with TC_EPI_STORE_F32 (else ldo)
  size_t out_plane = 0;
  int out_slices = 1;
  float *der = nullptr;
  const float *scale = nullptr;
  int lds = 0, group = 1;
  // TC_EPI_COEF with few tiles: split K, FP32 partials in ws (ws_floats)
  float *ws = nullptr;
  size_t ws_floats = 0;
  const double *coef = nullptr;  // TC_EPI_COEF
  int ldc = 0;
  double cs = 0.0, sc = 0.0;     // TC_EPI_COEF (cs), TC_EPI_FIELD_T (sc, cs)
  const int *acc = nullptr;      // TC_EPI_FIELD_T
  float *m = nullptr;
  const float *Mf = nullptr;
  int ldm = 0;
};
cudaError_t launch_tc_gemm(const TcGemmArgs &a, cudaStream_t st);
// Per-group Gram matrices on the tensor cores: for c < C, with J_c the g x K
// block of rows c g .. c g + g - 1 of the stacked bf16 slice planes J (row
// pitch ldj, plane stride plane, nslice planes; pairs i + j < nslice),
// out[(c g + i) ldo + j] = (J_c J_c^T)[i, j] in FP32 for i, j < g (g <= 128).
cudaError_t launch_tc_gram(int C, int g, int K, const __nv_bfloat16 *J, int ldj, size_t plane,
                           int nslice, float *out, int ldo, cudaStream_t st);
// Split FP32/FP64 values into bf16 slice planes (x ~= sum_s slice_s).
cudaError_t launch_split_bf16_f64(int rows, int cols, const double *src, int lds,
                                  __nv_bfloat16 *dst, int ldd, size_t plane, int nslice,
                                  cudaStream_t st);
// Jacobian start on the tensor path: P = W_L .* der (both fp32) as bf16 slices
cudaError_t launch_jac_init_bf16(int C, int d_y, int w, const float *WL, const float *der,
                                 int ldd, __nv_bfloat16 *P, int ldp, size_t plane, int nslice,
                                 cudaStream_t st);

}  // namespace dino
