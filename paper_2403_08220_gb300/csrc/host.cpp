// Host runtime behind the C ABI in include/dino.h: contexts, surrogates,
// chain pools and the per-step launch sequence.  Setup work (building the
// reduced basis, uploading weights) runs here once per surrogate; every
// per-step operation is a CUDA kernel launched on the context's stream.
#include "../../include/dino.h"

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <thread>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "dino_internal.h"

namespace dino {

struct Error {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  throw Error{code, buf};
}

#define CK(expr)                                                                         \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess) fail(DINO_ECUDA, "%s: %s", #expr, cudaGetErrorString(_e)); \
  } while (0)

static inline int pad8(int x) { return (x + 7) & ~7; }
// bf16 slices of the operands of the tensor-core complement projections and
// of the Jacobian rows that feed the tensor-core Gram matrices
constexpr int kFieldSlices = 3;
constexpr int kGramSlices = 3;

// One device allocation carved into aligned sub-buffers.
struct Arena {
  char *base = nullptr;
  size_t bytes = 0, off = 0;
  size_t reserve(size_t n) {
    off = (off + 255) & ~(size_t)255;
    const size_t at = off;
    off += n;
    return at;
  }
};

struct Surrogate;
struct Pool;
struct Server;
struct Diag;

}  // namespace dino

struct dino_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0, used = 0;
  unsigned flags = 0;
  std::recursive_mutex mu;
  std::string err;
  int next_id = 1;
  std::map<int, std::unique_ptr<dino::Surrogate>> surrogates;
  std::map<int, std::unique_ptr<dino::Pool>> pools;
  uint64_t launches = 0;
  struct KTime {
    double ms = 0;
    uint64_t n = 0;
  };
  std::map<std::string, KTime> ktimes;
  struct Pending {
    std::string name;
    cudaEvent_t e0, e1;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  std::unique_ptr<dino::Server> server;
  std::map<int, std::unique_ptr<dino::Diag>> diags;
  // streams that dino_chains_step_many spreads pools over (created on first use)
  std::vector<cudaStream_t> aux_streams;
  // the device reads pageable host memory coherently (Grace: over NVLink-C2C)
  bool pageable_access = false;
};

namespace dino {

// ---------------------------------------------------------------------------
// device memory accounting
void *dev_alloc(dino_ctx *ctx, size_t bytes) {
  if (bytes == 0) return nullptr;
  if (ctx->used + bytes > ctx->budget)
    fail(DINO_ENOMEM, "HBM budget exceeded: need %zu more bytes, %zu of %zu used", bytes,
         ctx->used, ctx->budget);
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(DINO_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  ctx->used += bytes;
  return p;
}

void dev_free(dino_ctx *ctx, void *p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  ctx->used -= std::min(ctx->used, bytes);
}

// Stream-ordered allocation for pools that come and go while other pools run
// (serving): no device-wide synchronisation on free.
void *dev_alloc_async(dino_ctx *ctx, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return nullptr;
  if (ctx->used + bytes > ctx->budget)
    fail(DINO_ENOMEM, "HBM budget exceeded: need %zu more bytes, %zu of %zu used", bytes,
         ctx->used, ctx->budget);
  void *p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(DINO_ENOMEM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
  }
  ctx->used += bytes;
  return p;
}

void dev_free_async(dino_ctx *ctx, void *p, size_t bytes, cudaStream_t st) {
  if (!p) return;
  cudaFreeAsync(p, st);
  ctx->used -= std::min(ctx->used, bytes);
}

template <typename T>
T *upload(dino_ctx *ctx, const T *host, size_t n) {
  T *d = (T *)dev_alloc(ctx, n * sizeof(T));
  CK(cudaMemcpyAsync(d, host, n * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
  return d;
}

// ---------------------------------------------------------------------------
// kernel launch bookkeeping (count + optional CUDA-event timing)
template <class F>
void launch(dino_ctx *ctx, cudaStream_t st, const char *name, F &&fn) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const bool timing = (ctx->flags & DINO_FLAG_TIMING) != 0;
  if (timing) {
    for (cudaEvent_t *e : {&e0, &e1}) {
      if (!ctx->event_pool.empty()) {
        *e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
      } else {
        CK(cudaEventCreate(e));
      }
    }
    CK(cudaEventRecord(e0, st));
  }
  cudaError_t err = fn();
  ctx->launches += 1;
  if (err != cudaSuccess) fail(DINO_ECUDA, "kernel %s: %s", name, cudaGetErrorString(err));
  if (timing) {
    CK(cudaEventRecord(e1, st));
    ctx->pending.push_back({name, e0, e1});
  }
}

void collect_times(dino_ctx *ctx) {
  if (ctx->pending.empty()) return;
  for (auto &p : ctx->pending) {
    float ms = 0;
    CK(cudaEventSynchronize(p.e1));
    CK(cudaEventElapsedTime(&ms, p.e0, p.e1));
    auto &kt = ctx->ktimes[p.name];
    kt.ms += ms;
    kt.n += 1;
    ctx->event_pool.push_back(p.e0);
    ctx->event_pool.push_back(p.e1);
  }
  ctx->pending.clear();
}

// ---------------------------------------------------------------------------
// reduced bases (setup, host)

struct Modes {
  std::vector<int> kx, ky;
  std::vector<double> kappa;
};

static std::vector<double> lap1d_eigs(int n) {
  const double h = 1.0 / (n + 1);
  std::vector<double> s(n);
  for (int k = 1; k <= n; ++k) {
    const double t = std::sin(k * M_PI * h / 2.0);
    s[k - 1] = 4.0 / (h * h) * t * t;
  }
  return s;
}

// Sine matrix S[k-1][i] = sqrt(2/(n+1)) sin(k (i+1) pi/(n+1)) (symmetric, orthogonal).
static std::vector<double> sine_matrix(int n) {
  std::vector<double> S((size_t)n * n);
  const double c = std::sqrt(2.0 / (n + 1));
  for (int k = 1; k <= n; ++k)
    for (int i = 1; i <= n; ++i) S[(size_t)(k - 1) * n + (i - 1)] = c * std::sin(k * i * M_PI / (n + 1));
  return S;
}

// KLE order: increasing kappa (decreasing lambda), ties by smaller kx.
static Modes kle_modes(int n) {
  const auto s = lap1d_eigs(n);
  std::vector<int> idx((size_t)n * n);
  std::iota(idx.begin(), idx.end(), 0);
  auto kap = [&](int q) { return s[q % n] + s[q / n]; };  // q = (kx-1) + n (ky-1)
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
    const double ka = kap(a), kb = kap(b);
    if (ka != kb) return ka < kb;
    return (a % n) < (b % n);
  });
  Modes m;
  for (int q : idx) {
    m.kx.push_back(q % n + 1);
    m.ky.push_back(q / n + 1);
    m.kappa.push_back(kap(q));
  }
  return m;
}

static void build_kle(int n, double gamma, double delta, int r, std::vector<double> &E,
                      std::vector<double> &D) {
  const int N = n * n;
  const auto S = sine_matrix(n);
  const Modes md = kle_modes(n);
  E.assign((size_t)r * N, 0.0);
  D.assign((size_t)N * r, 0.0);
  for (int j = 0; j < r; ++j) {
    const double lam_sqrt = 1.0 / (delta + gamma * md.kappa[j]);  // sqrt(lambda)
    const double *vx = &S[(size_t)(md.kx[j] - 1) * n];
    const double *vy = &S[(size_t)(md.ky[j] - 1) * n];
    for (int jj = 0; jj < n; ++jj)
      for (int i = 0; i < n; ++i) {
        const double eta = vx[i] * vy[jj];
        const int p = i + n * jj;
        E[(size_t)j * N + p] = eta / lam_sqrt;
        D[(size_t)p * r + j] = lam_sqrt * eta;
      }
  }
}

// Thin Householder QR of G (N x r, row-major) -> Q (N x r, row-major) with
// positive diag(R).  Works on a column-major copy so every reflector
// application streams contiguous columns.
static std::vector<double> thin_q(const double *G, int N, int r) {
  std::vector<double> A((size_t)N * r);  // column j at A[j*N ...]
  for (int p = 0; p < N; ++p)
    for (int j = 0; j < r; ++j) A[(size_t)j * N + p] = G[(size_t)p * r + j];
  std::vector<double> beta(r, 0.0), rdiag(r, 0.0);
  std::vector<double> vs((size_t)r * N, 0.0);  // reflector j at vs[j*N ...], zero above j
  for (int j = 0; j < r; ++j) {
    double *a = &A[(size_t)j * N];
    double nrm = 0.0;
    for (int p = j; p < N; ++p) nrm += a[p] * a[p];
    nrm = std::sqrt(nrm);
    const double alpha = a[j] >= 0 ? -nrm : nrm;  // R_jj = alpha
    double *v = &vs[(size_t)j * N];
    v[j] = a[j] - alpha;
    for (int p = j + 1; p < N; ++p) v[p] = a[p];
    double vv = 0.0;
    for (int p = j; p < N; ++p) vv += v[p] * v[p];
    beta[j] = vv > 0 ? 2.0 / vv : 0.0;
    rdiag[j] = alpha;
    for (int k = j; k < r; ++k) {
      double *ak = &A[(size_t)k * N];
      double d = 0.0;
      for (int p = j; p < N; ++p) d += v[p] * ak[p];
      d *= beta[j];
      for (int p = j; p < N; ++p) ak[p] -= d * v[p];
    }
  }
  // Q = H_0 H_1 ... H_{r-1} [I_r; 0], built column by column
  std::vector<double> Qc((size_t)r * N, 0.0);
  for (int k = 0; k < r; ++k) {
    double *q = &Qc[(size_t)k * N];
    q[k] = 1.0;
    for (int j = std::min(k, r - 1); j >= 0; --j) {
      const double *v = &vs[(size_t)j * N];
      double d = 0.0;
      for (int p = j; p < N; ++p) d += v[p] * q[p];
      d *= beta[j];
      for (int p = j; p < N; ++p) q[p] -= d * v[p];
    }
  }
  std::vector<double> Q((size_t)N * r);
  for (int k = 0; k < r; ++k) {
    const double sg = rdiag[k] < 0 ? -1.0 : 1.0;
    for (int p = 0; p < N; ++p) Q[(size_t)p * r + k] = sg * Qc[(size_t)k * N + p];
  }
  return Q;
}

// y = A^-1 x for one field (n x n) through the sine transform: A^-1 = S diag(1/(delta+gamma kappa)) S.
static void apply_Ainv(int n, double gamma, double delta, const std::vector<double> &S,
                       const std::vector<double> &s1, const double *x, double *y,
                       std::vector<double> &t1, std::vector<double> &t2) {
  // t1 = S X  (X[j][i] = x[i + n j]); t2 = t1 S = S X S (spectral [ky][kx])
  for (int a = 0; a < n; ++a)
    for (int i = 0; i < n; ++i) {
      double acc = 0;
      for (int j = 0; j < n; ++j) acc += S[(size_t)a * n + j] * x[i + n * j];
      t1[(size_t)a * n + i] = acc;
    }
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      double acc = 0;
      for (int i = 0; i < n; ++i) acc += t1[(size_t)a * n + i] * S[(size_t)i * n + b];
      t2[(size_t)a * n + b] = acc / (delta + gamma * (s1[a] + s1[b]));
    }
  for (int a = 0; a < n; ++a)
    for (int i = 0; i < n; ++i) {
      double acc = 0;
      for (int b = 0; b < n; ++b) acc += t2[(size_t)a * n + b] * S[(size_t)b * n + i];
      t1[(size_t)a * n + i] = acc;
    }
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      double acc = 0;
      for (int a = 0; a < n; ++a) acc += S[(size_t)a * n + j] * t1[(size_t)a * n + i];
      y[i + n * j] = acc;
    }
}

static void build_dis(int n, double gamma, double delta, int r, const double *G,
                      std::vector<double> &E, std::vector<double> &D) {
  const int N = n * n;
  const double h2 = 1.0 / ((n + 1.0) * (n + 1.0));
  const auto Q = thin_q(G, N, r);
  const auto S = sine_matrix(n);
  const auto s1 = lap1d_eigs(n);
  E.assign((size_t)r * N, 0.0);
  D.assign((size_t)N * r, 0.0);
  std::vector<double> q(N), y(N), t1((size_t)n * n), t2((size_t)n * n);
  for (int j = 0; j < r; ++j) {
    for (int p = 0; p < N; ++p) q[p] = Q[(size_t)p * r + j];
    apply_Ainv(n, gamma, delta, S, s1, q.data(), y.data(), t1, t2);
    for (int p = 0; p < N; ++p) D[(size_t)p * r + j] = y[p];
    for (int jj = 0; jj < n; ++jj)
      for (int i = 0; i < n; ++i) {
        const int p = i + n * jj;
        double lap = -4.0 * q[p];
        if (i > 0) lap += q[p - 1];
        if (i < n - 1) lap += q[p + 1];
        if (jj > 0) lap += q[p - n];
        if (jj < n - 1) lap += q[p + n];
        E[(size_t)j * N + p] = delta * q[p] - gamma * lap / h2;  // (A q)_p
      }
  }
}

static double max_ed_error(const std::vector<double> &E, const std::vector<double> &D, int r,
                           int N) {
  double worst = 0.0;
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < r; ++j) {
      double acc = 0.0;
      for (int p = 0; p < N; ++p) acc += E[(size_t)i * N + p] * D[(size_t)p * r + j];
      worst = std::max(worst, std::fabs(acc - (i == j ? 1.0 : 0.0)));
    }
  return worst;
}

// ---------------------------------------------------------------------------
// surrogate

struct Surrogate {
  int id = 0;
  int n_grid = 0, N = 0;
  double gamma = 0, delta = 0;
  int r = 0, d_y = 0, L = 0, act = 0, precision = 0, fwd_slices = 1, jac_slices = 1;
  std::vector<int> widths;
  std::vector<std::vector<double>> W, b;
  std::vector<double> E, D, y;
  double noise_var = 0;
  bool has_data = false;
  // d_y < r: chains use the Woodbury path (d_y x d_y factor, perturbation noise map)
  bool wb = false;
  // Woodbury path on the tensor path with d_y <= 128 and a hidden layer: the
  // d_y x d_y Gram matrices J J^T come from the tensor cores
  bool tc_gram = false;
  // eigen map (d_y < r): I + K K^T eigendecomposed instead of factored; the
  // pools keep the perturbation path's J state (wb is set too)
  bool eig = false;
  // Jacobian order: forward mode (push the r input directions) when r < d_y
  // and it takes fewer flops than reverse mode (pull the d_y outputs), the
  // min{d_y, r} rule of Sec. 4.3; the tensor path then keeps FP32 W_0^T and
  // jac_slices bf16 planes of W_1 .. W_{L-1} (pitch ldWj)
  bool jac_fwd = false;
  float *fW0T = nullptr;
  std::vector<__nv_bfloat16 *> bWj;
  std::vector<int> ldWj;
  std::vector<size_t> plWj;
  int pools = 0;
  // device
  std::vector<std::pair<void *, size_t>> allocs;
  double *dE = nullptr, *dD = nullptr, *dS = nullptr, *dSqrtLam = nullptr, *dy = nullptr;
  float *fS = nullptr, *fSqrtLam = nullptr;  // prior draw on the tensor path
  // tensor path: bf16 slice planes of E (r x N, pitch ldE) and D (N x r, pitch ldD)
  // for the complement projections
  __nv_bfloat16 *bE = nullptr, *bD = nullptr;
  int ldE = 0, ldD = 0;
  size_t plE = 0, plD = 0;
  std::vector<double *> dW, dWT, db;
  std::vector<float *> fb, fW;
  std::vector<__nv_bfloat16 *> bW, bWT;
  std::vector<int> ldW, ldWT;
  std::vector<size_t> plW, plWT;
  int widest = 0;  // max hidden/output width used by the Jacobian buffers
  // delayed acceptance (Algorithm 1's second stage): the true map
  // G(m) = f_t(E_t m), an MLP on an r_t-dimensional encoding of the field
  struct TrueModel {
    bool on = false;
    int r_t = 0, L = 0, act = 0, widest = 0;
    std::vector<int> widths;
    std::vector<std::pair<void *, size_t>> allocs;
    double *dEt = nullptr, *dEtD = nullptr;  // E_t (r_t x N), E_t D (r_t x r)
    std::vector<double *> dW, db;
    // tensor path: three bf16 slices of E_t (r_t x ldE), E_t D (r_t x ldD)
    // and of each W_l (pitch ldW[l]); FP32 biases
    __nv_bfloat16 *bEt = nullptr, *bEtD = nullptr;
    size_t plEt = 0, plEtD = 0;
    std::vector<__nv_bfloat16 *> bW;
    std::vector<int> ldW;
    std::vector<size_t> plW;
    std::vector<float *> fb;
  } tm;
};

// bf16 slices of the true model's operands (FP32-level, like the surrogate's forward)
constexpr int kTrueSlices = 3;

template <typename T>
static T *sur_alloc(dino_ctx *ctx, Surrogate *s, size_t n) {
  T *p = (T *)dev_alloc(ctx, n * sizeof(T));
  s->allocs.push_back({p, n * sizeof(T)});
  return p;
}

template <typename T>
static T *sur_upload(dino_ctx *ctx, Surrogate *s, const T *host, size_t n) {
  T *p = sur_alloc<T>(ctx, s, n);
  CK(cudaMemcpyAsync(p, host, n * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
  return p;
}

static std::vector<float> to_f32(const std::vector<double> &v) {
  return std::vector<float>(v.begin(), v.end());
}

// bf16 slice planes of a rows x cols matrix with row pitch ld: plane s holds
// the s-th term of x ~= sum_s x_s, each the bf16 rounding of what remains.
static std::vector<__nv_bfloat16> split_planes(const std::vector<double> &x, int rows, int cols,
                                               int ld, int nslice, size_t &plane) {
  plane = (size_t)rows * ld;
  std::vector<__nv_bfloat16> out(plane * nslice, __float2bfloat16(0.0f));
  for (int i = 0; i < rows; ++i)
    for (int j = 0; j < cols; ++j) {
      float rem = (float)x[(size_t)i * cols + j];
      for (int s = 0; s < nslice; ++s) {
        const __nv_bfloat16 h = __float2bfloat16_rn(rem);
        out[s * plane + (size_t)i * ld + j] = h;
        rem -= __bfloat162float(h);
      }
    }
  return out;
}

static void upload_data(dino_ctx *ctx, Surrogate *s) {
  if (!s->dy) s->dy = sur_alloc<double>(ctx, s, std::max(1, s->d_y));
  CK(cudaMemcpyAsync(s->dy, s->y.data(), s->d_y * sizeof(double), cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
}

static void free_true_model(dino_ctx *ctx, Surrogate *s) {
  cudaStreamSynchronize(ctx->stream);
  for (auto &a : s->tm.allocs) dev_free(ctx, a.first, a.second);
  s->tm = Surrogate::TrueModel{};
}

static void free_surrogate(dino_ctx *ctx, Surrogate *s) {
  cudaStreamSynchronize(ctx->stream);
  for (auto &a : s->allocs) dev_free(ctx, a.first, a.second);
  s->allocs.clear();
  free_true_model(ctx, s);
}

template <typename T>
static T *tm_upload(dino_ctx *ctx, Surrogate *s, const T *host, size_t n) {
  T *p = (T *)dev_alloc(ctx, n * sizeof(T));
  s->tm.allocs.push_back({p, n * sizeof(T)});
  CK(cudaMemcpyAsync(p, host, n * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
  return p;
}

// Attach (or with d == nullptr detach) the true map of delayed acceptance.
static void set_true_model(dino_ctx *ctx, Surrogate *s, const dino_true_model_desc *d) {
  if (s->pools > 0) fail(DINO_ESTATE, "surrogate has live chain pools");
  free_true_model(ctx, s);
  if (!d) return;
  const int N = s->N, r = s->r;
  if (d->r_t < 1 || d->r_t > N || !d->E_t || d->n_layers < 1 || !d->widths || !d->W || !d->b)
    fail(DINO_EINVAL, "true model: 1 <= r_t <= N, n_layers >= 1, non-NULL E_t, widths, W, b");
  if (d->activation < 0 || d->activation > 2) fail(DINO_EINVAL, "unknown activation");
  auto &t = s->tm;
  t.r_t = d->r_t;
  t.L = d->n_layers;
  t.act = d->activation;
  t.widths.assign(d->widths, d->widths + d->n_layers + 1);
  if (t.widths[0] != t.r_t || t.widths.back() != s->d_y)
    fail(DINO_EINVAL, "true model widths must run from r_t=%d to d_y=%d", t.r_t, s->d_y);
  for (int w : t.widths)
    if (w < 1) fail(DINO_EINVAL, "every width must be >= 1");
  std::vector<double> Et(d->E_t, d->E_t + (size_t)t.r_t * N);
  for (double v : Et)
    if (!std::isfinite(v)) fail(DINO_ENUMERIC, "non-finite entry of E_t");
  // E_t D (r_t x r), the map of the complement coefficient into E_t coordinates
  std::vector<double> EtD((size_t)t.r_t * r, 0.0);
  for (int i = 0; i < t.r_t; ++i)
    for (int p = 0; p < N; ++p) {
      const double e = Et[(size_t)i * N + p];
      if (e == 0.0) continue;
      const double *Dp = &s->D[(size_t)p * r];
      double *o = &EtD[(size_t)i * r];
      for (int j = 0; j < r; ++j) o[j] += e * Dp[j];
    }
  std::vector<std::vector<double>> W, b;
  for (int l = 0; l < t.L; ++l) {
    if (!d->W[l] || !d->b[l]) fail(DINO_EINVAL, "true model W[%d] or b[%d] is NULL", l, l);
    const size_t nw = (size_t)t.widths[l + 1] * t.widths[l];
    W.emplace_back(d->W[l], d->W[l] + nw);
    b.emplace_back(d->b[l], d->b[l] + t.widths[l + 1]);
    for (double v : W.back())
      if (!std::isfinite(v)) fail(DINO_ENUMERIC, "non-finite weight in true layer %d", l);
    if (l >= 1) t.widest = std::max(t.widest, t.widths[l]);
  }
  try {
    t.dEt = tm_upload(ctx, s, Et.data(), Et.size());
    t.dEtD = tm_upload(ctx, s, EtD.data(), EtD.size());
    for (int l = 0; l < t.L; ++l) {
      t.dW.push_back(tm_upload(ctx, s, W[l].data(), W[l].size()));
      t.db.push_back(tm_upload(ctx, s, b[l].data(), b[l].size()));
      if (s->precision == DINO_PREC_BF16) {
        const int wo = t.widths[l + 1], wi = t.widths[l], ldw = pad8(wi);
        size_t pl = 0;
        const auto bw = split_planes(W[l], wo, wi, ldw, kTrueSlices, pl);
        t.bW.push_back(tm_upload(ctx, s, bw.data(), bw.size()));
        t.ldW.push_back(ldw);
        t.plW.push_back(pl);
        const auto fb = to_f32(b[l]);
        t.fb.push_back(tm_upload(ctx, s, fb.data(), fb.size()));
      }
    }
    if (s->precision == DINO_PREC_BF16) {
      const auto be = split_planes(Et, t.r_t, N, s->ldE, kTrueSlices, t.plEt);
      const auto bd = split_planes(EtD, t.r_t, r, s->ldD, kTrueSlices, t.plEtD);
      t.bEt = tm_upload(ctx, s, be.data(), be.size());
      t.bEtD = tm_upload(ctx, s, bd.data(), bd.size());
    }
    CK(cudaStreamSynchronize(ctx->stream));
  } catch (...) {
    free_true_model(ctx, s);
    throw;
  }
  t.on = true;
}

static Surrogate *get_surrogate(dino_ctx *ctx, int id) {
  auto it = ctx->surrogates.find(id);
  if (it == ctx->surrogates.end()) fail(DINO_ENOTFOUND, "unknown surrogate id %d", id);
  return it->second.get();
}

static int load_surrogate(dino_ctx *ctx, const dino_surrogate_desc *d) {
  if (!d) fail(DINO_EINVAL, "desc is NULL");
  if (d->n_grid < 1 || d->r < 1 || d->n_layers < 1 || !d->widths || !d->W || !d->b)
    fail(DINO_EINVAL, "n_grid, r, n_layers must be >= 1 and widths/W/b non-NULL");
  if (!(d->prior_delta > 0) || !(d->prior_gamma >= 0))
    fail(DINO_EINVAL, "prior_delta must be > 0 and prior_gamma >= 0");
  if (d->precision != DINO_PREC_FP64 && d->precision != DINO_PREC_BF16)
    fail(DINO_EINVAL, "unknown precision %d", d->precision);
  if (d->activation < 0 || d->activation > 2) fail(DINO_EINVAL, "unknown activation");
  auto s = std::make_unique<Surrogate>();
  s->id = ctx->next_id++;
  s->n_grid = d->n_grid;
  s->N = d->n_grid * d->n_grid;
  if (prior_draw_smem_bytes(s->n_grid, 8) > kSmemLimit)
    fail(DINO_EINVAL, "n_grid=%d exceeds the per-chain prior draw's shared-memory budget",
         s->n_grid);
  s->gamma = d->prior_gamma;
  s->delta = d->prior_delta;
  s->r = d->r;
  s->L = d->n_layers;
  s->act = d->activation;
  s->precision = d->precision;
  s->widths.assign(d->widths, d->widths + d->n_layers + 1);
  if (s->widths[0] != s->r) fail(DINO_EINVAL, "widths[0]=%d must equal r=%d", s->widths[0], s->r);
  for (int w : s->widths)
    if (w < 1) fail(DINO_EINVAL, "every width must be >= 1");
  s->d_y = s->widths.back();
  if (s->r > s->N) fail(DINO_EINVAL, "r=%d exceeds N=%d", s->r, s->N);
  if (s->r > kMaxR) fail(DINO_EINVAL, "r=%d exceeds the supported maximum %d", s->r, kMaxR);
  if (geometry_smem_bytes(s->r, s->d_y, 1) > kSmemLimit ||
      geometry_smem_bytes(s->r, s->d_y, 0) > kSmemLimit)
    fail(DINO_EINVAL, "r=%d, d_y=%d exceed the per-chain shared-memory budget", s->r, s->d_y);
  if (d->noise_map == DINO_NOISE_AUTO)
    s->wb = s->d_y < s->r && s->d_y <= kMaxWbDy;
  else if (d->noise_map == DINO_NOISE_CHOLESKY)
    s->wb = false;
  else if (d->noise_map == DINO_NOISE_EIGEN) {
    if (!(s->d_y < s->r && s->d_y <= kMaxEigDy))
      fail(DINO_EINVAL, "the eigen noise map needs d_y < r and d_y <= %d (d_y=%d, r=%d)",
           kMaxEigDy, s->d_y, s->r);
    if (eig_smem_bytes(s->r, s->d_y) > kSmemLimit)
      fail(DINO_EINVAL, "r=%d, d_y=%d exceed the eigen map's shared-memory budget", s->r, s->d_y);
    s->wb = true;
    s->eig = true;
  } else if (d->noise_map == DINO_NOISE_PERTURBATION) {
    if (!(s->d_y < s->r && s->d_y <= kMaxWbDy))
      fail(DINO_EINVAL, "the perturbation noise map needs d_y < r and d_y <= %d (d_y=%d, r=%d)",
           kMaxWbDy, s->d_y, s->r);
    s->wb = true;
  } else {
    fail(DINO_EINVAL, "unknown noise map %d", d->noise_map);
  }
  s->tc_gram = s->wb && s->precision == DINO_PREC_BF16 && s->L >= 2 && s->d_y <= 128;
  if (s->wb && (wb_smem_bytes(s->r, s->d_y, 1) > kSmemLimit ||
                wb_smem_bytes(s->r, s->d_y, 0) > kSmemLimit))
    fail(DINO_EINVAL, "d_y=%d < r=%d: the d_y x d_y factor exceeds the shared-memory budget",
         s->d_y, s->r);  // not reached for r <= kMaxR
  if (d->precision == DINO_PREC_BF16 && s->L < 2)
    fail(DINO_EINVAL, "the tensor-core path needs at least one hidden layer");
  if (d->precision == DINO_PREC_BF16) {
    s->fwd_slices = d->fwd_slices ? d->fwd_slices : 3;
    s->jac_slices = d->jac_slices ? d->jac_slices : 2;
    if (s->fwd_slices < 1 || s->fwd_slices > 3 || s->jac_slices < 1 || s->jac_slices > 3)
      fail(DINO_EINVAL, "fwd_slices/jac_slices must be in 1..3");
  }
  for (int l = 0; l < s->L; ++l) {
    if (!d->W[l] || !d->b[l]) fail(DINO_EINVAL, "W[%d] or b[%d] is NULL", l, l);
    const size_t nw = (size_t)s->widths[l + 1] * s->widths[l];
    s->W.emplace_back(d->W[l], d->W[l] + nw);
    s->b.emplace_back(d->b[l], d->b[l] + s->widths[l + 1]);
    for (double v : s->W.back())
      if (!std::isfinite(v)) fail(DINO_ENUMERIC, "non-finite weight in layer %d", l);
  }
  // basis
  const int N = s->N, r = s->r;
  if (d->basis_kind == DINO_BASIS_KLE) {
    build_kle(s->n_grid, s->gamma, s->delta, r, s->E, s->D);
  } else if (d->basis_kind == DINO_BASIS_DIS) {
    if (!d->basis_gauss) fail(DINO_EINVAL, "DIS basis needs basis_gauss (N x r)");
    build_dis(s->n_grid, s->gamma, s->delta, r, d->basis_gauss, s->E, s->D);
  } else if (d->basis_kind == DINO_BASIS_EXPLICIT) {
    if (!d->E || !d->D) fail(DINO_EINVAL, "EXPLICIT basis needs E and D");
    s->E.assign(d->E, d->E + (size_t)r * N);
    s->D.assign(d->D, d->D + (size_t)N * r);
  } else {
    fail(DINO_EINVAL, "unknown basis kind %d", d->basis_kind);
  }
  const double ed = max_ed_error(s->E, s->D, r, N);
  if (!(ed <= 1e-8)) fail(DINO_ENUMERIC, "E D differs from I_r by %g", ed);

  // device copies
  const int n = s->n_grid;
  const auto S = sine_matrix(n);
  const auto s1 = lap1d_eigs(n);
  std::vector<double> sqrtlam((size_t)N);
  for (int ky = 0; ky < n; ++ky)
    for (int kx = 0; kx < n; ++kx)
      sqrtlam[kx + (size_t)n * ky] = 1.0 / (s->delta + s->gamma * (s1[kx] + s1[ky]));
  s->dE = sur_upload(ctx, s.get(), s->E.data(), s->E.size());
  s->dD = sur_upload(ctx, s.get(), s->D.data(), s->D.size());
  s->dS = sur_upload(ctx, s.get(), S.data(), S.size());
  s->dSqrtLam = sur_upload(ctx, s.get(), sqrtlam.data(), sqrtlam.size());
  for (int l = 0; l < s->L; ++l) {
    const int wo = s->widths[l + 1], wi = s->widths[l];
    std::vector<double> WT((size_t)wi * wo);
    for (int i = 0; i < wo; ++i)
      for (int j = 0; j < wi; ++j) WT[(size_t)j * wo + i] = s->W[l][(size_t)i * wi + j];
    s->dW.push_back(sur_upload(ctx, s.get(), s->W[l].data(), s->W[l].size()));
    s->dWT.push_back(sur_upload(ctx, s.get(), WT.data(), WT.size()));
    s->db.push_back(sur_upload(ctx, s.get(), s->b[l].data(), s->b[l].size()));
    if (l >= 1) s->widest = std::max(s->widest, wi);
    if (s->precision == DINO_PREC_BF16) {
      const auto fb = to_f32(s->b[l]);
      s->fb.push_back(sur_upload(ctx, s.get(), fb.data(), fb.size()));
      const auto fw = to_f32(s->W[l]);
      s->fW.push_back(sur_upload(ctx, s.get(), fw.data(), fw.size()));
      size_t pl = 0, plt = 0;
      const int ldw = pad8(wi), ldwt = pad8(wo);
      const auto bw = split_planes(s->W[l], wo, wi, ldw, s->fwd_slices, pl);
      const auto bwt = split_planes(WT, wi, wo, ldwt, s->jac_slices, plt);
      s->bW.push_back(sur_upload(ctx, s.get(), bw.data(), bw.size()));
      s->bWT.push_back(sur_upload(ctx, s.get(), bwt.data(), bwt.size()));
      s->ldW.push_back(ldw);
      s->ldWT.push_back(ldwt);
      s->plW.push_back(pl);
      s->plWT.push_back(plt);
    }
  }
  {
    // flops per chain of one slice product: reverse 2 d_y sum_{l=0}^{L-2} w_l w_{l+1},
    // forward 2 r sum_{l=1}^{L-1} w_l w_{l+1}
    double rev = 0.0, fwd = 0.0;
    for (int l = 0; l + 1 < s->L; ++l) rev += 2.0 * s->d_y * s->widths[l] * s->widths[l + 1];
    for (int l = 1; l < s->L; ++l) fwd += 2.0 * s->r * s->widths[l] * s->widths[l + 1];
    s->jac_fwd = s->L >= 2 && !s->wb && s->r < s->d_y && fwd < rev;
  }
  if (s->jac_fwd && s->precision == DINO_PREC_BF16) {
    const int w1 = s->widths[1];
    std::vector<double> W0T((size_t)r * w1);
    for (int i = 0; i < w1; ++i)
      for (int j = 0; j < r; ++j) W0T[(size_t)j * w1 + i] = s->W[0][(size_t)i * r + j];
    const auto f0t = to_f32(W0T);
    s->fW0T = sur_upload(ctx, s.get(), f0t.data(), f0t.size());
    s->bWj.assign(s->L, nullptr);
    s->ldWj.assign(s->L, 0);
    s->plWj.assign(s->L, 0);
    for (int l = 1; l < s->L; ++l) {
      const int wo = s->widths[l + 1], wi = s->widths[l];
      s->ldWj[l] = pad8(wi);
      const auto bw = split_planes(s->W[l], wo, wi, s->ldWj[l], s->jac_slices, s->plWj[l]);
      s->bWj[l] = sur_upload(ctx, s.get(), bw.data(), bw.size());
    }
  }
  if (s->precision == DINO_PREC_BF16) {
    const auto fS = to_f32(S), fL = to_f32(sqrtlam);
    s->fS = sur_upload(ctx, s.get(), fS.data(), fS.size());
    s->fSqrtLam = sur_upload(ctx, s.get(), fL.data(), fL.size());
    s->ldE = pad8(s->N);
    s->ldD = pad8(s->r);
    const auto be = split_planes(s->E, s->r, s->N, s->ldE, kFieldSlices, s->plE);
    const auto bd = split_planes(s->D, s->N, s->r, s->ldD, kFieldSlices, s->plD);
    s->bE = sur_upload(ctx, s.get(), be.data(), be.size());
    s->bD = sur_upload(ctx, s.get(), bd.data(), bd.size());
  }
  if (d->y) {
    if (!(d->noise_var > 0)) fail(DINO_EINVAL, "noise_var must be > 0");
    s->y.assign(d->y, d->y + s->d_y);
    s->noise_var = d->noise_var;
    s->has_data = true;
    upload_data(ctx, s.get());
  }
  CK(cudaStreamSynchronize(ctx->stream));
  const int id = s->id;
  ctx->surrogates[id] = std::move(s);
  return id;
}

// ---------------------------------------------------------------------------
// workspace for evaluating the surrogate (forward + Jacobian) at C points

struct Work {
  int C = 0;
  // FP64 path
  std::vector<double *> act64, der64;
  double *f64 = nullptr, *P64[2] = {nullptr, nullptr}, *J64 = nullptr;
  // tensor path
  __nv_bfloat16 *xb = nullptr;
  int ldx = 0;
  size_t plx = 0;
  std::vector<__nv_bfloat16 *> actb;
  std::vector<int> ldact;
  std::vector<size_t> plact;
  std::vector<float *> der32;
  float *f32 = nullptr, *J32 = nullptr;
  // forward-mode Jacobian: J^T per chain (C x r x d_y), FP64 or FP32
  void *Jt = nullptr;
  __nv_bfloat16 *Pb[2] = {nullptr, nullptr};
  int ldp = 0;
  size_t plp = 0;
  // Gram matrices on the tensor cores: J as bf16 slices (rows x ldjb) and
  // G (C x d_y x ldg, FP32)
  __nv_bfloat16 *Jb = nullptr;
  int ldjb = 0, ldg = 0;
  size_t pljb = 0;
  float *G = nullptr;
  // ... and K b, K a formed right after the Jacobian (warp per row): b and
  // the state m_r as double-float pairs (C x r) in, Kb, Ka (C x d_y) out
  float2 *b_df = nullptr, *a_df = nullptr;
  double *Kb = nullptr, *Ka = nullptr;
};

// Lays out (or, with base != nullptr, assigns) the workspace in an arena.
static void layout_work(const Surrogate *s, int C, Arena &ar, Work &w, bool assign, bool gram) {
  auto take = [&](size_t bytes) -> char * {
    const size_t at = ar.reserve(bytes);
    return assign ? ar.base + at : nullptr;
  };
  w.C = C;
  const int L = s->L, dy = s->d_y;
  const size_t rows = (size_t)C * dy;
  // rows of the stacked Jacobian accumulation: d_y per chain in reverse mode, r in forward
  const size_t prows = s->jac_fwd ? (size_t)C * std::max(dy, s->r) : rows;
  w.act64.assign(L, nullptr);
  w.der64.assign(L, nullptr);
  w.der32.assign(L, nullptr);
  w.actb.assign(L, nullptr);
  w.ldact.assign(L, 0);
  w.plact.assign(L, 0);
  if (s->precision == DINO_PREC_FP64) {
    for (int l = 0; l + 1 < L; ++l) {
      w.act64[l] = (double *)take((size_t)C * s->widths[l + 1] * 8);
      w.der64[l] = (double *)take((size_t)C * s->widths[l + 1] * 8);
    }
    w.f64 = (double *)take((size_t)C * dy * 8);
    if (L >= 2) {
      w.P64[0] = (double *)take(prows * s->widest * 8);
      w.P64[1] = (double *)take(prows * s->widest * 8);
    }
    w.J64 = (double *)take(rows * s->r * 8);
    if (s->jac_fwd) w.Jt = take(rows * s->r * 8);
  } else {
    w.ldx = pad8(s->r);
    w.plx = (size_t)C * w.ldx;
    w.xb = (__nv_bfloat16 *)take(w.plx * s->fwd_slices * 2);
    for (int l = 0; l + 1 < L; ++l) {
      const int wd = s->widths[l + 1];
      w.ldact[l] = pad8(wd);
      w.plact[l] = (size_t)C * w.ldact[l];
      w.actb[l] = (__nv_bfloat16 *)take(w.plact[l] * s->fwd_slices * 2);
      w.der32[l] = (float *)take((size_t)C * wd * 4);
    }
    w.f32 = (float *)take((size_t)C * dy * 4);
    if (L >= 2) {
      w.ldp = pad8(s->widest);
      w.plp = prows * w.ldp;
      w.Pb[0] = (__nv_bfloat16 *)take(w.plp * s->jac_slices * 2);
      w.Pb[1] = (__nv_bfloat16 *)take(w.plp * s->jac_slices * 2);
    }
    w.J32 = (float *)take(rows * s->r * 4);
    if (s->jac_fwd) w.Jt = take(rows * s->r * 4);
    if (gram) {
      w.ldjb = pad8(s->r);
      w.pljb = rows * w.ldjb;
      w.Jb = (__nv_bfloat16 *)take(w.pljb * kGramSlices * 2);
      w.ldg = (dy + 3) & ~3;
      w.G = (float *)take(rows * w.ldg * 4);
      w.b_df = (float2 *)take((size_t)C * s->r * 8);
      w.a_df = (float2 *)take((size_t)C * s->r * 8);
      w.Kb = (double *)take(rows * 8);
      w.Ka = (double *)take(rows * 8);
    }
  }
}

// Forward pass and Jacobian at the C points in `x` (FP64 C x r; the tensor
// path reads the bf16 planes in w.xb, which the caller has filled).
// with_a: the pool's state pairs w.a_df are valid (a step, not the initial
// geometry), so K a is formed beside K b.
static void eval_surrogate(dino_ctx *ctx, const Surrogate *s, Work &w, const double *x,
                           cudaStream_t st, bool with_a = false) {
  const int C = w.C, L = s->L, dy = s->d_y, r = s->r;
  if (s->precision == DINO_PREC_FP64) {
    const double *a = x;
    int lda = r;
    for (int l = 0; l + 1 < L; ++l) {
      const int wo = s->widths[l + 1], wi = s->widths[l];
      launch(ctx, st, "mlp_f64", [&] {
        return gemm_bias_act<double>(C, wo, wi, a, lda, s->dW[l], wi, s->db[l], s->act,
                                     w.act64[l], w.der64[l], wo, st);
      });
      a = w.act64[l];
      lda = wo;
    }
    launch(ctx, st, "mlp_f64", [&] {
      return gemm_bias_act<double>(C, dy, s->widths[L - 1], a, lda, s->dW[L - 1],
                                   s->widths[L - 1], s->db[L - 1], 0, w.f64, nullptr, dy, st);
    });
    if (L == 1) {
      launch(ctx, st, "jac_broadcast", [&] {
        return launch_broadcast<double>(C, (size_t)dy * r, s->dW[0], w.J64, st);
      });
      return;
    }
    if (s->jac_fwd) {
      // forward mode on J^T: T = W_0^T .* d_0 (r x w_1 per chain);
      // T <- (T W_l^T) .* d_l; J^T = T W_{L-1}^T, then J per chain
      const int w1 = s->widths[1];
      launch(ctx, st, "jac_init_f64", [&] {
        return launch_jac_init<double>(C, r, w1, s->dWT[0], w.der64[0], w1, w.P64[0], st);
      });
      int cur = 0;
      for (int l = 1; l + 1 < L; ++l) {
        const int wi = s->widths[l], wo = s->widths[l + 1];
        launch(ctx, st, "jac_gemm_f64", [&] {
          return gemm_scale_group<double>(C * r, wo, wi, w.P64[cur], wi, s->dW[l], wi,
                                          w.der64[l], wo, r, w.P64[1 - cur], wo, st);
        });
        cur = 1 - cur;
      }
      const int wl = s->widths[L - 1];
      launch(ctx, st, "jac_gemm_f64", [&] {
        return gemm_store<double>(C * r, dy, wl, w.P64[cur], wl, s->dW[L - 1], wl,
                                  (double *)w.Jt, dy, st);
      });
      launch(ctx, st, "jac_transpose", [&] {
        return launch_batched_transpose(C, r, dy, w.Jt, 0, w.J64, st);
      });
      return;
    }
    // reverse mode: P = W_{L-1} .* d_{L-2}; P <- (P W_l) .* d_{l-1}; J = P W_0
    const int wl = s->widths[L - 1];
    launch(ctx, st, "jac_init_f64", [&] {
      return launch_jac_init<double>(C, dy, wl, s->dW[L - 1], w.der64[L - 2], wl, w.P64[0], st);
    });
    int cur = 0;
    for (int l = L - 2; l >= 1; --l) {
      const int wi = s->widths[l], wo = s->widths[l + 1];
      launch(ctx, st, "jac_gemm_f64", [&] {
        return gemm_scale_group<double>(C * dy, wi, wo, w.P64[cur], wo, s->dWT[l], wo,
                                        w.der64[l - 1], wi, dy, w.P64[1 - cur], wi, st);
      });
      cur = 1 - cur;
    }
    launch(ctx, st, "jac_gemm_f64", [&] {
      return gemm_store<double>(C * dy, r, s->widths[1], w.P64[cur], s->widths[1], s->dWT[0],
                                s->widths[1], w.J64, r, st);
    });
    return;
  }
  // tensor-core path
  const __nv_bfloat16 *a = w.xb;
  int lda = w.ldx;
  size_t pla = w.plx;
  for (int l = 0; l + 1 < L; ++l) {
    TcGemmArgs g;
    g.M = C;
    g.N = s->widths[l + 1];
    g.K = s->widths[l];
    g.A = a;
    g.lda = lda;
    g.a_plane = pla;
    g.B = s->bW[l];
    g.ldb = s->ldW[l];
    g.b_plane = s->plW[l];
    g.nslice = s->fwd_slices;
    g.epi = TC_EPI_BIAS_ACT;
    g.bias = s->fb[l];
    g.act = s->act;
    g.out_bf = w.actb[l];
    g.ldo = w.ldact[l];
    g.out_plane = w.plact[l];
    g.out_slices = s->fwd_slices;
    g.der = w.der32[l];
    launch(ctx, st, "mlp_tc", [&] { return launch_tc_gemm(g, st); });
    a = w.actb[l];
    lda = w.ldact[l];
    pla = w.plact[l];
  }
  {
    TcGemmArgs g;
    g.M = C;
    g.N = dy;
    g.K = s->widths[L - 1];
    g.A = a;
    g.lda = lda;
    g.a_plane = pla;
    g.B = s->bW[L - 1];
    g.ldb = s->ldW[L - 1];
    g.b_plane = s->plW[L - 1];
    g.nslice = s->fwd_slices;
    g.epi = TC_EPI_BIAS_F32;
    g.bias = s->fb[L - 1];
    g.outf = w.f32;
    g.ldo = dy;
    launch(ctx, st, "mlp_tc", [&] { return launch_tc_gemm(g, st); });
  }
  if (s->jac_fwd) {
    // forward mode on J^T (see the FP64 path), bf16 slices of T, W_l as B
    const int w1 = s->widths[1];
    launch(ctx, st, "jac_init_tc", [&] {
      return launch_jac_init_bf16(C, r, w1, s->fW0T, w.der32[0], w1, w.Pb[0], w.ldp, w.plp,
                                  s->jac_slices, st);
    });
    int cur = 0;
    for (int l = 1; l < L; ++l) {
      const bool last = l + 1 == L;
      TcGemmArgs g;
      g.M = C * r;
      g.N = s->widths[l + 1];
      g.K = s->widths[l];
      g.A = w.Pb[cur];
      g.lda = w.ldp;
      g.a_plane = w.plp;
      g.B = s->bWj[l];
      g.ldb = s->ldWj[l];
      g.b_plane = s->plWj[l];
      g.nslice = s->jac_slices;
      if (last) {
        g.epi = TC_EPI_STORE_F32;
        g.outf = (float *)w.Jt;
        g.ldo = dy;
      } else {
        g.epi = TC_EPI_SCALE_GROUP;
        g.scale = w.der32[l];
        g.lds = s->widths[l + 1];
        g.group = r;
        g.out_bf = w.Pb[1 - cur];
        g.ldo = w.ldp;
        g.out_plane = w.plp;
        g.out_slices = s->jac_slices;
      }
      launch(ctx, st, "jac_tc", [&] { return launch_tc_gemm(g, st); });
      cur = 1 - cur;
    }
    launch(ctx, st, "jac_transpose", [&] {
      return launch_batched_transpose(C, r, dy, w.Jt, 1, w.J32, st);
    });
    return;
  }
  const int wl = s->widths[L - 1];
  launch(ctx, st, "jac_init_tc", [&] {
    return launch_jac_init_bf16(C, dy, wl, s->fW[L - 1], w.der32[L - 2], wl, w.Pb[0], w.ldp,
                                w.plp, s->jac_slices, st);
  });
  int cur = 0;
  for (int l = L - 2; l >= 1; --l) {
    TcGemmArgs g;
    g.M = C * dy;
    g.N = s->widths[l];
    g.K = s->widths[l + 1];
    g.A = w.Pb[cur];
    g.lda = w.ldp;
    g.a_plane = w.plp;
    g.B = s->bWT[l];
    g.ldb = s->ldWT[l];
    g.b_plane = s->plWT[l];
    g.nslice = s->jac_slices;
    g.epi = TC_EPI_SCALE_GROUP;
    g.scale = w.der32[l - 1];
    g.lds = s->widths[l];
    g.group = dy;
    g.out_bf = w.Pb[1 - cur];
    g.ldo = w.ldp;
    g.out_plane = w.plp;
    g.out_slices = s->jac_slices;
    launch(ctx, st, "jac_tc", [&] { return launch_tc_gemm(g, st); });
    cur = 1 - cur;
  }
  TcGemmArgs g;
  g.M = C * dy;
  g.N = r;
  g.K = s->widths[1];
  g.A = w.Pb[cur];
  g.lda = w.ldp;
  g.a_plane = w.plp;
  g.B = s->bWT[0];
  g.ldb = s->ldWT[0];
  g.b_plane = s->plWT[0];
  g.nslice = s->jac_slices;
  g.epi = TC_EPI_STORE_F32;
  g.outf = w.J32;
  g.ldo = r;
  if (w.Jb) {  // also the slices the Gram matrices are formed from
    g.out_bf = w.Jb;
    g.ldob = w.ldjb;
    g.out_plane = w.pljb;
    g.out_slices = kGramSlices;
  }
  launch(ctx, st, "jac_tc", [&] { return launch_tc_gemm(g, st); });
  if (w.Kb)  // K b = J b / sigma (K a likewise) in double-float
    launch(ctx, st, "rowprod", [&] {
      return launch_rowprod(C * dy, r, dy, w.J32, w.b_df, with_a ? w.a_df : nullptr,
                            std::sqrt(1.0 / s->noise_var), w.Kb, with_a ? w.Ka : nullptr, st);
    });
  if (w.G)
    launch(ctx, st, "gram_tc", [&] {
      return launch_tc_gram(C, dy, r, w.Jb, w.ldjb, w.pljb, kGramSlices, w.G, w.ldg, st);
    });
}

// ---------------------------------------------------------------------------
// chain pools

struct Pool {
  int id = 0;
  Surrogate *s = nullptr;
  cudaStream_t st = nullptr;  // stream all of this pool's work goes to
  bool async_mem = false;     // arena from the stream-ordered allocator
  int C = 0;
  double dt = 0, sc = 0;
  uint64_t seed = 0, id_base = 0;
  uint32_t step = 0;
  Arena ar;
  bool eig = false;  // eigen map (with wb: the J state of the d_y-sized path)
  bool wb = false;  // Woodbury path (the surrogate's d_y < r); scratch pools of
                    // surrogate_eval always take the r-sized path
  // state
  double *mr, *g, *phi, *hld, *L;
  int *cur;  // per-chain slot (0/1) of the current factor in L
  void *Js;  // Woodbury path: J at each chain's current point
  void *m;  // C x N, double (FP64 path) or float (tensor path)
  double *b, *mu, *lq_fwd, *coef, *log_rho, *log_u;
  int *acc;
  unsigned long long *acc_count, *counters;
  double *sum_alpha;
  int *err;  // raised by a kernel whose bounded wait gave up
  // field scratch
  void *Mf, *coef2;
  // tensor path: bf16 slice planes of the prior draw (C x ldE) and of coef2 (C x ldD)
  __nv_bfloat16 *Ms = nullptr, *coef2s = nullptr;
  Work w;
  // caller-supplied noise of the next transition (dino_chains_set_noise):
  // one device buffer [xi C x r | xi2 C x d_y | z C x N | log_u C], and which
  // parts are set
  double *ext = nullptr;
  size_t ext_bytes = 0;
  bool ext_xi = false, ext_xi2 = false, ext_z = false, ext_log_u = false, ext_log_u2 = false;
  // delayed acceptance (the surrogate has a true model): chain state E_t m
  // (C x r_t) and Phi(m); the first stage's staging (Phi~, half log det, g);
  // E_t m^dagger and its pieces; the true map's output and work buffers;
  // log rho^(2), log u2 and the first-stage flags of the last transition
  bool da = false;
  double *mt = nullptr, *phi_t = nullptr, *phi_st = nullptr, *hld_st = nullptr,
         *g_st = nullptr, *xt = nullptr, *lr2 = nullptr, *lu2 = nullptr;
  int *st1 = nullptr;
  void *EtM = nullptr, *EtDc = nullptr, *ft = nullptr;
  std::vector<double *> tact64;              // FP64: hidden activations of f_t
  __nv_bfloat16 *xtb = nullptr;              // tensor path: slices of xt
  int ldxt = 0;
  std::vector<__nv_bfloat16 *> tactb;        // tensor path: hidden activations as slices
  std::vector<int> ldtact;
  float *tder = nullptr;                     // tensor path: derivative scratch of f_t
};

static void layout_pool(Pool &p, bool assign) {
  const Surrogate *s = p.s;
  const int C = p.C, r = s->r, N = s->N;
  const size_t fe = s->precision == DINO_PREC_FP64 ? 8 : 4;
  Arena &ar = p.ar;
  ar.off = 0;
  auto take = [&](size_t bytes) -> char * {
    const size_t at = ar.reserve(bytes);
    return assign ? ar.base + at : nullptr;
  };
  p.mr = (double *)take((size_t)C * r * 8);
  p.g = (double *)take((size_t)C * r * 8);
  p.phi = (double *)take((size_t)C * 8);
  p.hld = (double *)take((size_t)C * 8);
  const size_t ss = p.eig ? eig_slot_stride(s->d_y)
                          : p.wb ? wb_slot_stride(s->d_y) : slot_stride(r);
  p.L = (double *)take(2 * (size_t)C * ss * 8);  // two slots
  p.cur = (int *)take((size_t)C * 4);
  p.Js = p.wb ? take((size_t)C * s->d_y * r * fe) : nullptr;
  p.m = take((size_t)C * N * fe);
  p.b = (double *)take((size_t)C * r * 8);
  p.mu = (double *)take((size_t)C * r * 8);
  p.lq_fwd = (double *)take((size_t)C * 8);
  p.coef = (double *)take((size_t)C * r * 8);
  p.log_rho = (double *)take((size_t)C * 8);
  p.log_u = (double *)take((size_t)C * 8);
  p.acc = (int *)take((size_t)C * 4);
  p.acc_count = (unsigned long long *)take((size_t)C * 8);
  p.counters = (unsigned long long *)take(4 * 8);
  p.sum_alpha = (double *)take(8);
  p.err = (int *)take(16);
  // FP64 at init even on the FP32 path; also holds a zero data vector in surrogate_eval
  p.Mf = take(std::max((size_t)C * N, (size_t)s->d_y) * std::max(fe, (size_t)8));
  // FP64 path only: the tensor path keeps coef2 as bf16 slices (coef2s)
  p.coef2 = s->precision == DINO_PREC_FP64 ? take((size_t)C * r * 8) : nullptr;
  if (s->precision != DINO_PREC_FP64) {
    p.Ms = (__nv_bfloat16 *)take((size_t)C * s->ldE * kFieldSlices * 2);
    p.coef2s = (__nv_bfloat16 *)take((size_t)C * s->ldD * kFieldSlices * 2);
  }
  layout_work(s, C, ar, p.w, assign, p.wb && s->tc_gram);
  p.da = s->tm.on;
  if (p.da) {
    const auto &t = s->tm;
    const size_t rt = t.r_t, dy = s->d_y;
    p.mt = (double *)take(C * rt * 8);
    p.phi_t = (double *)take((size_t)C * 8);
    p.phi_st = (double *)take((size_t)C * 8);
    p.hld_st = (double *)take((size_t)C * 8);
    p.g_st = p.wb ? nullptr : (double *)take((size_t)C * r * 8);
    p.xt = (double *)take(C * rt * 8);
    p.lr2 = (double *)take((size_t)C * 8);
    p.lu2 = (double *)take((size_t)C * 8);
    p.st1 = (int *)take((size_t)C * 4);
    p.EtM = take(C * rt * fe);
    p.EtDc = take(C * rt * fe);
    p.ft = take(C * dy * fe);
    p.tact64.assign(t.L, nullptr);
    p.tactb.assign(t.L, nullptr);
    p.ldtact.assign(t.L, 0);
    if (s->precision == DINO_PREC_FP64) {
      for (int l = 0; l + 1 < t.L; ++l) p.tact64[l] = (double *)take((size_t)C * t.widths[l + 1] * 8);
    } else {
      p.ldxt = pad8(t.r_t);
      p.xtb = (__nv_bfloat16 *)take((size_t)C * p.ldxt * kTrueSlices * 2);
      for (int l = 0; l + 1 < t.L; ++l) {
        p.ldtact[l] = pad8(t.widths[l + 1]);
        p.tactb[l] = (__nv_bfloat16 *)take((size_t)C * p.ldtact[l] * kTrueSlices * 2);
      }
      p.tder = (float *)take((size_t)C * std::max(1, t.widest) * 4);
    }
  }
}

static Pool *get_pool(dino_ctx *ctx, int id) {
  auto it = ctx->pools.find(id);
  if (it == ctx->pools.end()) fail(DINO_ENOTFOUND, "unknown pool id %d", id);
  return it->second.get();
}

static ReducedArgs reduced_args(const Pool &p) {
  const Surrogate *s = p.s;
  ReducedArgs a;
  a.C = p.C;
  a.r = s->r;
  a.d_y = s->d_y;
  a.s = p.sc;
  a.dt = p.dt;
  a.noise_var = s->noise_var;
  a.seed = p.seed;
  a.id_base = p.id_base;
  a.step = p.step;
  a.mr = p.mr;
  a.g = p.g;
  a.phi = p.phi;
  a.hld = p.hld;
  a.L = p.L;
  a.cur = p.cur;
  a.L_slot = (size_t)p.C * (p.eig  ? eig_slot_stride(s->d_y)
                           : p.wb ? wb_slot_stride(s->d_y) : slot_stride(s->r));
  a.Js = p.Js;
  a.G = p.w.G;
  a.ldg = p.w.ldg;
  a.b_df = p.w.b_df;
  a.a_df = p.w.a_df;
  a.Kb_pre = p.w.Kb;
  a.Ka_pre = p.w.Ka;
  a.b = p.b;
  a.mu = p.mu;
  a.lq_fwd = p.lq_fwd;
  a.y = s->dy;
  a.coef = p.coef;
  a.log_rho = p.log_rho;
  a.log_u = p.log_u;
  a.acc = p.acc;
  a.acc_count = p.acc_count;
  a.counters = p.counters;
  a.sum_alpha = p.sum_alpha;
  a.err = p.err;
  if (p.ext) {
    const size_t C = p.C;
    a.ext_xi = p.ext_xi ? p.ext : nullptr;
    a.ext_xi2 = p.ext_xi2 ? p.ext + C * s->r : nullptr;
    a.ext_log_u = p.ext_log_u ? p.ext + C * (s->r + s->d_y + (size_t)s->N) : nullptr;
  }
  if (p.da) {
    a.da = 1;
    a.phi_st = p.phi_st;
    a.hld_st = p.hld_st;
    a.g_st = p.g_st;
  }
  if (s->precision == DINO_PREC_FP64) {
    a.J = p.w.J64;
    a.f = p.w.f64;
    a.jf_f32 = 0;
  } else {
    a.J = p.w.J32;
    a.f = p.w.f32;
    a.jf_f32 = 1;
    a.b_bf16 = p.w.xb;
    a.b_slices = s->fwd_slices;
    a.b_ld = p.w.ldx;
    a.b_plane = p.w.plx;
  }
  return a;
}

static void split_input(dino_ctx *ctx, const Surrogate *s, Work &w, const double *x,
                        cudaStream_t st) {
  if (s->precision != DINO_PREC_BF16) return;
  launch(ctx, st, "split_bf16", [&] {
    return launch_split_bf16_f64(w.C, s->r, x, s->r, w.xb, w.ldx, w.plx, s->fwd_slices, st);
  });
}

static size_t pool_footprint(const Surrogate *s, int C);

// The true map f_t at the C points x_t = p.xt (FP64 path) or its slices
// p.xtb (tensor path), into p.ft.
static void true_forward(dino_ctx *ctx, const Surrogate *s, Pool &p, cudaStream_t st) {
  const auto &t = s->tm;
  const int C = p.C, L = t.L, dy = s->d_y;
  if (s->precision == DINO_PREC_FP64) {
    const double *a = p.xt;
    int lda = t.r_t;
    for (int l = 0; l < L; ++l) {
      const int wo = t.widths[l + 1], wi = t.widths[l];
      const bool last = l + 1 == L;
      double *out = last ? (double *)p.ft : p.tact64[l];
      launch(ctx, st, "true_mlp_f64", [&] {
        return gemm_bias_act<double>(C, wo, wi, a, lda, t.dW[l], wi, t.db[l], last ? 0 : t.act,
                                     out, nullptr, wo, st);
      });
      a = out;
      lda = wo;
    }
    return;
  }
  const __nv_bfloat16 *a = p.xtb;
  int lda = p.ldxt;
  for (int l = 0; l < L; ++l) {
    const bool last = l + 1 == L;
    TcGemmArgs g;
    g.M = C;
    g.N = t.widths[l + 1];
    g.K = t.widths[l];
    g.A = a;
    g.lda = lda;
    g.a_plane = (size_t)C * lda;
    g.B = t.bW[l];
    g.ldb = t.ldW[l];
    g.b_plane = t.plW[l];
    g.nslice = kTrueSlices;
    g.bias = t.fb[l];
    if (last) {
      g.epi = TC_EPI_BIAS_F32;
      g.outf = (float *)p.ft;
      g.ldo = dy;
    } else {
      g.epi = TC_EPI_BIAS_ACT;
      g.act = t.act;
      g.out_bf = p.tactb[l];
      g.ldo = p.ldtact[l];
      g.out_plane = (size_t)C * p.ldtact[l];
      g.out_slices = kTrueSlices;
      g.der = p.tder;
    }
    launch(ctx, st, "true_mlp_tc", [&] { return launch_tc_gemm(g, st); });
    if (!last) {
      a = p.tactb[l];
      lda = p.ldtact[l];
    }
  }
}

// E_t m^dagger = s E_t m + cs E_t M + (E_t D) coef2, the true map there,
// log rho^(2), the second test and the commit (Algorithm 1's second stage).
static void da_stage(dino_ctx *ctx, Pool &p, double cs, cudaStream_t st) {
  const Surrogate *s = p.s;
  const auto &t = s->tm;
  const int C = p.C, r = s->r, N = s->N, rt = t.r_t;
  const bool tc = s->precision != DINO_PREC_FP64;
  if (!tc) {
    launch(ctx, st, "da_proj_f64", [&] {
      return gemm_store<double>(C, rt, N, (const double *)p.Mf, N, t.dEt, N, (double *)p.EtM, rt,
                                st);
    });
    launch(ctx, st, "da_proj_f64", [&] {
      return gemm_store<double>(C, rt, r, (const double *)p.coef2, r, t.dEtD, r,
                                (double *)p.EtDc, rt, st);
    });
  } else {
    auto proj = [&](const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, size_t bpl, int K,
                    void *out) {
      TcGemmArgs g;
      g.M = C;
      g.N = rt;
      g.K = K;
      g.A = A;
      g.lda = lda;
      g.a_plane = (size_t)C * lda;
      g.B = B;
      g.ldb = lda;
      g.b_plane = bpl;
      g.nslice = kFieldSlices;
      g.epi = TC_EPI_STORE_F32;
      g.outf = (float *)out;
      g.ldo = rt;
      launch(ctx, st, "da_proj_tc", [&] { return launch_tc_gemm(g, st); });
    };
    proj(p.Ms, s->ldE, t.bEt, t.plEt, N, p.EtM);          // E_t M
    proj(p.coef2s, s->ldD, t.bEtD, t.plEtD, r, p.EtDc);   // (E_t D) coef2
  }
  launch(ctx, st, "da_assemble", [&] {
    return launch_da_assemble(C, rt, p.sc, cs, p.mt, p.EtM, p.EtDc, tc ? 1 : 0, p.xt, p.xtb,
                              p.ldxt, (size_t)C * p.ldxt, kTrueSlices, st);
  });
  true_forward(ctx, s, p, st);
  DaArgs a;
  a.C = C;
  a.r = r;
  a.d_y = s->d_y;
  a.r_t = rt;
  a.noise_var = s->noise_var;
  a.seed = p.seed;
  a.id_base = p.id_base;
  a.step = p.step;
  a.acc = p.acc;
  a.stage1 = p.st1;
  a.mt = p.mt;
  a.phi_t = p.phi_t;
  a.xt = p.xt;
  a.ft = p.ft;
  a.ft_f32 = tc ? 1 : 0;
  a.y = s->dy;
  a.mr = p.mr;
  a.phi = p.phi;
  a.hld = p.hld;
  a.g = p.g;
  a.b = p.b;
  a.phi_st = p.phi_st;
  a.hld_st = p.hld_st;
  a.g_st = p.g_st;
  a.cur = p.cur;
  if (p.wb) {
    a.J = tc ? (const void *)p.w.J32 : (const void *)p.w.J64;
    a.Js = p.Js;
    a.j_f32 = tc ? 1 : 0;
    a.b_df = p.w.b_df;
    a.a_df = p.w.a_df;
  }
  a.acc_count = p.acc_count;
  a.counters = p.counters;
  a.log_rho2 = p.lr2;
  a.log_u2 = p.lu2;
  a.ext_log_u2 = p.ext && p.ext_log_u2 ? p.ext + (size_t)C * (r + s->d_y + (size_t)N + 1) : nullptr;
  launch(ctx, st, "da_decide", [&] { return launch_da_decide(a, st); });
}

// Initial true-model state of a DA pool from its FP64 initial field m64.
static void da_init(dino_ctx *ctx, Pool &p, const double *m64, cudaStream_t st) {
  const Surrogate *s = p.s;
  const auto &t = s->tm;
  const int C = p.C, N = s->N, rt = t.r_t;
  const bool tc = s->precision != DINO_PREC_FP64;
  launch(ctx, st, "da_encode_f64", [&] {
    return gemm_store<double>(C, rt, N, m64, N, t.dEt, N, p.mt, rt, st);
  });
  launch(ctx, st, "da_assemble", [&] {
    return launch_da_assemble(C, rt, 1.0, 0.0, p.mt, nullptr, nullptr, tc ? 1 : 0, p.xt, p.xtb,
                              p.ldxt, (size_t)C * p.ldxt, kTrueSlices, st);
  });
  true_forward(ctx, s, p, st);
  launch(ctx, st, "da_misfit", [&] {
    return launch_da_misfit(C, s->d_y, p.ft, tc ? 1 : 0, s->dy, s->noise_var, p.phi_t, st);
  });
}

static Pool *create_pool_on(dino_ctx *ctx, int sid, int C, double dt, uint64_t seed,
                            uint64_t id_base, const double *m0, cudaStream_t st,
                            bool serving) {
  Surrogate *s = get_surrogate(ctx, sid);
  if (C < 1) fail(DINO_EINVAL, "n_chains must be >= 1");
  if (!(dt > 0) || !std::isfinite(dt)) fail(DINO_EINVAL, "dt must be > 0");
  if (!s->has_data) fail(DINO_ESTATE, "surrogate %d has no data (dino_set_data)", sid);
  auto p = std::make_unique<Pool>();
  p->id = ctx->next_id++;
  p->s = s;
  p->C = C;
  p->dt = dt;
  p->sc = (4.0 - dt) / (4.0 + dt);
  p->seed = seed;
  p->id_base = id_base;
  p->st = st;
  p->async_mem = serving;
  p->wb = s->wb;
  p->eig = s->eig;
  layout_pool(*p, false);
  p->ar.bytes = p->ar.off;
  p->ar.base = (char *)(serving ? dev_alloc_async(ctx, p->ar.bytes, st)
                                : dev_alloc(ctx, p->ar.bytes));
  try {
    layout_pool(*p, true);
    const int r = s->r, N = s->N;
    CK(cudaMemsetAsync(p->acc_count, 0, (size_t)C * 8, st));
    CK(cudaMemsetAsync(p->counters, 0, 32, st));
    CK(cudaMemsetAsync(p->sum_alpha, 0, 8, st));
    CK(cudaMemsetAsync(p->err, 0, 16, st));
    CK(cudaMemsetAsync(p->cur, 0, (size_t)C * 4, st));
    CK(cudaMemsetAsync(p->acc, 0, (size_t)C * 4, st));
    double *m64 = (double *)p->Mf;  // FP64 initial field
    if (m0 && !serving && ctx->pageable_access) {
      // synchronous create on a device that reads pageable host memory
      // coherently (Grace: NVLink-C2C): a kernel reads m0 in place; the call
      // returns only after the stream has drained
      launch(ctx, st, "field_in", [&] { return launch_copy_f64((size_t)C * N, m0, m64, st); });
    } else if (m0) {
      CK(cudaMemcpyAsync(m64, m0, (size_t)C * N * 8, cudaMemcpyHostToDevice, st));
    } else {
      launch(ctx, st, "prior_draw_f64", [&] {
        return launch_prior_draw<double>(C, s->n_grid, s->dSqrtLam, s->dS, seed, id_base,
                                         STREAM_INIT_ID, 0, m64, N, st);
      });
    }
    // m_r = E m0 (eq:projector), then the geometry at m_r
    launch(ctx, st, "encode_f64", [&] {
      return gemm_store<double>(C, r, N, m64, N, s->dE, N, p->b, r, st);
    });
    if (s->precision == DINO_PREC_FP64) {
      CK(cudaMemcpyAsync(p->m, m64, (size_t)C * N * 8, cudaMemcpyDeviceToDevice, st));
    } else {
      launch(ctx, st, "convert", [&] {
        return launch_f64_to_f32((size_t)C * N, m64, (float *)p->m, st);
      });
    }
    split_input(ctx, s, p->w, p->b, st);
    if (p->w.b_df)  // b = m_r as double-float pairs, for K b in the Jacobian GEMM
      launch(ctx, st, "to_df", [&] {
        return launch_to_df((size_t)C * r, p->b, p->w.b_df, p->w.a_df, st);
      });
    eval_surrogate(ctx, s, p->w, p->b, st);
    ReducedArgs ra = reduced_args(*p);
    launch(ctx, st, "geometry_init", [&] {
      return p->eig ? launch_eig_geometry(ra, 0, st)
             : p->wb ? launch_wb_geometry(ra, 0, st) : launch_geometry(ra, 0, st);
    });
    if (p->da) da_init(ctx, *p, m64, st);
    if (!serving) CK(cudaStreamSynchronize(st));
  } catch (...) {
    if (serving)
      dev_free_async(ctx, p->ar.base, p->ar.bytes, st);
    else
      dev_free(ctx, p->ar.base, p->ar.bytes);
    throw;
  }
  s->pools += 1;
  Pool *raw = p.get();
  ctx->pools[p->id] = std::move(p);
  return raw;
}

static int create_pool(dino_ctx *ctx, int sid, int C, double dt, uint64_t seed,
                       uint64_t id_base, const double *m0) {
  return create_pool_on(ctx, sid, C, dt, seed, id_base, m0, ctx->stream, false)->id;
}

static size_t pool_footprint(const Surrogate *s, int C) {
  Pool p;
  p.s = const_cast<Surrogate *>(s);
  p.C = C;
  p.wb = s->wb;
  p.eig = s->eig;
  layout_pool(p, false);
  return p.ar.off;
}

// One transition of every chain of the pool.
static void step_pool(dino_ctx *ctx, Pool &p) {
  const Surrogate *s = p.s;
  const int C = p.C, r = s->r, N = s->N;
  cudaStream_t st = p.st;
  const double cs = std::sqrt(1.0 - p.sc * p.sc);
  ReducedArgs ra = reduced_args(p);
  const double *ext_z =
      p.ext && p.ext_z ? p.ext + (size_t)C * (r + s->d_y) : nullptr;
  launch(ctx, st, "propose", [&] {
    return p.eig ? launch_eig_propose(ra, st) : p.wb ? launch_wb_propose(ra, st)
                                                     : launch_propose(ra, st);
  });
  eval_surrogate(ctx, s, p.w, p.b, st, true);
  launch(ctx, st, "geometry", [&] {
    return p.eig ? launch_eig_geometry(ra, 1, st)
           : p.wb ? launch_wb_geometry(ra, 1, st) : launch_geometry(ra, 1, st);
  });
  // complement (Prop. 5.1): M prior draw, coef2 = (b - s a) - cs E M, m <- s m + cs M + D coef2
  if (s->precision == DINO_PREC_FP64) {
    double *Mf = (double *)p.Mf, *coef2 = (double *)p.coef2, *m = (double *)p.m;
    launch(ctx, st, "prior_draw_f64", [&] {
      return launch_prior_draw<double>(C, s->n_grid, s->dSqrtLam, s->dS, p.seed, p.id_base,
                                       STREAM_Z_ID, p.step, Mf, N, st, nullptr, 0, 0, 0, ext_z,
                                       p.da ? p.acc : nullptr);
    });
    launch(ctx, st, "field_coef_f64", [&] {
      return gemm_coef<double>(C, r, N, Mf, N, s->dE, N, p.coef, r, cs, coef2, r, st);
    });
    if (p.da) da_stage(ctx, p, cs, st);
    launch(ctx, st, "field_update_f64", [&] {
      return gemm_field<double>(C, N, r, coef2, r, s->dD, r, p.acc, p.sc, cs, m, Mf, N, st);
    });
  } else {
    // FP32 draw plus its bf16 slices; both projections on the tensor cores
    // with three slices (six products, FP32-level operands)
    float *Mf = (float *)p.Mf, *m = (float *)p.m;
    launch(ctx, st, "prior_draw_f32", [&] {
      return launch_prior_draw<float>(C, s->n_grid, s->fSqrtLam, s->fS, p.seed, p.id_base,
                                      STREAM_Z_ID, p.step, Mf, N, st, p.Ms, s->ldE,
                                      (size_t)C * s->ldE, kFieldSlices, ext_z,
                                      p.da ? p.acc : nullptr);
    });
    launch(ctx, st, "field_coef_tc", [&] {
      // coef2 (C x r) = coef - cs M E^T, written as bf16 slices
      TcGemmArgs g;
      g.M = C;
      g.N = r;
      g.K = N;
      g.A = p.Ms;
      g.lda = s->ldE;
      g.a_plane = (size_t)C * s->ldE;
      g.B = s->bE;
      g.ldb = s->ldE;
      g.b_plane = s->plE;
      g.nslice = kFieldSlices;
      g.epi = TC_EPI_COEF;
      // split-K partials (small pools) in the Jacobian's P buffer, free once
      // the Jacobian is formed
      g.ws = reinterpret_cast<float *>(p.w.Pb[0]);
      g.ws_floats = p.w.Pb[0] ? p.w.plp * s->jac_slices / 2 : 0;
      g.coef = p.coef;
      g.ldc = r;
      g.cs = cs;
      g.out_bf = p.coef2s;
      g.ldo = s->ldD;
      g.out_plane = (size_t)C * s->ldD;
      g.out_slices = kFieldSlices;
      return launch_tc_gemm(g, st);
    });
    if (p.da) da_stage(ctx, p, cs, st);
    launch(ctx, st, "field_update_tc", [&] {
      // (D coef2^T) (N x C), added where accepted: m <- s m + cs M + D coef2
      TcGemmArgs g;
      g.M = N;
      g.N = C;
      g.K = r;
      g.A = s->bD;
      g.lda = s->ldD;
      g.a_plane = s->plD;
      g.B = p.coef2s;
      g.ldb = s->ldD;
      g.b_plane = (size_t)C * s->ldD;
      g.nslice = kFieldSlices;
      g.epi = TC_EPI_FIELD_T;
      g.acc = p.acc;
      g.sc = p.sc;
      g.cs = cs;
      g.m = m;
      g.Mf = Mf;
      g.ldm = N;
      return launch_tc_gemm(g, st);
    });
  }
  p.step += 1;
  p.ext_xi = p.ext_xi2 = p.ext_z = p.ext_log_u = p.ext_log_u2 = false;  // one-shot
}

static void destroy_pool(dino_ctx *ctx, int id) {
  Pool *p = get_pool(ctx, id);
  if (p->ext) {
    cudaStreamSynchronize(p->st);
    dev_free(ctx, p->ext, p->ext_bytes);
    p->ext = nullptr;
  }
  if (p->async_mem) {
    dev_free_async(ctx, p->ar.base, p->ar.bytes, p->st);
  } else {
    cudaStreamSynchronize(p->st);
    dev_free(ctx, p->ar.base, p->ar.bytes);
  }
  p->s->pools -= 1;
  ctx->pools.erase(id);
}

// ---------------------------------------------------------------------------
// surrogate evaluation at caller points (setup / testing entry point)

static void surrogate_eval(dino_ctx *ctx, int sid, int n, const double *x_host, double *f,
                           double *J, double *phi, double *g, double *Lfull, double *hld) {
  Surrogate *s = get_surrogate(ctx, sid);
  if (n < 1 || !x_host) fail(DINO_EINVAL, "need n >= 1 points");
  const int r = s->r, dy = s->d_y;
  Pool p;  // scratch pool-shaped workspace; only the geometry fields are used
  p.s = s;
  p.C = n;
  p.dt = 1.0;
  p.sc = 0.6;
  layout_pool(p, false);
  p.ar.bytes = p.ar.off;
  p.ar.base = (char *)dev_alloc(ctx, p.ar.bytes);
  std::vector<double> yzero;
  double *ysave = s->dy;
  try {
    layout_pool(p, true);
    cudaStream_t st = ctx->stream;
    CK(cudaMemsetAsync(p.err, 0, 16, st));
    CK(cudaMemsetAsync(p.cur, 0, (size_t)n * 4, st));
    if (!s->has_data) {
      // geometry needs some data vector: evaluate against zeros (phi and g then meaningless)
      yzero.assign(dy, 0.0);
      s->dy = (double *)p.Mf;
      CK(cudaMemcpyAsync(s->dy, yzero.data(), dy * 8, cudaMemcpyHostToDevice, st));
    }
    CK(cudaMemcpyAsync(p.b, x_host, (size_t)n * r * 8, cudaMemcpyHostToDevice, st));
    split_input(ctx, s, p.w, p.b, st);
    eval_surrogate(ctx, s, p.w, p.b, st);
    ReducedArgs ra = reduced_args(p);
    ra.noise_var = s->has_data ? s->noise_var : 1.0;
    launch(ctx, st, "geometry_init", [&] { return launch_geometry(ra, 0, st); });
    CK(cudaStreamSynchronize(st));
    std::vector<double> tmp;
    auto fetch = [&](const void *src, size_t cnt, bool f32, double *dst) {
      if (!dst) return;
      if (f32) {
        std::vector<float> t(cnt);
        CK(cudaMemcpy(t.data(), src, cnt * 4, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < cnt; ++i) dst[i] = t[i];
      } else {
        CK(cudaMemcpy(dst, src, cnt * 8, cudaMemcpyDeviceToHost));
      }
    };
    const bool tc = s->precision == DINO_PREC_BF16;
    fetch(tc ? (const void *)p.w.f32 : p.w.f64, (size_t)n * dy, tc, f);
    fetch(tc ? (const void *)p.w.J32 : p.w.J64, (size_t)n * dy * r, tc, J);
    fetch(p.phi, n, false, phi);
    fetch(p.g, (size_t)n * r, false, g);
    fetch(p.hld, n, false, hld);
    if (Lfull) {
      const size_t ts = slot_stride(r);
      std::vector<double> packed((size_t)n * ts);
      CK(cudaMemcpy(packed.data(), p.L, packed.size() * 8, cudaMemcpyDeviceToHost));
      for (int c = 0; c < n; ++c)
        for (int i = 0; i < r; ++i)
          for (int j = 0; j < r; ++j)
            Lfull[(size_t)c * r * r + (size_t)i * r + j] =
                j <= i ? packed[(size_t)c * ts + (size_t)i * (i + 1) / 2 + j] : 0.0;
    }
  } catch (...) {
    s->dy = ysave;
    dev_free(ctx, p.ar.base, p.ar.bytes);
    throw;
  }
  s->dy = ysave;
  dev_free(ctx, p.ar.base, p.ar.bytes);
}

// ---------------------------------------------------------------------------
// derivative-informed subspace from the surrogate's Jacobians (setup)

static void dis_from_surrogate(dino_ctx *ctx, int sid, int n, uint64_t seed, int r_new,
                               double *eig, double *P_out, double *E_out, double *D_out) {
  Surrogate *s = get_surrogate(ctx, sid);
  const int r = s->r, dy = s->d_y, N = s->N;
  if (n < 1 || r_new < 1 || r_new > r) fail(DINO_EINVAL, "need n >= 1 and 1 <= r_new <= r");
  cudaStream_t st = ctx->stream;
  Pool p;  // scratch pool-shaped workspace for the surrogate evaluation at n points
  p.s = s;
  p.C = n;
  p.dt = 1.0;
  p.sc = 0.6;
  layout_pool(p, false);
  p.ar.bytes = p.ar.off;
  const size_t K = (size_t)n * dy, rr = (size_t)r * r;
  const size_t wbytes = (K * r + 4 * rr + r + (size_t)N * r + 2 * (size_t)N * r_new +
                         (size_t)r_new * r) * 8;
  p.ar.base = (char *)dev_alloc(ctx, p.ar.bytes);
  double *w = nullptr;
  try {
    w = (double *)dev_alloc(ctx, wbytes);
    layout_pool(p, true);
    double *At = w, *H = At + K * r, *G = H + rr, *Q = G + rr, *sig = Q + rr, *Et = sig + r + rr,
           *Dn = Et + (size_t)N * r, *En = Dn + (size_t)N * r_new, *PrT = En + (size_t)N * r_new;
    // encoded prior draws m_r ~ N(0, I_r) and the surrogate's Jacobian there
    launch(ctx, st, "normals", [&] { return launch_normals(seed, STREAM_DIS_ID, n, r, p.b, st); });
    split_input(ctx, s, p.w, p.b, st);
    eval_surrogate(ctx, s, p.w, p.b, st);
    const bool tc = s->precision == DINO_PREC_BF16;
    // H_mc = (1/n) sum_i J_i^T J_i / noise_var = At At^T, At = J^T / sqrt(n noise_var)
    launch(ctx, st, "transpose", [&] {
      return launch_transpose((int)K, r, tc ? (const void *)p.w.J32 : (const void *)p.w.J64,
                              tc ? 1 : 0, r, 1.0 / std::sqrt((double)n * s->noise_var), At, st);
    });
    launch(ctx, st, "dis_gram", [&] {
      return gemm_store<double>(r, r, (int)K, At, (int)K, At, (int)K, H, r, st);
    });
    CK(cudaMemcpyAsync(G, H, rr * 8, cudaMemcpyDeviceToDevice, st));
    launch(ctx, st, "jacobi", [&] { return launch_jacobi(r, G, Q, sig, nullptr, st); });
    std::vector<double> lam(r), Qh(rr);
    CK(cudaMemcpyAsync(lam.data(), sig, r * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(Qh.data(), Q, rr * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    // decreasing eigenvalues (H_mc is positive semidefinite: column norms = eigenvalues)
    std::vector<int> order(r);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lam[a] > lam[b]; });
    std::vector<double> prt((size_t)r_new * r);
    for (int i = 0; i < r_new; ++i)
      for (int k = 0; k < r; ++k) prt[(size_t)i * r + k] = Qh[(size_t)order[i] * r + k];
    if (eig)
      for (int i = 0; i < r; ++i) eig[i] = lam[order[i]];
    if (P_out)
      for (int k = 0; k < r; ++k)
        for (int i = 0; i < r_new; ++i) P_out[(size_t)k * r_new + i] = prt[(size_t)i * r + k];
    CK(cudaMemcpyAsync(PrT, prt.data(), prt.size() * 8, cudaMemcpyHostToDevice, st));
    // D' = D P_r' and E' = P_r'^T E
    launch(ctx, st, "dis_basis", [&] {
      return gemm_store<double>(N, r_new, r, s->dD, r, PrT, r, Dn, r_new, st);
    });
    launch(ctx, st, "transpose", [&] { return launch_transpose(r, N, s->dE, 0, N, 1.0, Et, st); });
    launch(ctx, st, "dis_basis", [&] {
      return gemm_store<double>(r_new, N, r, PrT, r, Et, r, En, N, st);
    });
    if (D_out) CK(cudaMemcpyAsync(D_out, Dn, (size_t)N * r_new * 8, cudaMemcpyDeviceToHost, st));
    if (E_out) CK(cudaMemcpyAsync(E_out, En, (size_t)N * r_new * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  } catch (...) {
    cudaStreamSynchronize(st);
    if (w) dev_free(ctx, w, wbytes);
    dev_free(ctx, p.ar.base, p.ar.bytes);
    throw;
  }
  dev_free(ctx, w, wbytes);
  dev_free(ctx, p.ar.base, p.ar.bytes);
}

// ---------------------------------------------------------------------------
// chain diagnostics: a device trajectory of n_c chains x d degrees of freedom

struct Diag {
  int id = 0, n_c = 0, d = 0, max_s = 0, n_s = 0;
  double *traj = nullptr, *means = nullptr, *ess = nullptr, *sqjump = nullptr;
  size_t bytes = 0;
  cudaEvent_t ready = nullptr;  // recorded after the last append
};

static Diag *get_diag(dino_ctx *ctx, int id) {
  auto it = ctx->diags.find(id);
  if (it == ctx->diags.end()) fail(DINO_ENOTFOUND, "unknown diagnostics id %d", id);
  return it->second.get();
}

static void free_diag(dino_ctx *ctx, Diag *g) {
  if (g->ready) {
    cudaEventSynchronize(g->ready);
    cudaEventDestroy(g->ready);
  }
  dev_free(ctx, g->traj, g->bytes);
}

static int diag_create(dino_ctx *ctx, int n_c, int d, int max_s) {
  if (n_c < 2 || d < 1 || max_s < 2 || n_c > 6144)
    fail(DINO_EINVAL, "diagnostics need 2 <= n_chains <= 6144, n_dof >= 1, max_samples >= 2");
  auto g = std::make_unique<Diag>();
  g->id = ctx->next_id++;
  g->n_c = n_c;
  g->d = d;
  g->max_s = max_s;
  const size_t nt = (size_t)d * n_c * max_s, nm = (size_t)d * n_c;
  g->bytes = (nt + nm + 2 * (size_t)d) * sizeof(double);
  g->traj = (double *)dev_alloc(ctx, g->bytes);
  g->means = g->traj + nt;
  g->ess = g->means + nm;
  g->sqjump = g->ess + d;
  if (cudaEventCreateWithFlags(&g->ready, cudaEventDisableTiming) != cudaSuccess) {
    dev_free(ctx, g->traj, g->bytes);
    fail(DINO_ECUDA, "cudaEventCreate failed");
  }
  const int id = g->id;
  ctx->diags[id] = std::move(g);
  return id;
}

// Append the current state of chains [chain0, chain0 + n_c) of a pool.
static void diag_record(dino_ctx *ctx, Diag *g, Pool *p, int what, int chain0) {
  const Surrogate *s = p->s;
  if (g->n_s >= g->max_s) fail(DINO_ENOMEM, "diagnostics trajectory is full (%d samples)", g->max_s);
  if (chain0 < 0 || chain0 + g->n_c > p->C) fail(DINO_EINVAL, "chains out of the pool's range");
  const void *src;
  int f32 = 0, ld;
  if (what == DINO_DIAG_REDUCED) {
    if (g->d != s->r) fail(DINO_EINVAL, "n_dof %d != r %d", g->d, s->r);
    src = p->mr + (size_t)chain0 * s->r;
    ld = s->r;
  } else if (what == DINO_DIAG_FIELD) {
    if (g->d != s->N) fail(DINO_EINVAL, "n_dof %d != N %d", g->d, s->N);
    f32 = s->precision == DINO_PREC_FP64 ? 0 : 1;
    src = (const char *)p->m + (size_t)chain0 * s->N * (f32 ? 4 : 8);
    ld = s->N;
  } else {
    fail(DINO_EINVAL, "unknown record kind %d", what);
  }
  launch(ctx, p->st, "diag_record", [&] {
    return launch_diag_record(g->n_c, g->d, src, f32, ld, g->traj, g->max_s, g->n_s, p->st);
  });
  CK(cudaEventRecord(g->ready, p->st));
  g->n_s += 1;
}

static void diag_push(dino_ctx *ctx, Diag *g, const double *sample) {
  if (!sample) fail(DINO_EINVAL, "sample is NULL");
  if (g->n_s >= g->max_s) fail(DINO_ENOMEM, "diagnostics trajectory is full (%d samples)", g->max_s);
  const size_t n = (size_t)g->n_c * g->d;
  double *tmp = (double *)dev_alloc(ctx, n * 8);
  try {
    CK(cudaMemcpyAsync(tmp, sample, n * 8, cudaMemcpyHostToDevice, ctx->stream));
    launch(ctx, ctx->stream, "diag_record", [&] {
      return launch_diag_record(g->n_c, g->d, tmp, 0, g->d, g->traj, g->max_s, g->n_s,
                                ctx->stream);
    });
    CK(cudaStreamSynchronize(ctx->stream));
  } catch (...) {
    dev_free(ctx, tmp, n * 8);
    throw;
  }
  dev_free(ctx, tmp, n * 8);
  g->n_s += 1;
}

static void diag_compute(dino_ctx *ctx, Diag *g, int want_mpsrf, double *ess_out,
                         dino_diag_result *res) {
  const int n_c = g->n_c, d = g->d, n_s = g->n_s;
  if (n_s < 2) fail(DINO_ESTATE, "need at least 2 recorded samples (have %d)", n_s);
  if (want_mpsrf && d > 1024) fail(DINO_EINVAL, "MPSRF needs n_dof <= 1024 (have %d)", d);
  cudaStream_t st = ctx->stream;
  CK(cudaStreamWaitEvent(st, g->ready, 0));
  launch(ctx, st, "diag_ess", [&] {
    return launch_diag_ess(d, n_c, n_s, g->traj, g->max_s, g->means, g->ess, g->sqjump, st);
  });
  std::vector<double> ess(d), sj(d);
  CK(cudaMemcpyAsync(ess.data(), g->ess, d * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(sj.data(), g->sqjump, d * 8, cudaMemcpyDeviceToHost, st));
  double out[3] = {0, 0, 0};
  int sweeps = 0;
  if (want_mpsrf) {
    const size_t K = (size_t)n_c * n_s, dd = (size_t)d * d;
    const size_t bytes = ((size_t)d * K + (size_t)d * n_c + 9 * dd + d + 4) * 8;
    double *w = (double *)dev_alloc(ctx, bytes);
    try {
      double *Xc = w, *Mc = Xc + (size_t)d * K, *Wr = Mc + (size_t)d * n_c, *Br = Wr + dd,
             *W = Br + dd, *V = W + dd, *G = V + dd, *Q = G + dd, *Wh = Q + dd, *T = Wh + dd,
             *M = T + dd, *sig = M + dd, *o = sig + d;
      launch(ctx, st, "diag_center", [&] {
        return launch_diag_center(d, n_c, n_s, g->traj, g->max_s, g->means, Xc, Mc, st);
      });
      launch(ctx, st, "diag_gram", [&] {
        return gemm_store<double>(d, d, (int)K, Xc, (int)K, Xc, (int)K, Wr, d, st);
      });
      launch(ctx, st, "diag_gram", [&] {
        return gemm_store<double>(d, d, n_c, Mc, n_c, Mc, n_c, Br, d, st);
      });
      launch(ctx, st, "diag_wv", [&] { return launch_diag_wv(d, n_c, n_s, Wr, Br, W, V, st); });
      // W = Q diag(lam) Q^T (W symmetric: its rows are its columns)
      CK(cudaMemcpyAsync(G, W, dd * 8, cudaMemcpyDeviceToDevice, st));
      launch(ctx, st, "jacobi", [&] { return launch_jacobi(d, G, Q, sig, nullptr, st); });
      launch(ctx, st, "sym_sqrt", [&] { return launch_sym_sqrt(d, Q, sig, Wh, st); });
      launch(ctx, st, "small_mm", [&] { return launch_small_mm(d, Wh, V, T, st); });
      launch(ctx, st, "small_mm", [&] { return launch_small_mm(d, T, Wh, M, st); });
      // eigenvalues of W^1/2 V W^1/2 (symmetric positive semidefinite)
      launch(ctx, st, "jacobi", [&] {
        return launch_jacobi(d, M, nullptr, sig, reinterpret_cast<int *>(o + 3), st);
      });
      launch(ctx, st, "mpsrf_final", [&] { return launch_mpsrf_final(d, W, V, sig, o, st); });
      CK(cudaMemcpyAsync(out, o, 24, cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(&sweeps, o + 3, 4, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    } catch (...) {
      cudaStreamSynchronize(st);
      dev_free(ctx, w, bytes);
      throw;
    }
    dev_free(ctx, w, bytes);
  }
  CK(cudaStreamSynchronize(st));
  if (ess_out) std::memcpy(ess_out, ess.data(), d * 8);
  if (res) {
    double msj = 0.0;
    for (double x : sj) msj += x;
    res->n_samples = n_s;
    res->msj = msj / ((double)n_c * (n_s - 1));
    res->mpsrf_w = want_mpsrf ? out[0] : std::nan("");
    res->trace_w = want_mpsrf ? out[1] : std::nan("");
    res->trace_v = want_mpsrf ? out[2] : std::nan("");
    res->jacobi_sweeps = sweeps;
    double e = 0.0;
    std::vector<double> sorted(ess);
    std::sort(sorted.begin(), sorted.end());
    e = d % 2 ? sorted[d / 2] : 0.5 * (sorted[d / 2 - 1] + sorted[d / 2]);
    res->ess_median = e;
  }
}

// ---------------------------------------------------------------------------
// serving: continuous batching of chain ensembles
//
// A background thread owns admission and issue.  Requests wait in a queue
// until their pool's device footprint fits the context's HBM budget (the
// least estimated work first, requests older than starve_s before all); each
// admitted request gets its own pool on one of several CUDA streams, and its
// transitions are issued in rounds of `steps_per_round` with at most two
// rounds in flight, so requests that arrive while others run join between
// rounds and their kernels overlap on the device.  A request's results depend
// only on its surrogate, seed, chain ids, step count and initial fields, not
// on what else is running.

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  uint64_t ticket = 0;
  dino_request req{};
  std::vector<double> m0;
  size_t footprint = 0;
  double work = 0;  // estimated cost: proposals x per-proposal work of the surrogate
  double t_submit = 0, t_admit = 0, t_done = 0;
  int state = 0;  // 0 queued, 1 active, 2 done, 3 failed
  int status = DINO_OK;
  std::string err;
  Pool *pool = nullptr;
  int issued = 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int ev_issued[2] = {0, 0};  // steps issued when each event was recorded
  int in_flight = 0, next_ev = 0;
  dino_step_stats stats{};
};

struct Server {
  dino_ctx *ctx;
  std::thread th;
  std::condition_variable_any cv;
  bool stop = false;
  std::deque<Request *> queue;
  std::vector<Request *> active;
  std::map<uint64_t, std::unique_ptr<Request>> reqs;
  std::vector<cudaStream_t> streams;
  std::vector<int> load;          // resident requests per stream
  std::vector<int> stream_rounds; // rounds in flight per stream
  int steps_per_round = 8;
  int max_active = 32;
  size_t max_queue = 100000;
  // admission order: requests that have waited longer than starve_s first
  // (oldest first), then the others by estimated work, smallest first
  double starve_s = 20.0;
  // an internal error outside any one request stops the server: every
  // resident and queued request fails with it and submit refuses new ones
  bool broken = false;
  int broken_code = DINO_OK;
  std::string broken_msg;
  uint64_t next_ticket = 1;
  int peak_active = 0;
  size_t peak_used = 0;

  Server(dino_ctx *c, int nstreams, int spr, int max_act)
      : ctx(c), steps_per_round(spr), max_active(max_act) {
    for (int k = 0; k < nstreams; ++k) {
      cudaStream_t st;
      CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      streams.push_back(st);
      load.push_back(0);
      stream_rounds.push_back(0);
    }
    th = std::thread([this] { loop(); });
  }

  // After the thread has stopped: free the pools still resident (on their
  // live streams), then the events and streams.
  void release() {
    for (auto &kv : reqs) {
      Request *r = kv.second.get();
      if (r->pool) {
        const int id = r->pool->id;
        cudaStreamSynchronize(r->pool->st);
        try {
          destroy_pool(ctx, id);
        } catch (...) {
        }
        r->pool = nullptr;
      }
      for (cudaEvent_t e : r->ev)
        if (e) cudaEventDestroy(e);
      r->ev[0] = r->ev[1] = nullptr;
    }
    for (cudaStream_t st : streams) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
    streams.clear();
  }

  void fail_request(Request *r, int code, const std::string &msg) {
    r->state = 3;
    r->status = code;
    r->err = msg;
    r->t_done = now_s();
    if (r->pool) {
      const int id = r->pool->id;
      for (size_t k = 0; k < streams.size(); ++k)
        if (streams[k] == r->pool->st) {
          load[k] -= 1;
          stream_rounds[k] -= r->in_flight;
        }
      r->in_flight = 0;
      cudaStreamSynchronize(r->pool->st);
      try {
        destroy_pool(ctx, id);
      } catch (...) {
      }
      r->pool = nullptr;
    }
  }

  void finish(Request *r) {
    Pool *p = r->pool;
    const int C = p->C, rr = p->s->r, N = p->s->N;
    CK(cudaStreamSynchronize(p->st));
    unsigned long long c[3];
    double a = 0;
    int err = 0;
    CK(cudaMemcpy(c, p->counters, 24, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&a, p->sum_alpha, 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&err, p->err, 4, cudaMemcpyDeviceToHost));
    if (err) fail(DINO_ETIMEOUT, "a device wait gave up (code %d)", err);
    if (r->req.m_r_out)
      CK(cudaMemcpy(r->req.m_r_out, p->mr, (size_t)C * rr * 8, cudaMemcpyDeviceToHost));
    if (r->req.phi_out) CK(cudaMemcpy(r->req.phi_out, p->phi, (size_t)C * 8, cudaMemcpyDeviceToHost));
    if (r->req.accepts_out)
      CK(cudaMemcpy(r->req.accepts_out, p->acc_count, (size_t)C * 8, cudaMemcpyDeviceToHost));
    if (r->req.m_out) {
      if (p->s->precision == DINO_PREC_FP64) {
        CK(cudaMemcpy(r->req.m_out, p->m, (size_t)C * N * 8, cudaMemcpyDeviceToHost));
      } else {
        std::vector<float> t((size_t)C * N);
        CK(cudaMemcpy(t.data(), p->m, t.size() * 4, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < t.size(); ++i) r->req.m_out[i] = t[i];
      }
    }
    r->stats.proposals = (uint64_t)C * (uint64_t)r->req.n_steps;
    r->stats.accepts = c[0];
    r->stats.nan_rejects = c[1];
    r->stats.sum_alpha = a;
    r->stats.stage1_accepts = c[2];
    const int id = p->id;
    for (size_t k = 0; k < streams.size(); ++k)
      if (streams[k] == p->st) load[k] -= 1;
    destroy_pool(ctx, id);
    r->pool = nullptr;
    r->state = 2;
    r->t_done = now_s();
  }

  // One scheduling pass under the context lock; true when it did any work.
  bool pass() {
    bool did = false;
    // completed rounds and requests
    for (size_t k = 0; k < active.size();) {
      Request *r = active[k];
      bool removed = false;
      while (r->in_flight > 0) {
        const int slot = (r->next_ev + 2 - r->in_flight) % 2;
        const cudaError_t q = cudaEventQuery(r->ev[slot]);
        if (q == cudaErrorNotReady) break;
        r->in_flight -= 1;
        for (size_t j = 0; j < streams.size(); ++j)
          if (r->pool && streams[j] == r->pool->st) stream_rounds[j] -= 1;
        did = true;
        if (q != cudaSuccess) {
          cudaGetLastError();
          fail_request(r, DINO_ECUDA, cudaGetErrorString(q));
          removed = true;
          break;
        }
      }
      if (!removed && r->in_flight == 0 && r->issued >= r->req.n_steps) {
        try {
          finish(r);
        } catch (const Error &e) {
          fail_request(r, e.code, e.msg);
        }
        removed = true;
        did = true;
      }
      if (removed) {
        active.erase(active.begin() + k);
      } else {
        ++k;
      }
    }
    // admission: shortest estimated job first among the requests that fit
    // the free budget (first fit), except that requests waiting longer than
    // starve_s go first in arrival order, and while the oldest of them does
    // not fit nothing else is admitted (it cannot be passed over forever)
    const double tnow = now_s();
    std::vector<Request *> order(queue.begin(), queue.end());
    std::stable_sort(order.begin(), order.end(), [&](const Request *a, const Request *b) {
      const bool sa = tnow - a->t_submit > starve_s, sb = tnow - b->t_submit > starve_s;
      if (sa != sb) return sa;
      if (sa) return a->ticket < b->ticket;
      return a->work < b->work;
    });
    for (Request *r : order) {
      if ((int)active.size() >= max_active) break;
      if (ctx->used + r->footprint > ctx->budget) {
        if (tnow - r->t_submit > starve_s) break;  // the starved request goes next
        continue;
      }
      queue.erase(std::find(queue.begin(), queue.end(), r));
      int k = 0;
      for (size_t j = 1; j < streams.size(); ++j)
        if (load[j] < load[k]) k = (int)j;
      try {
        r->pool = create_pool_on(ctx, r->req.surrogate_id, r->req.n_chains, r->req.dt,
                                 r->req.seed, r->req.chain_id_base,
                                 r->m0.empty() ? nullptr : r->m0.data(), streams[k], true);
        load[k] += 1;
        for (int e = 0; e < 2; ++e)
          if (!r->ev[e]) CK(cudaEventCreateWithFlags(&r->ev[e], cudaEventDisableTiming));
        r->state = 1;
        r->t_admit = now_s();
        active.push_back(r);
      } catch (const Error &e) {
        fail_request(r, e.code, e.msg);
      }
      did = true;
    }
    // issue rounds: at most two in flight per request and per stream, so the
    // launch queues stay short and this thread never blocks in a launch.
    // Only as many residents as there are streams progress at a time, those
    // with the least remaining work (under overload this lets short requests
    // finish instead of sharing the device evenly with long ones).
    std::vector<Request *> prog(active.begin(), active.end());
    auto remaining = [](const Request *r) {
      return r->work * (double)(r->req.n_steps - r->issued) / std::max(1, r->req.n_steps);
    };
    std::stable_sort(prog.begin(), prog.end(), [&](const Request *a, const Request *b) {
      return remaining(a) < remaining(b);
    });
    int progressing = 0;
    for (Request *r : prog) {
      if (r->issued >= r->req.n_steps) continue;
      if (progressing++ >= (int)streams.size()) break;
      if (r->in_flight >= 2) continue;
      size_t sj = 0;
      for (size_t j = 0; j < streams.size(); ++j)
        if (streams[j] == r->pool->st) sj = j;
      if (stream_rounds[sj] >= 2) continue;
      const int k = std::min(steps_per_round, r->req.n_steps - r->issued);
      try {
        for (int s = 0; s < k; ++s) step_pool(ctx, *r->pool);
        CK(cudaEventRecord(r->ev[r->next_ev], r->pool->st));
      } catch (const Error &e) {
        fail_request(r, e.code, e.msg);
        continue;
      }
      r->issued += k;
      r->next_ev ^= 1;
      r->in_flight += 1;
      stream_rounds[sj] += 1;
      did = true;
    }
    active.erase(std::remove_if(active.begin(), active.end(),
                                [](Request *r) { return r->state == 3; }),
                 active.end());
    peak_active = std::max(peak_active, (int)active.size());
    peak_used = std::max(peak_used, ctx->used);
    return did;
  }

  // Fails every resident and queued request with `code` and stops admission.
  void break_down(int code, const std::string &msg) {
    broken = true;
    broken_code = code;
    broken_msg = msg;
    for (Request *r : active)
      if (r->state == 1) fail_request(r, code, "serving stopped: " + msg);
    active.clear();
    for (Request *r : queue) {
      r->state = 3;
      r->status = code;
      r->err = "serving stopped before admission: " + msg;
      r->t_done = now_s();
    }
    queue.clear();
  }

  void loop() {
    std::unique_lock<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    while (!stop) {
      bool did = false;
      if (!broken) {
        try {
          did = pass();
        } catch (const Error &e) {
          break_down(e.code, e.msg);
        } catch (const std::exception &e) {
          break_down(DINO_ECUDA, std::string("internal error: ") + e.what());
        } catch (...) {
          break_down(DINO_ECUDA, "unknown internal error");
        }
      }
      if (!did) {
        cv.wait_for(lk, std::chrono::microseconds(200));
      } else {
        lk.unlock();
        std::this_thread::yield();
        lk.lock();
      }
    }
  }
};

static void stop_server(dino_ctx *ctx) {
  if (!ctx->server) return;
  {
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    ctx->server->stop = true;
  }
  ctx->server->cv.notify_all();
  if (ctx->server->th.joinable()) ctx->server->th.join();
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  ctx->server->release();
  ctx->server.reset();
}

}  // namespace dino

// ===========================================================================
// C ABI
using namespace dino;

template <class F>
static int guarded(dino_ctx *ctx, F &&fn) {
  if (!ctx) return DINO_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  ctx->err.clear();
  try {
    fn();
    return DINO_OK;
  } catch (const Error &e) {
    ctx->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc &) {
    ctx->err = "host allocation failed";
    return DINO_ENOMEM;
  } catch (...) {
    ctx->err = "unexpected internal error";
    return DINO_ECUDA;
  }
}

extern "C" {

int dino_version(void) { return 101; }

int dino_init(dino_ctx **out, int device, size_t hbm_budget_bytes, void *stream,
              unsigned flags) {
  if (!out) return DINO_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= device || device < 0) {
    cudaGetLastError();
    return DINO_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return DINO_ECUDA;
  auto ctx = new dino_ctx();
  ctx->device = device;
  ctx->flags = flags;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    delete ctx;
    return DINO_ECUDA;
  }
  ctx->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)fr);
  int pma = 0;
  if (!(flags & DINO_FLAG_NO_DIRECT_HOST) &&
      cudaDeviceGetAttribute(&pma, cudaDevAttrPageableMemoryAccess, device) == cudaSuccess)
    ctx->pageable_access = pma != 0;
  if (stream) {
    ctx->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return DINO_ECUDA;
    }
    ctx->own_stream = true;
  }
  *out = ctx;
  return DINO_OK;
}

int dino_destroy(dino_ctx *ctx) {
  if (!ctx) return DINO_EINVAL;
  stop_server(ctx);
  {
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto &kv : ctx->pools) {
      dev_free(ctx, kv.second->ar.base, kv.second->ar.bytes);
      dev_free(ctx, kv.second->ext, kv.second->ext_bytes);
    }
    ctx->pools.clear();
    for (auto &kv : ctx->diags) free_diag(ctx, kv.second.get());
    ctx->diags.clear();
    for (auto &kv : ctx->surrogates) free_surrogate(ctx, kv.second.get());
    ctx->surrogates.clear();
    for (auto &p : ctx->pending) {
      cudaEventDestroy(p.e0);
      cudaEventDestroy(p.e1);
    }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    for (auto st : ctx->aux_streams) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  }
  delete ctx;
  return DINO_OK;
}

const char *dino_last_error(const dino_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int dino_sync(dino_ctx *ctx) {
  return guarded(ctx, [&] {
    cudaSetDevice(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
  });
}

int dino_load_surrogate(dino_ctx *ctx, const dino_surrogate_desc *desc, int *surrogate_id) {
  return guarded(ctx, [&] {
    if (!surrogate_id) fail(DINO_EINVAL, "surrogate_id is NULL");
    cudaSetDevice(ctx->device);
    *surrogate_id = load_surrogate(ctx, desc);
  });
}

int dino_set_data(dino_ctx *ctx, int surrogate_id, const double *y, double noise_var) {
  return guarded(ctx, [&] {
    cudaSetDevice(ctx->device);
    Surrogate *s = get_surrogate(ctx, surrogate_id);
    if (!y) fail(DINO_EINVAL, "y is NULL");
    if (!(noise_var > 0) || !std::isfinite(noise_var)) fail(DINO_EINVAL, "noise_var must be > 0");
    if (s->pools > 0) fail(DINO_ESTATE, "surrogate has live chain pools");
    for (int i = 0; i < s->d_y; ++i)
      if (!std::isfinite(y[i])) fail(DINO_ENUMERIC, "non-finite data value");
    s->y.assign(y, y + s->d_y);
    s->noise_var = noise_var;
    s->has_data = true;
    upload_data(ctx, s);
  });
}

int dino_unload_surrogate(dino_ctx *ctx, int surrogate_id) {
  return guarded(ctx, [&] {
    cudaSetDevice(ctx->device);
    Surrogate *s = get_surrogate(ctx, surrogate_id);
    if (s->pools > 0) fail(DINO_ESTATE, "surrogate has live chain pools");
    free_surrogate(ctx, s);
    ctx->surrogates.erase(surrogate_id);
  });
}

int dino_read_basis(dino_ctx *ctx, int surrogate_id, double *E, double *D) {
  return guarded(ctx, [&] {
    Surrogate *s = get_surrogate(ctx, surrogate_id);
    if (E) std::memcpy(E, s->E.data(), s->E.size() * 8);
    if (D) std::memcpy(D, s->D.data(), s->D.size() * 8);
  });
}

int dino_surrogate_eval(dino_ctx *ctx, int surrogate_id, int n, const double *m_r, double *f,
                        double *J, double *phi, double *g, double *L, double *hld) {
  return guarded(ctx, [&] {
    cudaSetDevice(ctx->device);
    surrogate_eval(ctx, surrogate_id, n, m_r, f, J, phi, g, L, hld);
    collect_times(ctx);
  });
}

int dino_chains_create(dino_ctx *ctx, int surrogate_id, int n_chains, double dt, uint64_t seed,
                       uint64_t chain_id_base, const double *m0, int *pool_id) {
  return guarded(ctx, [&] {
    if (!pool_id) fail(DINO_EINVAL, "pool_id is NULL");
    cudaSetDevice(ctx->device);
    *pool_id = create_pool(ctx, surrogate_id, n_chains, dt, seed, chain_id_base, m0);
    collect_times(ctx);
  });
}

int dino_chains_step(dino_ctx *ctx, int pool_id, int n_steps, dino_step_stats *stats) {
  return guarded(ctx, [&] {
    if (n_steps < 0) fail(DINO_EINVAL, "n_steps must be >= 0");
    cudaSetDevice(ctx->device);
    Pool *p = get_pool(ctx, pool_id);
    unsigned long long c0[3] = {0, 0, 0};
    double a0 = 0;
    if (stats) {
      CK(cudaMemcpyAsync(c0, p->counters, 24, cudaMemcpyDeviceToHost, p->st));
      CK(cudaMemcpyAsync(&a0, p->sum_alpha, 8, cudaMemcpyDeviceToHost, p->st));
    }
    for (int k = 0; k < n_steps; ++k) step_pool(ctx, *p);
    if (stats) {
      unsigned long long c1[3];
      double a1 = 0;
      int err = 0;
      CK(cudaMemcpyAsync(c1, p->counters, 24, cudaMemcpyDeviceToHost, p->st));
      CK(cudaMemcpyAsync(&a1, p->sum_alpha, 8, cudaMemcpyDeviceToHost, p->st));
      CK(cudaMemcpyAsync(&err, p->err, 4, cudaMemcpyDeviceToHost, p->st));
      CK(cudaStreamSynchronize(p->st));
      if (err) fail(DINO_ETIMEOUT, "a device wait gave up (code %d); the pool state is invalid", err);
      stats->proposals = (uint64_t)p->C * (uint64_t)n_steps;
      stats->accepts = c1[0] - c0[0];
      stats->nan_rejects = c1[1] - c0[1];
      stats->sum_alpha = a1 - a0;
      stats->stage1_accepts = c1[2] - c0[2];
    }
    collect_times(ctx);
  });
}

int dino_chains_step_many(dino_ctx *ctx, int n_pools, const int *pool_ids, int n_steps) {
  return guarded(ctx, [&] {
    if (n_pools < 1 || !pool_ids || n_steps < 0) fail(DINO_EINVAL, "need pools and n_steps >= 0");
    cudaSetDevice(ctx->device);
    std::vector<Pool *> ps;
    for (int i = 0; i < n_pools; ++i) {
      Pool *p = get_pool(ctx, pool_ids[i]);
      if (p->async_mem) fail(DINO_EINVAL, "pool %d belongs to the serving loop", pool_ids[i]);
      for (Pool *q : ps)
        if (q == p) fail(DINO_EINVAL, "pool %d listed twice", pool_ids[i]);
      ps.push_back(p);
    }
    constexpr int kMaxAux = 16;
    while ((int)ctx->aux_streams.size() < std::min(n_pools, kMaxAux)) {
      cudaStream_t st;
      CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      ctx->aux_streams.push_back(st);
    }
    // each pool moves to its own stream after the work already on its stream,
    // steps there (issue interleaved over pools so that all streams fill), and
    // its own stream waits for the result
    std::vector<cudaStream_t> home(n_pools);
    std::vector<cudaEvent_t> evs;
    auto event_on = [&](cudaStream_t st) {
      cudaEvent_t e;
      CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      evs.push_back(e);
      CK(cudaEventRecord(e, st));
      return e;
    };
    try {
      for (int i = 0; i < n_pools; ++i) {
        home[i] = ps[i]->st;
        cudaStream_t aux = ctx->aux_streams[i % ctx->aux_streams.size()];
        CK(cudaStreamWaitEvent(aux, event_on(home[i]), 0));
        ps[i]->st = aux;
      }
      for (int k = 0; k < n_steps; ++k)
        for (Pool *p : ps) step_pool(ctx, *p);
    } catch (...) {
      for (int i = 0; i < n_pools; ++i)
        if (home[i]) {
          cudaStreamWaitEvent(home[i], event_on(ps[i]->st), 0);
          ps[i]->st = home[i];
        }
      for (cudaEvent_t e : evs) cudaEventDestroy(e);
      throw;
    }
    for (int i = 0; i < n_pools; ++i) {
      CK(cudaStreamWaitEvent(home[i], event_on(ps[i]->st), 0));
      ps[i]->st = home[i];
    }
    for (cudaEvent_t e : evs) cudaEventDestroy(e);
    collect_times(ctx);
  });
}

int dino_measure_fp32_peak(dino_ctx *ctx, double *tflops) {
  return guarded(ctx, [&] {
    if (!tflops) fail(DINO_EINVAL, "tflops is NULL");
    cudaSetDevice(ctx->device);
    float ms = 0;
    double f = 0;
    CK(measure_fma_peak(ctx->stream, &ms, &f));
    if (!(ms > 0)) fail(DINO_ECUDA, "the FMA timing returned no time");
    *tflops = f / (ms * 1e-3) / 1e12;
  });
}

int dino_chains_read(dino_ctx *ctx, int pool_id, double *m, double *m_r, double *phi,
                     uint64_t *accepts) {
  return guarded(ctx, [&] {
    cudaSetDevice(ctx->device);
    Pool *p = get_pool(ctx, pool_id);
    const int C = p->C, r = p->s->r, N = p->s->N;
    int err = 0;
    CK(cudaMemcpyAsync(&err, p->err, 4, cudaMemcpyDeviceToHost, p->st));
    CK(cudaStreamSynchronize(p->st));
    if (err) fail(DINO_ETIMEOUT, "a device wait gave up (code %d); the pool state is invalid", err);
    if (m) {
      if (p->s->precision == DINO_PREC_FP64) {
        CK(cudaMemcpy(m, p->m, (size_t)C * N * 8, cudaMemcpyDeviceToHost));
      } else {
        std::vector<float> t((size_t)C * N);
        CK(cudaMemcpy(t.data(), p->m, t.size() * 4, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < t.size(); ++i) m[i] = t[i];
      }
    }
    if (m_r) CK(cudaMemcpy(m_r, p->mr, (size_t)C * r * 8, cudaMemcpyDeviceToHost));
    if (phi) CK(cudaMemcpy(phi, p->phi, (size_t)C * 8, cudaMemcpyDeviceToHost));
    if (accepts) CK(cudaMemcpy(accepts, p->acc_count, (size_t)C * 8, cudaMemcpyDeviceToHost));
  });
}

int dino_chains_read_last(dino_ctx *ctx, int pool_id, double *b, double *mu, double *log_rho,
                          double *log_u, int *accepted) {
  return guarded(ctx, [&] {
    cudaSetDevice(ctx->device);
    Pool *p = get_pool(ctx, pool_id);
    const int C = p->C, r = p->s->r;
    CK(cudaStreamSynchronize(p->st));
    if (b) CK(cudaMemcpy(b, p->b, (size_t)C * r * 8, cudaMemcpyDeviceToHost));
    if (mu) CK(cudaMemcpy(mu, p->mu, (size_t)C * r * 8, cudaMemcpyDeviceToHost));
    if (log_rho) CK(cudaMemcpy(log_rho, p->log_rho, (size_t)C * 8, cudaMemcpyDeviceToHost));
    if (log_u) CK(cudaMemcpy(log_u, p->log_u, (size_t)C * 8, cudaMemcpyDeviceToHost));
    if (accepted) CK(cudaMemcpy(accepted, p->acc, (size_t)C * 4, cudaMemcpyDeviceToHost));
  });
}

int dino_surrogate_query(dino_ctx *ctx, int surrogate_id, dino_surrogate_info *info) {
  return guarded(ctx, [&] {
    if (!info) fail(DINO_EINVAL, "info is NULL");
    const Surrogate *s = get_surrogate(ctx, surrogate_id);
    info->N = s->N;
    info->r = s->r;
    info->d_y = s->d_y;
    info->n_layers = s->L;
    info->precision = s->precision;
    info->noise_map = s->eig ? DINO_NOISE_EIGEN
                      : s->wb ? DINO_NOISE_PERTURBATION : DINO_NOISE_CHOLESKY;
    info->gram_on_tensor_cores = s->tc_gram ? 1 : 0;
    info->fwd_slices = s->precision == DINO_PREC_BF16 ? s->fwd_slices : 0;
    info->jac_slices = s->precision == DINO_PREC_BF16 ? s->jac_slices : 0;
    info->true_model_rank = s->tm.on ? s->tm.r_t : 0;
    info->jac_forward = s->jac_fwd ? 1 : 0;
  });
}

int dino_chains_set_noise(dino_ctx *ctx, int pool_id, const double *xi, const double *xi2,
                          const double *z, const double *log_u, const double *log_u2) {
  return guarded(ctx, [&] {
    cudaSetDevice(ctx->device);
    Pool *p = get_pool(ctx, pool_id);
    const Surrogate *s = p->s;
    if (xi2 && !p->wb)
      fail(DINO_EINVAL, "xi2 is only drawn by the perturbation noise map (this pool: Cholesky)");
    const size_t C = p->C, r = s->r, dy = s->d_y, N = s->N;
    if (log_u2 && !p->da)
      fail(DINO_EINVAL, "log_u2 is only drawn by delayed acceptance (no true model)");
    const size_t bytes = C * (r + dy + N + 2) * sizeof(double);
    if (!p->ext) {
      p->ext = (double *)dev_alloc(ctx, bytes);
      p->ext_bytes = bytes;
    }
    auto put = [&](const double *src, size_t off, size_t n) {
      CK(cudaMemcpyAsync(p->ext + off, src, n * sizeof(double), cudaMemcpyHostToDevice, p->st));
    };
    if (xi) put(xi, 0, C * r);
    if (xi2) put(xi2, C * r, C * dy);
    if (z) put(z, C * (r + dy), C * N);
    if (log_u) put(log_u, C * (r + dy + N), C);
    if (log_u2) put(log_u2, C * (r + dy + N + 1), C);
    CK(cudaStreamSynchronize(p->st));  // host arrays are not used after return
    p->ext_xi = xi != nullptr;
    p->ext_xi2 = xi2 != nullptr;
    p->ext_z = z != nullptr;
    p->ext_log_u = log_u != nullptr;
    p->ext_log_u2 = log_u2 != nullptr;
  });
}

int dino_set_true_model(dino_ctx *ctx, int surrogate_id, const dino_true_model_desc *desc) {
  return guarded(ctx, [&] {
    cudaSetDevice(ctx->device);
    set_true_model(ctx, get_surrogate(ctx, surrogate_id), desc);
  });
}

int dino_chains_read_da(dino_ctx *ctx, int pool_id, double *phi_true, double *log_rho2,
                        double *log_u2, int *stage1) {
  return guarded(ctx, [&] {
    cudaSetDevice(ctx->device);
    Pool *p = get_pool(ctx, pool_id);
    if (!p->da) fail(DINO_ESTATE, "pool %d does not run delayed acceptance", pool_id);
    const size_t C = p->C;
    CK(cudaStreamSynchronize(p->st));
    if (phi_true) CK(cudaMemcpy(phi_true, p->phi_t, C * 8, cudaMemcpyDeviceToHost));
    if (log_rho2) CK(cudaMemcpy(log_rho2, p->lr2, C * 8, cudaMemcpyDeviceToHost));
    if (log_u2) CK(cudaMemcpy(log_u2, p->lu2, C * 8, cudaMemcpyDeviceToHost));
    if (stage1) CK(cudaMemcpy(stage1, p->st1, C * 4, cudaMemcpyDeviceToHost));
  });
}

int dino_dis_from_surrogate(dino_ctx *ctx, int surrogate_id, int n_samples, uint64_t seed,
                            int r_new, double *eigvals, double *P, double *E_new, double *D_new) {
  return guarded(ctx, [&] {
    cudaSetDevice(ctx->device);
    dis_from_surrogate(ctx, surrogate_id, n_samples, seed, r_new, eigvals, P, E_new, D_new);
  });
}

int dino_diag_create(dino_ctx *ctx, int n_chains, int n_dof, int max_samples, int *diag_id) {
  return guarded(ctx, [&] {
    if (!diag_id) fail(DINO_EINVAL, "diag_id is NULL");
    cudaSetDevice(ctx->device);
    *diag_id = diag_create(ctx, n_chains, n_dof, max_samples);
  });
}

int dino_diag_record(dino_ctx *ctx, int diag_id, int pool_id, int what, int chain0) {
  return guarded(ctx, [&] {
    cudaSetDevice(ctx->device);
    diag_record(ctx, get_diag(ctx, diag_id), get_pool(ctx, pool_id), what, chain0);
  });
}

int dino_diag_push(dino_ctx *ctx, int diag_id, const double *sample) {
  return guarded(ctx, [&] {
    cudaSetDevice(ctx->device);
    diag_push(ctx, get_diag(ctx, diag_id), sample);
  });
}

int dino_diag_compute(dino_ctx *ctx, int diag_id, int want_mpsrf, double *ess,
                      dino_diag_result *result) {
  return guarded(ctx, [&] {
    cudaSetDevice(ctx->device);
    diag_compute(ctx, get_diag(ctx, diag_id), want_mpsrf, ess, result);
  });
}

int dino_diag_destroy(dino_ctx *ctx, int diag_id) {
  return guarded(ctx, [&] {
    cudaSetDevice(ctx->device);
    free_diag(ctx, get_diag(ctx, diag_id));
    ctx->diags.erase(diag_id);
  });
}


int dino_chains_destroy(dino_ctx *ctx, int pool_id) {
  return guarded(ctx, [&] {
    cudaSetDevice(ctx->device);
    destroy_pool(ctx, pool_id);
  });
}

uint64_t dino_launch_count(const dino_ctx *ctx) { return ctx ? ctx->launches : 0; }

int dino_kernel_times(dino_ctx *ctx, char *names, double *total_ms, uint64_t *launches, int cap,
                      int *n, int reset) {
  return guarded(ctx, [&] {
    collect_times(ctx);
    int k = 0;
    for (auto &kv : ctx->ktimes) {
      if (k >= cap) break;
      if (names) {
        std::memset(names + 48 * k, 0, 48);
        std::strncpy(names + 48 * k, kv.first.c_str(), 47);
      }
      if (total_ms) total_ms[k] = kv.second.ms;
      if (launches) launches[k] = kv.second.n;
      ++k;
    }
    if (n) *n = (int)ctx->ktimes.size();
    if (reset) ctx->ktimes.clear();
  });
}

int dino_serve_config(dino_ctx *ctx, int n_streams, int steps_per_round, int max_active) {
  return guarded(ctx, [&] {
    if (ctx->server) fail(DINO_ESTATE, "serving already started");
    if (n_streams < 1 || n_streams > 32 || steps_per_round < 1 || max_active < 1)
      fail(DINO_EINVAL, "n_streams in 1..32, steps_per_round >= 1, max_active >= 1");
    cudaSetDevice(ctx->device);
    ctx->server.reset(new Server(ctx, n_streams, steps_per_round, max_active));
  });
}

int dino_serve_submit(dino_ctx *ctx, const dino_request *req, uint64_t *ticket) {
  return guarded(ctx, [&] {
    if (!req || !ticket) fail(DINO_EINVAL, "request and ticket must be non-NULL");
    Surrogate *s = get_surrogate(ctx, req->surrogate_id);
    if (!s->has_data) fail(DINO_ESTATE, "surrogate %d has no data", req->surrogate_id);
    if (req->n_chains < 1 || req->n_steps < 0 || !(req->dt > 0))
      fail(DINO_EINVAL, "n_chains >= 1, n_steps >= 0 and dt > 0 required");
    cudaSetDevice(ctx->device);
    if (!ctx->server) ctx->server.reset(new Server(ctx, 4, 8, 32));
    Server &sv = *ctx->server;
    if (sv.broken)
      fail(sv.broken_code, "serving stopped after an internal error: %s", sv.broken_msg.c_str());
    if (sv.queue.size() >= sv.max_queue) fail(DINO_EBUSY, "serving queue is full");
    auto r = std::make_unique<Request>();
    r->ticket = sv.next_ticket++;
    r->req = *req;
    r->footprint = pool_footprint(s, req->n_chains);
    {
      // per proposal: the factorisation of the smaller Gauss-Newton system
      // and the Jacobian GEMMs (orders of magnitude, for ordering only)
      const double k = std::min(s->r, s->d_y) + 1.0;
      double jac = 0.0;
      for (int l = 0; l + 1 < s->L; ++l) jac += 2.0 * s->widths[l] * s->widths[l + 1];
      r->work = (double)req->n_chains * req->n_steps *
                (12.0 * k * k * k / 3.0 + jac * std::min(s->r, s->d_y) / 50.0);
    }
    if (r->footprint > ctx->budget)
      fail(DINO_ENOMEM, "request needs %zu bytes, more than the whole HBM budget %zu",
           r->footprint, ctx->budget);
    if (req->m0) r->m0.assign(req->m0, req->m0 + (size_t)req->n_chains * s->N);
    r->t_submit = now_s();
    *ticket = r->ticket;
    sv.queue.push_back(r.get());
    sv.reqs[r->ticket] = std::move(r);
    sv.cv.notify_all();
  });
}

int dino_serve_poll(dino_ctx *ctx, uint64_t ticket, dino_result *res) {
  int pending = 0;
  const int rc = guarded(ctx, [&] {
    if (!ctx->server) fail(DINO_ENOTFOUND, "no request has been submitted");
    auto it = ctx->server->reqs.find(ticket);
    if (it == ctx->server->reqs.end()) fail(DINO_ENOTFOUND, "unknown ticket %llu",
                                            (unsigned long long)ticket);
    Request *r = it->second.get();
    if (r->state < 2) {
      pending = 1;
      return;
    }
    if (r->state == 3) fail(r->status, "request failed: %s", r->err.c_str());
    if (res) {
      res->stats = r->stats;
      res->queue_s = r->t_admit - r->t_submit;
      res->latency_s = r->t_done - r->t_submit;
    }
  });
  return rc == DINO_OK && pending ? DINO_PENDING : rc;
}

int dino_serve_wait(dino_ctx *ctx, uint64_t ticket, double timeout_s, dino_result *res) {
  if (!ctx) return DINO_EINVAL;
  const double deadline = now_s() + (timeout_s > 0 ? timeout_s : 0.0);
  while (true) {
    const int rc = dino_serve_poll(ctx, ticket, res);
    if (rc != DINO_PENDING) return rc;
    if (now_s() >= deadline) return DINO_ETIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
}

int dino_serve_status(dino_ctx *ctx, int *queued, int *active, int *peak_active,
                      size_t *hbm_used, size_t *peak_hbm_used) {
  return guarded(ctx, [&] {
    Server *sv = ctx->server.get();
    if (queued) *queued = sv ? (int)sv->queue.size() : 0;
    if (active) *active = sv ? (int)sv->active.size() : 0;
    if (peak_active) *peak_active = sv ? sv->peak_active : 0;
    if (hbm_used) *hbm_used = ctx->used;
    if (peak_hbm_used) *peak_hbm_used = sv ? sv->peak_used : ctx->used;
  });
}

}  // extern "C"
