// Allocation-free evaluation of the surrogate forward pass and its reduced
// Jacobian (FP64), for host code that is not allowed to allocate device memory.
//
// Such callers exist: a plugin running inside a framework that owns every
// device byte through its own pool, or a latency-critical loop in which the
// device-wide synchronisation that cudaMalloc/cudaFree may imply is not
// acceptable.  The entry point below therefore never allocates.  Inputs and
// outputs are device buffers the caller owns.  The intermediate products of
// the reverse-mode Jacobian live in one file-scope device array of fixed size.
// Every GPU that loads this library holds that array until the process exits.
//
// Set-up: the host cannot use the array's name as a device address (in host
// code it is only a stand-in symbol).  The first call on each device looks up
// the real address with cudaGetSymbolAddress while that device is current,
// and caches it.  That first call should therefore come before any stream
// capture on the device.
//
// Sharing: every call uses the same array, and it keeps the previous call's
// contents.  The kernel writes every scratch element before reading it, so
// nothing has to start at zero.  Two calls whose kernels overlap on the GPU
// (different streams, no ordering between them) race on the array: order
// them on one stream, or wait for one before issuing the other.
#include "../../include/dino.h"

#include <cuda_runtime.h>

#include <mutex>

namespace dino {
namespace {

constexpr int kMaxLayers = 16;
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;

static __device__ __align__(256) double g_noalloc_scratch[DINO_NOALLOC_SCRATCH_DOUBLES];

struct Net {
  int L, act;
  int w[kMaxLayers + 1];
  const double *W[kMaxLayers];
  const double *b[kMaxLayers];
};

__device__ __forceinline__ double act_fn(int kind, double z) {
  if (kind == DINO_ACT_TANH) return tanh(z);
  if (kind == DINO_ACT_GELU) return 0.5 * z * (1.0 + erf(z * 0.70710678118654752440));
  return z;
}

__device__ __forceinline__ double act_deriv(int kind, double z) {
  if (kind == DINO_ACT_TANH) {
    const double t = tanh(z);
    return 1.0 - t * t;
  }
  if (kind == DINO_ACT_GELU)
    return 0.5 * (1.0 + erf(z * 0.70710678118654752440)) +
           z * exp(-0.5 * z * z) * 0.39894228040143267794;
  return 1.0;
}

// One CTA per point.  Shared memory holds the activations and the activation
// derivatives; the d_y x w products of the reverse sweep go to a per-point
// slab of the scratch array (two ping-pong buffers of d_y * wmax doubles).
__global__ void __launch_bounds__(kThreads)
    k_jac_noalloc(const Net net, int wmax, const double *__restrict__ x, double *__restrict__ f,
                  double *__restrict__ J, double *__restrict__ scratch) {
  extern __shared__ double sm[];
  const int p = blockIdx.x, L = net.L, r = net.w[0], dy = net.w[L];
  double *a[kMaxLayers + 1];
  double *d[kMaxLayers];
  int off = 0;
  for (int l = 0; l < L; ++l) {  // a[0..L-1]: layer inputs; d[0..L-2]: derivatives
    a[l] = sm + off;
    off += net.w[l];
  }
  for (int l = 0; l + 1 < L; ++l) {
    d[l] = sm + off;
    off += net.w[l + 1];
  }
  for (int i = threadIdx.x; i < r; i += blockDim.x) a[0][i] = x[(size_t)p * r + i];
  __syncthreads();
  for (int l = 0; l < L; ++l) {
    const int wi = net.w[l], wo = net.w[l + 1];
    const double *W = net.W[l];
    for (int o = threadIdx.x; o < wo; o += blockDim.x) {
      double z = net.b[l][o];
      for (int i = 0; i < wi; ++i) z += W[(size_t)o * wi + i] * a[l][i];
      if (l + 1 < L) {
        a[l + 1][o] = act_fn(net.act, z);
        d[l][o] = act_deriv(net.act, z);
      } else {
        f[(size_t)p * dy + o] = z;
      }
    }
    __syncthreads();
  }
  double *Jp = J + (size_t)p * dy * r;
  if (L == 1) {
    for (int e = threadIdx.x; e < dy * r; e += blockDim.x) Jp[e] = net.W[0][e];
    return;
  }
  double *P = scratch + (size_t)p * 2 * dy * wmax;
  double *Q = P + (size_t)dy * wmax;
  const int wl = net.w[L - 1];
  for (int e = threadIdx.x; e < dy * wl; e += blockDim.x)
    P[e] = net.W[L - 1][e] * d[L - 2][e % wl];
  __syncthreads();
  for (int l = L - 2; l >= 1; --l) {  // P <- (P W_l) .* d_{l-1}
    const int wi = net.w[l], wo = net.w[l + 1];
    const double *W = net.W[l];
    for (int e = threadIdx.x; e < dy * wi; e += blockDim.x) {
      const int i = e / wi, j = e % wi;
      double acc = 0.0;
      for (int k = 0; k < wo; ++k) acc += P[(size_t)i * wo + k] * W[(size_t)k * wi + j];
      Q[e] = acc * d[l - 1][j];
    }
    __syncthreads();
    double *t = P;
    P = Q;
    Q = t;
  }
  const int w1 = net.w[1];
  for (int e = threadIdx.x; e < dy * r; e += blockDim.x) {  // J = P W_0
    const int i = e / r, j = e % r;
    double acc = 0.0;
    for (int k = 0; k < w1; ++k) acc += P[(size_t)i * w1 + k] * net.W[0][(size_t)k * r + j];
    Jp[e] = acc;
  }
}

std::mutex g_mu;
double *g_addr[kMaxDevices] = {nullptr};

}  // namespace
}  // namespace dino

extern "C" int dino_surrogate_jacobian_noalloc(int n, int n_layers, const int *widths,
                                               int activation, const double *const *W,
                                               const double *const *b, const double *x,
                                               double *f, double *J, void *stream) {
  using namespace dino;
  if (n < 1 || n_layers < 1 || n_layers > kMaxLayers || !widths || !W || !b || !x || !f || !J)
    return DINO_EINVAL;
  if (activation < DINO_ACT_IDENTITY || activation > DINO_ACT_GELU) return DINO_EINVAL;
  Net net{};
  net.L = n_layers;
  net.act = activation;
  int wmax = 0;
  size_t smem_doubles = 0;
  for (int l = 0; l <= n_layers; ++l) {
    if (widths[l] < 1) return DINO_EINVAL;
    net.w[l] = widths[l];
    if (l < n_layers) smem_doubles += widths[l];
    if (l >= 1 && l < n_layers) {
      wmax = widths[l] > wmax ? widths[l] : wmax;
      smem_doubles += widths[l];
    }
  }
  for (int l = 0; l < n_layers; ++l) {
    if (!W[l] || !b[l]) return DINO_EINVAL;
    net.W[l] = W[l];
    net.b[l] = b[l];
  }
  const size_t smem = smem_doubles * sizeof(double);
  if (smem > 200 * 1024) return DINO_EINVAL;
  // the fixed scratch must hold two d_y x wmax buffers per point
  const size_t need = (size_t)n * 2 * (size_t)widths[n_layers] * (size_t)wmax;
  if (need > (size_t)DINO_NOALLOC_SCRATCH_DOUBLES) return DINO_ENOMEM;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DINO_ECUDA;
  double *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return DINO_ECUDA;
      }
      g_addr[dev] = (double *)p;
    }
    scratch = g_addr[dev];
  }
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_jac_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return DINO_ECUDA;
  k_jac_noalloc<<<n, kThreads, smem, (cudaStream_t)stream>>>(net, wmax, x, f, J, scratch);
  return cudaGetLastError() == cudaSuccess ? DINO_OK : DINO_ECUDA;
}
