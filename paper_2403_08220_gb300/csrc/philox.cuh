// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11)
// and the uniforms / normals the sampler draws from it.
//
// key = (seed mod 2^32, seed >> 32); counter = (block, step, chain, stream).
// One block gives four 32-bit words; word x maps to u = (x + 1/2) 2^-32 in
// (0, 1); (u0, u1) and (u2, u3) are turned into two pairs of standard normals
// by the Box-Muller transform, so block k carries normals 4k .. 4k+3.
#pragma once
#include <cstdint>

namespace dino {

enum : uint32_t {
  STREAM_XI = 0, STREAM_U = 1, STREAM_Z = 2, STREAM_INIT = 3, STREAM_XI2 = 4, STREAM_U2 = 5
};

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = mulhi32(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = mulhi32(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__device__ __forceinline__ uint4 philox_block(uint64_t seed, uint32_t stream, uint32_t step,
                                              uint32_t chain, uint32_t block) {
  return philox4x32_10(make_uint4(block, step, chain, stream), (uint32_t)seed,
                       (uint32_t)(seed >> 32));
}

__device__ __forceinline__ double word_to_uniform(uint32_t x) {
  return ((double)x + 0.5) * 2.3283064365386963e-10;  // 2^-32
}

// Four float64 normals of one block.
__device__ __forceinline__ void normals4_f64(uint4 w, double out[4]) {
  const double u0 = word_to_uniform(w.x), u1 = word_to_uniform(w.y);
  const double u2 = word_to_uniform(w.z), u3 = word_to_uniform(w.w);
  const double r01 = sqrt(-2.0 * log(u0)), r23 = sqrt(-2.0 * log(u2));
  double s, c;
  sincospi(2.0 * u1, &s, &c);
  out[0] = r01 * c;
  out[1] = r01 * s;
  sincospi(2.0 * u3, &s, &c);
  out[2] = r23 * c;
  out[3] = r23 * s;
}

// Same definition evaluated in float32 (relative error ~1e-7).
__device__ __forceinline__ void normals4_f32(uint4 w, float out[4]) {
  const float k = 2.3283064365386963e-10f;
  const float u0 = ((float)w.x + 0.5f) * k, u1 = ((float)w.y + 0.5f) * k;
  const float u2 = ((float)w.z + 0.5f) * k, u3 = ((float)w.w + 0.5f) * k;
  const float r01 = sqrtf(-2.0f * logf(u0)), r23 = sqrtf(-2.0f * logf(u2));
  float s, c;
  sincospif(2.0f * u1, &s, &c);
  out[0] = r01 * c;
  out[1] = r01 * s;
  sincospif(2.0f * u3, &s, &c);
  out[2] = r23 * c;
  out[3] = r23 * s;
}

}  // namespace dino
