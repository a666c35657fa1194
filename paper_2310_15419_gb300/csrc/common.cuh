// common.cuh -- device generator, distribution transforms and small helpers
// shared by the sketch kernels (sm_103a).
//
// S(i, j) is a pure function of (seed, stream, i, j): the counter-based
// generator Philox4x32-10 (Salmon et al., SC'11; the paper's Sec. 4.2 names
// this family) is evaluated at counter (i_blk, j, stream, 0) under the key
// (seed lo32, seed hi32).  Any kernel, tile size or launch shape therefore
// sees the same S (Sec. 4.3's threading-independent reproducibility).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sk {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;  // round multipliers
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;  // Weyl key increments
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

constexpr int kPM1 = 0, kUniform = 1, kNormal = 2;

// One Philox round: two 32x32->64 multiplies (each one wide multiply,
// both halves used) and two three-input xors with the round key.
__device__ __forceinline__ uint4 philox_round(uint4 c, uint32_t k0, uint32_t k1) {
  const uint64_t p0 = static_cast<uint64_t>(kPhiloxM0) * c.x;
  const uint64_t p1 = static_cast<uint64_t>(kPhiloxM1) * c.z;
  return make_uint4(static_cast<uint32_t>(p1 >> 32) ^ c.y ^ k0, static_cast<uint32_t>(p1),
                    static_cast<uint32_t>(p0 >> 32) ^ c.w ^ k1, static_cast<uint32_t>(p0));
}

// Ten Philox rounds; the key advances by the Weyl increments after each.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0,
                                               uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    c = philox_round(c, k0, k1);
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return c;
}

__device__ __forceinline__ uint4 philox_block(uint32_t i_blk, uint32_t j,
                                              uint32_t stream, uint32_t k0,
                                              uint32_t k1) {
  return philox4x32_10(make_uint4(i_blk, j, stream, 0u), k0, k1);
}

// The ten round keys of a seed, computed once on the host.  A kernel that
// takes them as a __grid_constant__ parameter reads each from the constant
// bank as an operand of its xor, with no key arithmetic per block.
struct PhiloxKeys {
  uint32_t k0[10], k1[10];
};
inline PhiloxKeys philox_keys(uint32_t k0, uint32_t k1) {
  PhiloxKeys ks;
  for (int r = 0; r < 10; ++r) {
    ks.k0[r] = k0 + static_cast<uint32_t>(r) * kPhiloxW0;
    ks.k1[r] = k1 + static_cast<uint32_t>(r) * kPhiloxW1;
  }
  return ks;
}
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys& ks) {
#pragma unroll
  for (int r = 0; r < 10; ++r) c = philox_round(c, ks.k0[r], ks.k1[r]);
  return c;
}
__device__ __forceinline__ uint4 philox_block(uint32_t i_blk, uint32_t j, uint32_t stream,
                                              const PhiloxKeys& ks) {
  return philox4x32_10(make_uint4(i_blk, j, stream, 0u), ks);
}

// U(-1,1): top 24 bits as a signed integer u, S = (2u + 1) 2^-24.  The fma
// rounds an exactly representable value, so the result is exact.
__device__ __forceinline__ float uniform_from_word(uint32_t w) {
  const int32_t u = static_cast<int32_t>(w) >> 8;
  return fmaf(static_cast<float>(u), 0x1p-23f, 0x1p-24f);
}

// Box-Muller on one word pair: u1 in (0,1] from the radius word, u2 in [0,1)
// from the angle word; returns (r cos 2 pi u2, r sin 2 pi u2).
__device__ __forceinline__ float2 normal_pair(uint32_t w_radius,
                                              uint32_t w_angle) {
  const float u1 = static_cast<float>((w_radius >> 8) + 1u) * 0x1p-24f;
  const float u2 = static_cast<float>(w_angle >> 8) * 0x1p-24f;
  const float r = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  return make_float2(r * c, r * s);
}

// The four entries S(4 i_blk .. 4 i_blk + 3, j) for U or N.
template <int DIST>
__device__ __forceinline__ float4 four_entries(uint4 x) {
  if constexpr (DIST == kUniform) {
    return make_float4(uniform_from_word(x.x), uniform_from_word(x.y),
                       uniform_from_word(x.z), uniform_from_word(x.w));
  } else {
    const float2 a = normal_pair(x.x, x.y);
    const float2 b = normal_pair(x.z, x.w);
    return make_float4(a.x, a.y, b.x, b.y);
  }
}

// A single entry, for the test hook and for ragged edges.
__device__ __forceinline__ float S_entry(int dist, uint32_t k0, uint32_t k1,
                                         uint32_t stream, int64_t i,
                                         int64_t j) {
  if (dist == kPM1) {
    const uint4 x = philox_block(static_cast<uint32_t>(i >> 7),
                                 static_cast<uint32_t>(j), stream, k0, k1);
    const int b = static_cast<int>(i & 127);
    const uint32_t w = (b < 32) ? x.x : (b < 64) ? x.y : (b < 96) ? x.z : x.w;
    return ((w >> (b & 31)) & 1u) ? -1.0f : 1.0f;
  }
  const uint4 x = philox_block(static_cast<uint32_t>(i >> 2),
                               static_cast<uint32_t>(j), stream, k0, k1);
  const int q = static_cast<int>(i & 3);
  if (dist == kUniform) {
    const uint32_t w = (q == 0) ? x.x : (q == 1) ? x.y : (q == 2) ? x.z : x.w;
    return uniform_from_word(w);
  }
  const float2 p = (q < 2) ? normal_pair(x.x, x.y) : normal_pair(x.z, x.w);
  return (q & 1) ? p.y : p.x;
}

template <typename VT>
__device__ __forceinline__ float to_f32(VT v);
template <>
__device__ __forceinline__ float to_f32<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}

// Device status bits written by kernels that meet bad input.
constexpr int kStatusBadRow = 1;
constexpr int kStatusBadColptr = 2;
constexpr int kStatusTimeout = 4;  // a bounded wait inside a kernel gave up

// Column k's nonzeros [lo, hi) of a CSC with nnz entries, clamped so that
// 0 <= lo <= hi <= nnz whatever colptr holds: a malformed colptr (decreasing,
// negative or past nnz) is recorded in *status and never turns into an
// out-of-range read.  (Overlapping column ranges stay in bounds too; the
// kernels that scatter by such ranges check their write positions.)
__device__ __forceinline__ int2 column_range(const int32_t* __restrict__ colptr, int64_t k,
                                             int64_t nnz, int* status) {
  const int64_t p0 = colptr[k], p1 = colptr[k + 1];
  const int64_t lo64 = p0 < 0 ? 0 : (p0 > nnz ? nnz : p0);
  const int64_t hi64 = p1 < lo64 ? lo64 : (p1 > nnz ? nnz : p1);
  const int32_t lo = static_cast<int32_t>(lo64), hi = static_cast<int32_t>(hi64);
  if ((lo64 != p0 || hi64 != p1) && status) atomicOr(status, kStatusBadColptr);
  return make_int2(lo, hi);
}

}  // namespace sk
