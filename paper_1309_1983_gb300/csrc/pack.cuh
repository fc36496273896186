// pack.cuh - aligned multi-value loads and stores of one distribution
// plane, converted to and from FP32: pairs (x0, x0 + 1) for the two-node
// step kernel and groups of four (x0 .. x0 + 3) for the four-node kernel.
// Loads carry the 256-byte L2 prefetch hint (check.cuh).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "check.cuh"

namespace lbm {

// Loads and stores of an aligned pair of values, as two floats.
template <int S>
struct Pack16;

template <>
struct Pack16<0> {
  static __device__ __forceinline__ float2 load(const float *p) {
    return LBM_LDG(reinterpret_cast<const float2 *>(p));
  }
  static __device__ __forceinline__ void store(float *p, float lo, float hi) {
    LBM_ST(reinterpret_cast<float2 *>(p), make_float2(lo, hi));
  }
};

template <>
struct Pack16<1> {
  static __device__ __forceinline__ float2 load(const __half *p) {
    return unpack(ldg_pf_b32(p));
  }
  static __device__ __forceinline__ void store(__half *p, float lo, float hi) {
    LBM_ST(reinterpret_cast<unsigned int *>(p), pack(lo, hi));
  }
  static __device__ __forceinline__ float2 unpack(uint32_t v) {
    return __half22float2(*reinterpret_cast<const __half2 *>(&v));
  }
  static __device__ __forceinline__ uint32_t pack(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
  }
};

template <>
struct Pack16<2> {
  static __device__ __forceinline__ float2 load(const __nv_bfloat16 *p) {
    return unpack(ldg_pf_b32(p));
  }
  static __device__ __forceinline__ void store(__nv_bfloat16 *p, float lo, float hi) {
    LBM_ST(reinterpret_cast<unsigned int *>(p), pack(lo, hi));
  }
  static __device__ __forceinline__ float2 unpack(uint32_t v) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v));
  }
  static __device__ __forceinline__ uint32_t pack(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
  }
};

// An aligned group of four 16-bit values (x0 .. x0 + 3) of one plane, kept
// packed as loaded (two 32-bit words of two values); get<k>() converts value
// k to FP32.
template <int S>
struct Quad;

template <int S>
struct Quad16 {
  using V = uint2;
  template <class T>
  static __device__ __forceinline__ V load(const T *p) {
    return ldg_pf_v2b32(p);
  }
  template <int k>
  static __device__ __forceinline__ float get(const V &v) {
    const float2 f = Pack16<S>::unpack(k < 2 ? v.x : v.y);
    return (k & 1) ? f.y : f.x;
  }
};
template <>
struct Quad<1> : Quad16<1> {};
template <>
struct Quad<2> : Quad16<2> {};

}  // namespace lbm
