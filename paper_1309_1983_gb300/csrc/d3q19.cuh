// d3q19.cuh - device-side D3Q19 constants, storage traits and the fused
// BGK collision used by every kernel of liblbm.
//
// Velocity set: Eq. 4 (directions i = 0..18 in the printed column order).
// Weights: 1/3, 1/18 (i = 1..6), 1/36 (i = 7..18), c_s^2 = 1/3 (text after
// Eq. 5). Opposite pairs are (i, i+1) for odd i.
//
// All distributions are handled in SHIFTED form d_i = f_i - w_i. In exact
// arithmetic nothing changes (sum w_i = 1, sum w_i e_i = 0); in FP32 and in
// 16-bit storage it keeps the stored magnitudes small so rounding acts on the
// deviation from rest instead of on f_i ~ w_i.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "check.cuh"

namespace lbm {

constexpr int Q = 19;

// Eq. 4, columns i = 0..18.
constexpr int kEx[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1};
constexpr int kEy[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 1, -1, 1, -1, 0, 0, 0, 0};
constexpr int kEz[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, 1, -1};
constexpr int kOpp[Q] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
// compile-time opposite as a value (never an ODR-use of the table in device code)
template <int i>
constexpr int kOpp_v = kOpp[i];

__host__ __device__ constexpr float weight(int i) {
  return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}
__host__ __device__ constexpr double weight_d(int i) {
  return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Compile-time loop: f(std::integral_constant<int, I>) for I in [B, E).
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F &&f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// ---- storage traits: 0 = FP32, 1 = FP16, 2 = BF16 -------------------------
// ld(): read-only path (ld.global.nc), valid when the buffer is not written
// during the kernel. ld_l2(): L2-only path (ld.global.cg) for persistent
// kernels in which other blocks rewrite the buffer between grid barriers.
template <int S>
struct Store;

template <>
struct Store<0> {
  using T = float;
  static __device__ __forceinline__ float ld(const T *p) { return LBM_LDG(p); }
  static __device__ __forceinline__ float ld_l2(const T *p) { return LBM_LDCG(p); }
  static __device__ __forceinline__ float ld_smem(const T *p) { return *p; }
  static __device__ __forceinline__ void st(T *p, float v) { LBM_ST(p, v); }
};
template <>
struct Store<1> {
  using T = __half;
  static __device__ __forceinline__ float ld(const T *p) {
    return __half2float(__ushort_as_half(ldg_pf_b16(p)));
  }
  static __device__ __forceinline__ float ld_l2(const T *p) {
    return __half2float(LBM_LDCG(p));
  }
  static __device__ __forceinline__ float ld_smem(const T *p) { return __half2float(*p); }
  static __device__ __forceinline__ void st(T *p, float v) {
    LBM_ST(p, __float2half_rn(v));
  }
};
template <>
struct Store<2> {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ float ld(const T *p) {
    return __bfloat162float(__ushort_as_bfloat16(ldg_pf_b16(p)));
  }
  static __device__ __forceinline__ float ld_l2(const T *p) {
    return __bfloat162float(LBM_LDCG(p));
  }
  static __device__ __forceinline__ float ld_smem(const T *p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ void st(T *p, float v) {
    LBM_ST(p, __float2bfloat16_rn(v));
  }
};

template <int S, bool L2ONLY>
__device__ __forceinline__ float load_f(const typename Store<S>::T *p) {
  if constexpr (L2ONLY)
    return Store<S>::ld_l2(p);
  else
    return Store<S>::ld(p);
}

// ---- moments of shifted distributions (Eqs. 6-7) ---------------------------
// dr = rho - 1 = sum d_i; j = sum e_i d_i (= sum e_i f_i).
__device__ __forceinline__ void shifted_moments(const float (&d)[Q], float &dr,
                                                float &jx, float &jy,
                                                float &jz) {
  // pairwise grouping keeps the FP32 sums short
  dr = ((d[0] + (d[1] + d[2])) + ((d[3] + d[4]) + (d[5] + d[6]))) +
       (((d[7] + d[8]) + (d[9] + d[10])) + ((d[11] + d[12]) + (d[13] + d[14]))) +
       ((d[15] + d[16]) + (d[17] + d[18]));
  jx = ((d[1] - d[2]) + (d[7] - d[8])) + ((d[9] - d[10]) + (d[15] - d[16])) + (d[18] - d[17]);
  jy = ((d[3] - d[4]) + (d[7] - d[8])) + ((d[10] - d[9]) + (d[11] - d[12])) + (d[13] - d[14]);
  jz = ((d[5] - d[6]) + (d[11] - d[12])) + ((d[14] - d[13]) + (d[15] - d[16])) + (d[17] - d[18]);
}

// ---- BGK collision with optional Guo force, in place on shifted values -----
// In: d_i = g_i - w_i (post-streaming). Out: d*_i = f*_i - w_i with
//   f*_i = (1 - omega) g_i + omega f^eq_i + kf S_i,  kf = 1 - omega/2,
// and f^eq_i - w_i (Eq. 5) split into its parts even and odd in e_i, written
// with the momentum j = rho u = sum e_i g_i + F/2:
//   even_i = w_i [dr - 1.5 |j|^2 / rho + 4.5 (e_i . j)^2 / rho]
//   odd_i  = 3 w_i (e_i . j)                  (no division by rho enters it)
//   S_i    = w_i [3 (e_i - u) + 9 (e_i . u) e_i] . F                (Guo)
// Each opposite pair (i, i+1) shares its even part and negates its odd part.
//
// Momentum is the quantity that rounding must not bias. The odd parts return
// (2 c_A + 8 c_B) j with c_A = 3 w_A omega = omega/6 and c_B = omega/12, and
// the relaxed part (1 - omega) j. With FP32-rounded coefficients the sum is
// (1 + delta) j, delta ~ 1e-7, on every node and every step: over 1000 steps
// of a freely decaying flow that drift reaches ~1e-4 of the velocity. The
// host therefore sets omega within 2^-22 of 1/tau such that omega * (1/12)
// is exactly omega/12 in FP32 and 12 times it is exactly omega (see
// relaxation_rate); then c_A = 2 c_B, 2 c_A + 8 c_B = omega and 1 - omega
// are all exact, and the step conserves momentum up to unbiased per-node
// rounding.
// Returns rho and the velocity u = j / rho that the collision used.
template <bool FORCE>
__device__ __forceinline__ void collide(float (&d)[Q], float omega, float kf,
                                        float Fx, float Fy, float Fz,
                                        float &rho, float &ux, float &uy,
                                        float &uz) {
  float dr, jx, jy, jz;
  shifted_moments(d, dr, jx, jy, jz);
  rho = 1.0f + dr;
  const float rinv = __frcp_rn(rho);
  if constexpr (FORCE) {
    jx = fmaf(0.5f, Fx, jx);
    jy = fmaf(0.5f, Fy, jy);
    jz = fmaf(0.5f, Fz, jz);
  }
  ux = jx * rinv;
  uy = jy * rinv;
  uz = jz * rinv;
  const float keep = 1.0f - omega;              // exact
  const float cB = omega * (1.0f / 12.0f);      // exactly omega/12
  const float cA = 2.0f * cB;                   // exactly omega/6
  const float jsq = fmaf(jx, jx, fmaf(jy, jy, jz * jz));
  const float base = fmaf(-1.5f * jsq, rinv, dr);  // dr - 1.5 rho |u|^2
  const float k45 = 4.5f * rinv;
  // omega folded into the weights of the even part
  const float owA = omega * weight(1), owB = omega * weight(7);
  const float bA = owA * base, bB = owB * base;
  const float kA = owA * k45, kB = owB * k45;
  float uF = 0.0f, k9 = 0.0f;
  if constexpr (FORCE) {
    uF = fmaf(ux, Fx, fmaf(uy, Fy, uz * Fz));
    k9 = 9.0f * rinv;
  }

  // rest direction
  {
    constexpr float w = weight(0);
    float v = fmaf(keep, d[0], (omega * w) * base);
    if constexpr (FORCE) v = fmaf(kf, w * (-3.0f * uF), v);
    d[0] = v;
  }
  static_for<0, 9>([&](auto P) {
    constexpr int i = 2 * decltype(P)::value + 1;  // odd member of the pair
    constexpr int j = i + 1;                        // its opposite
    constexpr float w = weight(i);
    constexpr float cx = (float)kEx[i], cy = (float)kEy[i], cz = (float)kEz[i];
    const float b = i < 7 ? bA : bB, k = i < 7 ? kA : kB, c = i < 7 ? cA : cB;
    const float es = cx * jx + cy * jy + cz * jz;  // e.j; folds to adds/subs
    const float even = fmaf(es * es, k, b);
    const float odd = c * es;
    float vi = fmaf(keep, d[i], even + odd);
    float vj = fmaf(keep, d[j], even - odd);
    if constexpr (FORCE) {
      const float eF = cx * Fx + cy * Fy + cz * Fz;
      const float sEven = w * fmaf(k9 * es, eF, -3.0f * uF);  // 9 (e.u)(e.F) - 3 u.F
      const float sOdd = (3.0f * w) * eF;
      vi = fmaf(kf, sEven + sOdd, vi);
      vj = fmaf(kf, sEven - sOdd, vj);
    }
    d[i] = vi;
    d[j] = vj;
  });
}

// Shifted equilibrium f^eq_i(rho, u) - w_i (Eq. 5), for initialisation.
__device__ __forceinline__ void shifted_equilibrium(float rho, float ux,
                                                    float uy, float uz,
                                                    float (&d)[Q]) {
  const float dr = rho - 1.0f;
  const float usq15 = 1.5f * fmaf(ux, ux, fmaf(uy, uy, uz * uz));
  d[0] = weight(0) * fmaf(-rho, usq15, dr);
  static_for<0, 9>([&](auto P) {
    constexpr int i = 2 * decltype(P)::value + 1;
    constexpr float w = weight(i);
    constexpr float cx = (float)kEx[i], cy = (float)kEy[i], cz = (float)kEz[i];
    const float eu = cx * ux + cy * uy + cz * uz;
    const float even = w * fmaf(rho, fmaf(4.5f * eu, eu, -usq15), dr);
    const float odd = (3.0f * w) * rho * eu;
    d[i] = even + odd;
    d[i + 1] = even - odd;
  });
}

}  // namespace lbm
