// adjoint.cuh - per-node pieces of the discrete adjoint (the exact transpose
// of the forward step; the paper has no adjoint), shared by the single-lattice
// and the batched kernels.
//
// Forward step: f^{n+1} = C(P f^n; F), P = pull with bounce-back (affine; the
// lid term is a constant), C = per-node BGK collision with Guo forcing.
// Reverse step: lambda^n = P^T J_C(P f^n)^T lambda^{n+1}.
//
// Per node, with g = P f^n, rho = sum g, m = sum e g + F/2, u = m / rho and
// the weighted moments of lambda = lambda^{n+1}(x)
//   L0 = sum w_i lambda_i,  L1 = sum w_i lambda_i e_i,
//   L2 = sum w_i lambda_i e_i e_i^T,
// the collision Jacobian transpose is a rank-4 update of (1 - omega) I:
//   mu_j = (1 - omega) lambda_j + A + B . e_j,
//   a    = L0 + 3 u.L1 + 4.5 u.L2.u - 1.5 |u|^2 L0      (= sum lambda f^eq / rho)
//   b    = omega rho (3 L1 + 9 L2 u - 3 u L0) + kf (9 L2 F - 3 F L0)
//   A    = omega a - b.u / rho,  B = b / rho,  kf = 1 - omega/2,
// and the force cotangent gains kf (3 L1 - 3 u L0 + 9 L2 u) + b / (2 rho).
// P^T is a scatter: mu_i(x) goes to lambda^n_i(x - e_i), or to
// lambda^n_ibar(x) when x - e_i lies outside a walled axis. Every element of
// lambda^n receives exactly one contribution, so the scatter is a
// permutation and needs no atomics.
#pragma once

#include "d3q19.cuh"
#include "internal.h"
#include "stream.cuh"

namespace lbm {

struct LamMoments {
  float L0;
  float L1[3];
  float L2[6];  // xx, yy, zz, xy, xz, yz
};

__device__ __forceinline__ LamMoments lambda_moments(const float (&l)[Q]) {
  LamMoments m;
  m.L0 = weight(0) * l[0];
  m.L1[0] = m.L1[1] = m.L1[2] = 0.0f;
  for (int k = 0; k < 6; ++k) m.L2[k] = 0.0f;
  static_for<0, 9>([&](auto P) {
    constexpr int i = 2 * decltype(P)::value + 1;
    constexpr float w = weight(i);
    constexpr int ex = kEx[i], ey = kEy[i], ez = kEz[i];
    const float s = w * (l[i] + l[i + 1]);  // even part (e e^T, 1)
    const float t = w * (l[i] - l[i + 1]);  // odd part (e)
    m.L0 += s;
    if constexpr (ex != 0) m.L1[0] += ex * t;
    if constexpr (ey != 0) m.L1[1] += ey * t;
    if constexpr (ez != 0) m.L1[2] += ez * t;
    if constexpr (ex != 0) m.L2[0] += s;
    if constexpr (ey != 0) m.L2[1] += s;
    if constexpr (ez != 0) m.L2[2] += s;
    if constexpr (ex * ey != 0) m.L2[3] += (ex * ey) * s;
    if constexpr (ex * ez != 0) m.L2[4] += (ex * ez) * s;
    if constexpr (ey * ez != 0) m.L2[5] += (ey * ez) * s;
  });
  return m;
}

__device__ __forceinline__ void mat_vec(const float (&L2)[6], float vx, float vy,
                                        float vz, float &ox, float &oy, float &oz) {
  ox = fmaf(L2[0], vx, fmaf(L2[3], vy, L2[4] * vz));
  oy = fmaf(L2[3], vx, fmaf(L2[1], vy, L2[5] * vz));
  oz = fmaf(L2[4], vx, fmaf(L2[5], vy, L2[2] * vz));
}

// The scatter mode of adjoint_core for this node's warp: 2 (every face) with
// per-node selection, else by warp votes 2 if any active thread holds a y or
// z wall node, 1 if only x wall nodes, 0 if none, so that warps never split
// between paths (only x faces: 0.35% faster for the batched reverse step,
// 0.85% for the 256^3 cavity). Called by all active threads of the warp at
// the same point.
template <bool WALLS>
__device__ __forceinline__ int scatter_mode(const NodeIdx &n, bool wall_select) {
  if (!WALLS) return 0;
  if (wall_select) return 2;
  const unsigned m = __activemask();
  if (__any_sync(m, n.y0 | n.y1 | n.z0 | n.z1)) return 2;
  return __any_sync(m, n.x0 | n.x1) ? 1 : 0;
}

// lambda^{n+1} at the node (aligned loads). L2ONLY: through L2 only
// (ld.global.cg), for persistent kernels in which other blocks wrote
// lambda^{n+1} before the last grid barrier.
template <bool L2ONLY = false>
__device__ __forceinline__ void load_lambda(const float *__restrict__ lam_in, uint32_t plane,
                                            const NodeIdx &n, float (&lam)[Q]) {
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    lam[i] = L2ONLY ? LBM_LDCG(lam_in + (size_t)i * plane + n.c)
                    : LBM_LDG(lam_in + (size_t)i * plane + n.c);
  });
}

// Shared part of a reverse step at one node, given lambda^{n+1}(x) and the
// density rho and velocity u = (sum e g + F/2) / rho that the forward
// collision used there: form mu = J_C^T lambda^{n+1}(x) (which depends on g
// only through rho and u), scatter it by P^T into lambda_out, and add the
// force cotangent into gF (GRADF). `sel`: how the scatter applies the
// bounce-back rule on this node: 0 not at all (no wall node in the warp),
// 1 on the x faces only (only x-wall nodes in the warp: the ten e_x != 0
// directions select their address), 2 on every face.
template <bool FORCE, bool GRADF>
__device__ __forceinline__ void adjoint_core(
    float (&lam)[Q], float *__restrict__ lam_out, float *__restrict__ gF, uint32_t plane,
    const NodeIdx &n, int sel, uint32_t dc, uint32_t cells, float rho, float ux, float uy,
    float uz, float Fx, float Fy, float Fz, float omega, float kf) {
  const float rinv = __frcp_rn(rho);
  const float usq = fmaf(ux, ux, fmaf(uy, uy, uz * uz));

  const LamMoments m = lambda_moments(lam);
  float Lux, Luy, Luz;
  mat_vec(m.L2, ux, uy, uz, Lux, Luy, Luz);
  const float uL1 = fmaf(ux, m.L1[0], fmaf(uy, m.L1[1], uz * m.L1[2]));
  const float uLu = fmaf(ux, Lux, fmaf(uy, Luy, uz * Luz));
  const float av = fmaf(4.5f, uLu, fmaf(3.0f, uL1, m.L0 * fmaf(-1.5f, usq, 1.0f)));
  // s = 3 L1 + 9 L2 u - 3 u L0 (the velocity derivative of sum lambda f^eq / rho)
  const float sx = 3.0f * m.L1[0] + 9.0f * Lux - 3.0f * ux * m.L0;
  const float sy = 3.0f * m.L1[1] + 9.0f * Luy - 3.0f * uy * m.L0;
  const float sz = 3.0f * m.L1[2] + 9.0f * Luz - 3.0f * uz * m.L0;
  const float om = omega;
  float bx = om * rho * sx, by = om * rho * sy, bz = om * rho * sz;
  if constexpr (FORCE) {
    float LFx, LFy, LFz;
    mat_vec(m.L2, Fx, Fy, Fz, LFx, LFy, LFz);
    bx = fmaf(kf, 9.0f * LFx - 3.0f * Fx * m.L0, bx);
    by = fmaf(kf, 9.0f * LFy - 3.0f * Fy * m.L0, by);
    bz = fmaf(kf, 9.0f * LFz - 3.0f * Fz * m.L0, bz);
  }
  const float A = om * av - (bx * ux + by * uy + bz * uz) * rinv;
  const float Bx = bx * rinv, By = by * rinv, Bz = bz * rinv;
  const float keep = 1.0f - om;

  if constexpr (GRADF) {
    LBM_ACC(&gF[dc], fmaf(kf, sx, 0.5f * Bx));
    LBM_ACC(&gF[cells + dc], fmaf(kf, sy, 0.5f * By));
    LBM_ACC(&gF[2 * (size_t)cells + dc], fmaf(kf, sz, 0.5f * Bz));
  }

  // mu_j = (1 - omega) lambda_j + A + B . e_j, in place, then scattered by P^T
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr float cx = (float)kEx[i], cy = (float)kEy[i], cz = (float)kEz[i];
    lam[i] = fmaf(keep, lam[i], A + (cx * Bx + cy * By + cz * Bz));
  });
  if (sel == 2) {
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const size_t idx = bounces<i>(n) ? (size_t)kOpp_v<i> * plane + n.c
                                       : (size_t)i * plane + source_of<i>(n);
      LBM_ST(&lam_out[idx], lam[i]);
    });
  } else if (sel == 1) {
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      if constexpr (kEx[i] == 0) {
        LBM_ST(&lam_out[(size_t)i * plane + source_of<i>(n)], lam[i]);
      } else {
        const bool b = kEx[i] == 1 ? n.x0 : n.x1;
        const size_t idx = b ? (size_t)kOpp_v<i> * plane + n.c
                             : (size_t)i * plane + source_of<i>(n);
        LBM_ST(&lam_out[idx], lam[i]);
      }
    });
  } else {
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      LBM_ST(&lam_out[(size_t)i * plane + source_of<i>(n)], lam[i]);
    });
  }
}

// One reverse step at node (x, y, z) from the state f^n that entered the
// forward step: recompute g = P f^n there for rho and u, then adjoint_core.
// WALLS = false compiles the periodic form only; with WALLS the gather and
// the scatter apply the bounce-back rule either by per-direction address
// selection on every node (wall_select) or only in the warps that hold a
// node on a walled face (cheaper on long rows).
template <bool WALLS, bool FORCE, bool GRADF>
__device__ __forceinline__ void adjoint_node(
    const float *__restrict__ fn, const float *__restrict__ lam_in,
    float *__restrict__ lam_out, const float *__restrict__ force, float *__restrict__ gF,
    int nx, int ny, int nz, int pitch, uint32_t plane, uint32_t walls,
    const float (&lidc)[Q], float omega, float kf, uint32_t cells, int x, int y, int z,
    bool wall_select = true) {
  const NodeIdx n = node_index(nx, ny, nz, pitch, WALLS ? walls : 0u, x, y, z);
  const int sel = scatter_mode<WALLS>(n, wall_select);

  // recompute the post-streaming state g = P f^n of the forward step
  // (measured faster here than a periodic gather plus face fix-ups)
  float d[Q];
  if (sel != 0)
    gather_walled<0>(fn, plane, n, lidc, d);
  else
    gather<0>(fn, plane, n, d);
  float lam[Q];
  load_lambda(lam_in, plane, n, lam);

  const uint32_t dc = ((uint32_t)z * ny + y) * nx + x;
  float Fx = 0.f, Fy = 0.f, Fz = 0.f;
  if constexpr (FORCE) {
    Fx = LBM_LDG(force + dc);
    Fy = LBM_LDG(force + cells + dc);
    Fz = LBM_LDG(force + 2 * (size_t)cells + dc);
  }
  // the same FP32 arithmetic as the forward collision, so rho and u are
  // bit-identical to the ones lbm_step_moments stores
  float dr, jx, jy, jz;
  shifted_moments(d, dr, jx, jy, jz);
  const float rho = 1.0f + dr;
  const float rinv = __frcp_rn(rho);
  const float ux = fmaf(0.5f, Fx, jx) * rinv;
  const float uy = fmaf(0.5f, Fy, jy) * rinv;
  const float uz = fmaf(0.5f, Fz, jz) * rinv;
  adjoint_core<FORCE, GRADF>(lam, lam_out, gF, plane, n, sel, dc, cells, rho, ux, uy, uz, Fx,
                             Fy, Fz, omega, kf);
}

// One reverse step at node (x, y, z) from the moments rho^n, u^n that the
// forward step's collision used (dense fields, as lbm_step_moments writes
// them): no gather of f^n, 16 bytes per node instead of 76.
template <bool WALLS, bool FORCE, bool GRADF, bool L2ONLY = false>
__device__ __forceinline__ void adjoint_node_mom(
    const float *__restrict__ rho_n, const float *__restrict__ u_n,
    const float *__restrict__ lam_in, float *__restrict__ lam_out,
    const float *__restrict__ force, float *__restrict__ gF, int nx, int ny, int nz, int pitch,
    uint32_t plane, uint32_t walls, float omega, float kf, uint32_t cells, int x, int y, int z,
    bool wall_select = true) {
  const NodeIdx n = node_index(nx, ny, nz, pitch, WALLS ? walls : 0u, x, y, z);
  const int sel = scatter_mode<WALLS>(n, wall_select);
  const uint32_t dc = ((uint32_t)z * ny + y) * nx + x;
  float Fx = 0.f, Fy = 0.f, Fz = 0.f;
  if constexpr (FORCE) {
    Fx = LBM_LDG(force + dc);
    Fy = LBM_LDG(force + cells + dc);
    Fz = LBM_LDG(force + 2 * (size_t)cells + dc);
  }
  const float rho = LBM_LDG(rho_n + dc);
  const float ux = LBM_LDG(u_n + dc);
  const float uy = LBM_LDG(u_n + cells + dc);
  const float uz = LBM_LDG(u_n + 2 * (size_t)cells + dc);
  float lam[Q];
  load_lambda<L2ONLY>(lam_in, plane, n, lam);
  adjoint_core<FORCE, GRADF>(lam, lam_out, gF, plane, n, sel, dc, cells, rho, ux, uy, uz, Fx,
                             Fy, Fz, omega, kf);
}

// Loss seed at node (x, y, z) of a stored state f_T:
// lambda_j = (u - u_t) . (e_j - u) / rho with u = (sum e f - F/2)/rho, and the
// direct force term -(u - u_t)/(2 rho) written (not added) to gF when given.
// Returns the node's loss 1/2 |u - u_t|^2 in FP64.
template <bool FORCE>
__device__ __forceinline__ double seed_node(const float *__restrict__ f,
                                            const float *__restrict__ ut,
                                            float *__restrict__ lam, float *__restrict__ gF,
                                            const float *__restrict__ force, int nx, int ny,
                                            int pitch, uint32_t plane, uint32_t cells, int x,
                                            int y, int z) {
  const uint32_t c = ((uint32_t)z * ny + y) * pitch + x;
  const uint32_t dc = ((uint32_t)z * ny + y) * nx + x;
  float d[Q];
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    d[i] = LBM_LDG(f + (size_t)i * plane + c);
  });
  float dr, jx, jy, jz;
  shifted_moments(d, dr, jx, jy, jz);
  const float rho = 1.0f + dr, rinv = __frcp_rn(rho);
  float Fx = 0.f, Fy = 0.f, Fz = 0.f;
  if constexpr (FORCE) {
    Fx = LBM_LDG(force + dc);
    Fy = LBM_LDG(force + cells + dc);
    Fz = LBM_LDG(force + 2 * (size_t)cells + dc);
  }
  const float ux = fmaf(-0.5f, Fx, jx) * rinv;
  const float uy = fmaf(-0.5f, Fy, jy) * rinv;
  const float uz = fmaf(-0.5f, Fz, jz) * rinv;
  const float ex = ux - LBM_LDG(ut + dc);
  const float ey = uy - LBM_LDG(ut + cells + dc);
  const float ez = uz - LBM_LDG(ut + 2 * (size_t)cells + dc);
  const float du = fmaf(ex, ux, fmaf(ey, uy, ez * uz));
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr float cx = (float)kEx[i], cy = (float)kEy[i], cz = (float)kEz[i];
    LBM_ST(&lam[(size_t)i * plane + c], ((cx * ex + cy * ey + cz * ez) - du) * rinv);
  });
  if (gF) {
    const float h = -0.5f * rinv;
    LBM_ST(&gF[dc], h * ex);
    LBM_ST(&gF[cells + dc], h * ey);
    LBM_ST(&gF[2 * (size_t)cells + dc], h * ez);
  }
  return 0.5 * ((double)ex * ex + (double)ey * ey + (double)ez * ez);
}

// grad_u0 = sum_i lambda^0_i d f^eq_i(1, u0)/du0 = 3 L1 + 9 L2 u0 - 3 u0 L0
// at node (x, y, z); u0 may be null (zero).
__device__ __forceinline__ void u0grad_node(const float *__restrict__ lam0,
                                            const float *__restrict__ u0,
                                            float *__restrict__ grad, int nx, int ny, int pitch,
                                            uint32_t plane, uint32_t cells, int x, int y, int z) {
  const uint32_t c = ((uint32_t)z * ny + y) * pitch + x;
  const uint32_t dc = ((uint32_t)z * ny + y) * nx + x;
  float lam[Q];
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    lam[i] = LBM_LDG(lam0 + (size_t)i * plane + c);
  });
  float ux = 0.f, uy = 0.f, uz = 0.f;
  if (u0) {
    ux = LBM_LD(&u0[dc]);
    uy = LBM_LD(&u0[cells + dc]);
    uz = LBM_LD(&u0[2 * (size_t)cells + dc]);
  }
  const LamMoments m = lambda_moments(lam);
  float Lux, Luy, Luz;
  mat_vec(m.L2, ux, uy, uz, Lux, Luy, Luz);
  LBM_ST(&grad[dc], 3.0f * m.L1[0] + 9.0f * Lux - 3.0f * ux * m.L0);
  LBM_ST(&grad[cells + dc], 3.0f * m.L1[1] + 9.0f * Luy - 3.0f * uy * m.L0);
  LBM_ST(&grad[2 * (size_t)cells + dc], 3.0f * m.L1[2] + 9.0f * Luz - 3.0f * uz * m.L0);
}

// FP64 block sum of one value per thread; thread 0 writes it to *out.
template <int THREADS>
__device__ __forceinline__ void block_sum_to(double acc, double *out) {
  __shared__ double red[THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (wid == 0) {
    acc = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) LBM_ST(out, acc);
  }
}

}  // namespace lbm
