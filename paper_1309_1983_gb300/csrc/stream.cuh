// stream.cuh - node indexing for the pull gather (Alg. 3, first loop), the
// halfway bounce-back rule, and the transposed (scatter) form used by the
// adjoint. Shared by the forward and adjoint kernels.
#pragma once

#include "d3q19.cuh"
#include "internal.h"

namespace lbm {

// Offsets of a node and of its wrapped neighbours inside one direction
// plane of a pitched buffer, plus the walled faces the node touches.
struct NodeIdx {
  uint32_t zo[3], yo[3], xo[3];  // (plus, same, minus) neighbour per axis
  uint32_t c;                    // the node itself
  bool x0, x1, y0, y1, z0, z1;   // node on a walled low/high face
};

__device__ __forceinline__ NodeIdx node_index(int nx, int ny, int nz, int pitch,
                                              uint32_t walls, int x, int y,
                                              int z) {
  NodeIdx n;
  const uint32_t row = (uint32_t)ny * pitch;
  const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
  n.zo[0] = zp * row;
  n.zo[1] = z * row;
  n.zo[2] = zm * row;
  n.yo[0] = (uint32_t)yp * pitch;
  n.yo[1] = (uint32_t)y * pitch;
  n.yo[2] = (uint32_t)ym * pitch;
  n.xo[0] = (uint32_t)xp;
  n.xo[1] = (uint32_t)x;
  n.xo[2] = (uint32_t)xm;
  n.c = n.zo[1] + n.yo[1] + n.xo[1];
  n.x0 = (walls & LBM_WALL_X) && x == 0;
  n.x1 = (walls & LBM_WALL_X) && x == nx - 1;
  n.y0 = (walls & LBM_WALL_Y) && y == 0;
  n.y1 = (walls & LBM_WALL_Y) && y == ny - 1;
  n.z0 = (walls & LBM_WALL_Z) && z == 0;
  n.z1 = (walls & LBM_WALL_Z) && z == nz - 1;
  return n;
}

__device__ __forceinline__ bool on_wall(const NodeIdx &n) {
  return n.x0 | n.x1 | n.y0 | n.y1 | n.z0 | n.z1;
}

// Index of the source node x - e_i (periodically wrapped) in its plane. The
// offset tables hold (plus, same, minus) neighbours, so e = +1 (source at
// minus) is entry 2 and e = -1 is entry 0.
template <int i>
__device__ __forceinline__ uint32_t source_of(const NodeIdx &n) {
  constexpr int jx = 1 + kEx[i], jy = 1 + kEy[i], jz = 1 + kEz[i];
  return n.zo[jz] + n.yo[jy] + n.xo[jx];
}

// True when x - e_i lies outside a walled axis (bounce-back applies).
template <int i>
__device__ __forceinline__ bool bounces(const NodeIdx &n) {
  constexpr int ex = kEx[i], ey = kEy[i], ez = kEz[i];
  bool out = false;
  if constexpr (ex == 1) out |= n.x0;
  if constexpr (ex == -1) out |= n.x1;
  if constexpr (ey == 1) out |= n.y0;
  if constexpr (ey == -1) out |= n.y1;
  if constexpr (ez == 1) out |= n.z0;
  if constexpr (ez == -1) out |= n.z1;
  return out;
}

// Pull gather with periodic wrap on every axis: d_i = f_i(x - e_i).
template <int S, bool L2ONLY = false>
__device__ __forceinline__ void gather(const typename Store<S>::T *__restrict__ fin,
                                       uint32_t plane, const NodeIdx &n,
                                       float (&d)[Q]) {
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    d[i] = load_f<S, L2ONLY>(fin + (size_t)i * plane + source_of<i>(n));
  });
}

// Pull gather with the halfway bounce-back rule folded into the addresses:
// d_i = f_i(x - e_i), or f_ibar(x) + 6 w_i (e_i . u_w) when x - e_i lies
// outside a walled axis; u_w is the lid velocity when that source lies on
// the plane z = nz (e_z = -1 at the top face), pre-multiplied into
// lidc[i] = 6 w_i (e_i . u_w) by the host. Each direction is one load whose
// address is selected per node, so nodes on and off the walls run the same
// instructions (no divergence in warps that touch a wall).
template <int S, bool L2ONLY = false>
__device__ __forceinline__ void gather_walled(const typename Store<S>::T *__restrict__ fin,
                                              uint32_t plane, const NodeIdx &n,
                                              const float (&lidc)[Q], float (&d)[Q]) {
  d[0] = load_f<S, L2ONLY>(fin + n.c);
  static_for<1, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const bool bb = bounces<i>(n);
    const size_t idx = bb ? (size_t)kOpp_v<i> * plane + n.c
                          : (size_t)i * plane + source_of<i>(n);
    float v = load_f<S, L2ONLY>(fin + idx);
    if constexpr (kEz[i] == -1) v += n.z1 ? lidc[i] : 0.0f;  // z1 implies bb here
    d[i] = v;
  });
}

// Pull gather for a node whose warp holds x-wall nodes but no y or z wall
// node: only the ten e_x != 0 pulls can bounce, e_x = +1 ones on the x = 0
// node and e_x = -1 ones on the x = nx - 1 node (no lid term: the lid is the
// z = nz plane).
template <int S, bool L2ONLY = false>
__device__ __forceinline__ void gather_xwall(const typename Store<S>::T *__restrict__ fin,
                                             uint32_t plane, const NodeIdx &n, float (&d)[Q]) {
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (kEx[i] == 0) {
      d[i] = load_f<S, L2ONLY>(fin + (size_t)i * plane + source_of<i>(n));
    } else {
      const bool b = kEx[i] == 1 ? n.x0 : n.x1;
      const size_t idx = b ? (size_t)kOpp_v<i> * plane + n.c : (size_t)i * plane + source_of<i>(n);
      d[i] = load_f<S, L2ONLY>(fin + idx);
    }
  });
}

// Value of a bounced pull: f_ibar(x), plus the moving-wall term when the
// outside source x - e_i lies on the plane z = nz (e_z = -1 at the top face).
template <int S, bool L2ONLY, int i>
__device__ __forceinline__ float bounced_value(const typename Store<S>::T *__restrict__ fin,
                                               uint32_t plane, const NodeIdx &n,
                                               const float (&lidc)[Q]) {
  float v = load_f<S, L2ONLY>(fin + (size_t)kOpp_v<i> * plane + n.c);
  if constexpr (kEz[i] == -1) v += n.z1 ? lidc[i] : 0.0f;
  return v;
}

// Re-read, on a node of one walled face, the directions whose pull source
// lies beyond that face: component `axis` of e_i equal to `sgn`.
template <int S, bool L2ONLY, int axis, int sgn>
__device__ __forceinline__ void fix_face(const typename Store<S>::T *__restrict__ fin,
                                         uint32_t plane, const NodeIdx &n,
                                         const float (&lidc)[Q], float (&d)[Q]) {
  static_for<1, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int e = axis == 0 ? kEx[i] : axis == 1 ? kEy[i] : kEz[i];
    if constexpr (e == sgn) d[i] = bounced_value<S, L2ONLY, i>(fin, plane, n, lidc);
  });
}

// Halfway bounce-back applied after a plain periodic gather, only on nodes
// that touch a walled face (a branch; cheaper than gather_walled when wall
// nodes are a small fraction of each warp's nodes, i.e. on long rows). Each
// face re-reads only its five inward directions; a direction bouncing on two
// faces (edges, corners) is written twice with the same value.
template <int S, bool L2ONLY = false>
__device__ __forceinline__ void bounce_fixup(const typename Store<S>::T *__restrict__ fin,
                                             uint32_t plane, const NodeIdx &n,
                                             const float (&lidc)[Q], float (&d)[Q]) {
  if (n.x0) fix_face<S, L2ONLY, 0, 1>(fin, plane, n, lidc, d);
  if (n.x1) fix_face<S, L2ONLY, 0, -1>(fin, plane, n, lidc, d);
  if (n.y0) fix_face<S, L2ONLY, 1, 1>(fin, plane, n, lidc, d);
  if (n.y1) fix_face<S, L2ONLY, 1, -1>(fin, plane, n, lidc, d);
  if (n.z0) fix_face<S, L2ONLY, 2, 1>(fin, plane, n, lidc, d);
  if (n.z1) fix_face<S, L2ONLY, 2, -1>(fin, plane, n, lidc, d);
}

// One fused update of node (x, y, z) (Alg. 3): pull gather, boundary rule,
// moments, equilibrium, BGK (+ Guo force) collide, aligned store of the 19
// post-collision values at the node; optionally also rho and u into dense
// fields at index dc. Used by the single-lattice and the batched kernels.
// With wall_select, VOTE = true chooses the gather per warp (every face where
// a y or z wall node is present, the x faces only where only x wall nodes
// are, none elsewhere) instead of selecting on every face in every warp:
// 4.0% faster for the batched step sequence with moments (the adjoint's
// segment recompute) and 1.0% without, 0.5% slower for the persistent
// stepping kernel, which keeps per-node selection.
template <int S, bool WALLS, bool FORCE, bool MOM, bool L2ONLY, bool VOTE = false>
__device__ __forceinline__ void step_node(
    const typename Store<S>::T *__restrict__ fin, typename Store<S>::T *__restrict__ fout,
    int nx, int ny, int nz, int pitch, uint32_t plane, uint32_t walls,
    const float (&lidc)[Q], float omega, float kf, const float *__restrict__ force,
    float *__restrict__ rho_out, float *__restrict__ u_out, uint32_t cells, int x, int y,
    int z, bool wall_select = true) {
  const NodeIdx n = node_index(nx, ny, nz, pitch, walls, x, y, z);
  float d[Q];
  if constexpr (WALLS) {
    if (wall_select && VOTE) {
      const unsigned m = __activemask();
      if (__any_sync(m, n.y0 | n.y1 | n.z0 | n.z1))
        gather_walled<S, L2ONLY>(fin, plane, n, lidc, d);
      else if (__any_sync(m, n.x0 | n.x1))
        gather_xwall<S, L2ONLY>(fin, plane, n, d);
      else
        gather<S, L2ONLY>(fin, plane, n, d);
    } else if (wall_select) {
      gather_walled<S, L2ONLY>(fin, plane, n, lidc, d);
    } else {
      gather<S, L2ONLY>(fin, plane, n, d);
      bounce_fixup<S, L2ONLY>(fin, plane, n, lidc, d);
    }
  } else {
    gather<S, L2ONLY>(fin, plane, n, d);
  }
  const uint32_t dc = ((uint32_t)z * ny + y) * nx + x;
  float Fx = 0.f, Fy = 0.f, Fz = 0.f;
  if constexpr (FORCE) {
    Fx = LBM_LDG(force + dc);
    Fy = LBM_LDG(force + cells + dc);
    Fz = LBM_LDG(force + 2 * (size_t)cells + dc);
  }
  float rho, ux, uy, uz;
  collide<FORCE>(d, omega, kf, Fx, Fy, Fz, rho, ux, uy, uz);
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    Store<S>::st(fout + (size_t)i * plane + n.c, d[i]);
  });
  if constexpr (MOM) {
    LBM_ST(&rho_out[dc], rho);
    LBM_ST(&u_out[dc], ux);
    LBM_ST(&u_out[cells + dc], uy);
    LBM_ST(&u_out[2 * (size_t)cells + dc], uz);
  }
}

}  // namespace lbm
