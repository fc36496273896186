// lbm_step_x4.cu - the fused step (Alg. 3) with four x-adjacent nodes
// (x0 .. x0 + 3, x0 a multiple of 4) per thread, no data exchange between
// threads (LBM_KERNEL_X4).
//
// What four nodes of one row share in the SoA layout:
//   * every direction's pulls for the group come from one row: one aligned
//     4-value (8-byte) load holds the values of x0 .. x0 + 3 of the source
//     row;
//   * the 10 directions with e_x != 0 pull x0 - e_x .. x0 + 3 - e_x, which
//     is that group shifted by one: the one value that falls outside it
//     (x0 - 1 for e_x = +1, x0 + 4 for e_x = -1) is a single extra load;
//   * the results leave as two aligned 2-value stores per direction.
// Loads per node drop from 14.5 (two-node kernel) to 7.25.
//
// Walls cost almost nothing: only the extra value ever crosses a row end, so
// an x wall just points that load at the node's own opposite direction
// (bounce-back), one address choice per direction and thread with no
// divergence; a y or z wall bounces every node of the group at once (the
// group shares y and z), so the whole 4-value load moves to the opposite
// direction's group at the node. A warp spans one row segment of 128 nodes,
// so the y/z decisions are uniform across it; a vote sends the warps of rows
// off the y and z walls down a path without them.
//
// Measured on GB300 against the two-node kernel (384^3, FP16): 235 instead of
// 306 instructions per node and walls for free (the cavity runs as fast as
// the periodic lattice), but the four nodes' loaded groups and values take
// 122 registers, 14 warps per SM, and the kernel waits on memory latency:
// 73.8 against 80.6 GLUPS periodic, 74.9 against 77.0 in the cavity; capping
// registers at 96 or 80 spills and loses more. 16-bit storage only (FP32,
// which needs twice the registers per group, ran at 36.8 against 46.3).
// The arithmetic per node is that of the one-node kernel, so the results are
// bit-identical. When nx is not a multiple of 4 the last group of a row holds
// 1 to 3 padding nodes, which are loaded, computed and stored into the row
// padding (never used; their field reads and writes are skipped).
#include "d3q19.cuh"
#include "internal.h"
#include "pack.cuh"
#include "stream.cuh"

namespace lbm {

// Per-thread geometry of a group of four nodes.
struct Group {
  uint32_t zo[3], yo[3];   // (plus, same, minus) row offsets, as in NodeIdx
  uint32_t row;            // the group's own row: zo[1] + yo[1]
  int x0, klast;           // first node; index of the last real node (0..3)
  bool first, last;        // the group holds x = 0 / x = nx - 1
  bool y0, y1, z0, z1;     // the row lies on a walled y / z face
};

__device__ __forceinline__ Group make_group(int nx, int ny, int nz, int pitch, uint32_t walls,
                                            int x0, int y, int z) {
  Group g;
  const uint32_t rowz = (uint32_t)ny * pitch;
  const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
  g.zo[0] = zp * rowz;
  g.zo[1] = z * rowz;
  g.zo[2] = zm * rowz;
  g.yo[0] = (uint32_t)yp * pitch;
  g.yo[1] = (uint32_t)y * pitch;
  g.yo[2] = (uint32_t)ym * pitch;
  g.row = g.zo[1] + g.yo[1];
  g.x0 = x0;
  g.first = x0 == 0;
  g.last = x0 + 4 >= nx;
  g.klast = g.last ? nx - 1 - x0 : 3;
  g.y0 = (walls & LBM_WALL_Y) && y == 0;
  g.y1 = (walls & LBM_WALL_Y) && y == ny - 1;
  g.z0 = (walls & LBM_WALL_Z) && z == 0;
  g.z1 = (walls & LBM_WALL_Z) && z == nz - 1;
  return g;
}

// Whether direction i's pull crosses a walled y or z face (the same for all
// four nodes of the group).
template <int i>
__device__ __forceinline__ bool bounces_yz(const Group &g) {
  constexpr int ey = kEy[i], ez = kEz[i];
  bool out = false;
  if constexpr (ey == 1) out |= g.y0;
  if constexpr (ey == -1) out |= g.y1;
  if constexpr (ez == 1) out |= g.z0;
  if constexpr (ez == -1) out |= g.z1;
  return out;
}

// Loads of direction i for the group: `raw` the 4 values of the source row
// at x0 (or, if the pull bounces on a y/z wall, the opposite direction at
// the group itself), `extra` the value beyond the group (x0 - 1 or the last
// real node + 1: periodically wrapped, or the bounced value at an x wall).
template <int S, bool YZ, int i>
__device__ __forceinline__ void load_dir(const typename Store<S>::T *__restrict__ fin,
                                         uint32_t plane, const Group &g, int nx, bool xw,
                                         typename Quad<S>::V &raw, float &extra, bool &bb) {
  using T = typename Store<S>::T;
  constexpr int ex = kEx[i], jy = 1 + kEy[i], jz = 1 + kEz[i];
  constexpr int io = kOpp_v<i>;
  const T *base = fin + (size_t)i * plane;
  const T *opp = fin + (size_t)io * plane;
  const uint32_t srow = g.zo[jz] + g.yo[jy];
  bb = YZ ? bounces_yz<i>(g) : false;
  const T *gp = base + srow + g.x0;
  if constexpr (YZ) {
    if (bb) gp = opp + g.row + g.x0;
  }
  raw = Quad<S>::load(gp);
  if constexpr (ex == 1) {
    const T *p = base + srow + (g.first ? nx - 1 : g.x0 - 1);
    if (xw && g.first) p = opp + g.row;  // node 0 on the x = 0 wall
    extra = Store<S>::ld(p);
  } else if constexpr (ex == -1) {
    const T *p = base + srow + (g.last ? 0 : g.x0 + 4);
    if (xw && g.last) p = opp + g.row + (nx - 1);  // the last node on the x wall
    extra = Store<S>::ld(p);
  }
}

// Pulled value of direction i at node k of the group.
template <int S, bool YZ, bool NX4, int i, int k>
__device__ __forceinline__ float node_val(const typename Quad<S>::V &raw, float extra, bool bb,
                                          int klast, const Group &g, const float (&lidc)[Q]) {
  constexpr int ex = kEx[i], ey = kEy[i], ez = kEz[i];
  float v;
  if constexpr (ex == 0) {
    v = Quad<S>::template get<k>(raw);
  } else if constexpr (ex == 1) {
    if constexpr (k == 0)
      v = extra;
    else
      v = Quad<S>::template get<k - 1>(raw);
  } else {  // e_x = -1: node k pulls x0 + k + 1
    if constexpr (k == 3) {
      v = extra;
    } else {
      v = Quad<S>::template get<k + 1>(raw);
      if constexpr (!NX4) v = k < klast ? v : extra;
    }
  }
  if constexpr (YZ) {
    if constexpr (ex != 0 && (ey != 0 || ez != 0)) {
      if (bb) v = Quad<S>::template get<k>(raw);  // bounced: the group's own values
    }
    if constexpr (ez == -1) v += g.z1 ? lidc[i] : 0.0f;  // the moving plane z = nz
  }
  return v;
}

// Loads, collisions and stores of one group; YZ: the row may lie on a y or z
// wall (the bounce tests and the lid term are compiled in).
template <int S, bool YZ, bool FORCE, bool MOM, bool NX4>
__device__ __forceinline__ void x4_group(const StepArgs &a, const Group &g, int y, int z,
                                         bool xw) {
  using T = typename Store<S>::T;
  using V = typename Quad<S>::V;
  const T *__restrict__ fin = static_cast<const T *>(a.fin);
  T *__restrict__ fout = static_cast<T *>(a.fout);
  V raw[Q];
  float extra[Q];
  bool bb[Q];
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    extra[i] = 0.0f;
    load_dir<S, YZ, i>(fin, a.plane, g, a.nx, xw, raw[i], extra[i], bb[i]);
  });
  const uint32_t dc0 = ((uint32_t)z * a.ny + y) * a.nx + g.x0;
  static_for<0, 2>([&](auto H) {
    constexpr int k0 = 2 * decltype(H)::value, k1 = k0 + 1;
    float d0[Q], d1[Q];
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      d0[i] = node_val<S, YZ, NX4, i, k0>(raw[i], extra[i], bb[i], g.klast, g, a.lidc);
      d1[i] = node_val<S, YZ, NX4, i, k1>(raw[i], extra[i], bb[i], g.klast, g, a.lidc);
    });
    const bool has0 = NX4 || k0 <= g.klast, has1 = NX4 || k1 <= g.klast;
    float F0x = 0.f, F0y = 0.f, F0z = 0.f, F1x = 0.f, F1y = 0.f, F1z = 0.f;
    if constexpr (FORCE) {
      if (has0) {
        F0x = LBM_LDG(a.force + dc0 + k0);
        F0y = LBM_LDG(a.force + a.cells + dc0 + k0);
        F0z = LBM_LDG(a.force + 2 * (size_t)a.cells + dc0 + k0);
      }
      if (has1) {
        F1x = LBM_LDG(a.force + dc0 + k1);
        F1y = LBM_LDG(a.force + a.cells + dc0 + k1);
        F1z = LBM_LDG(a.force + 2 * (size_t)a.cells + dc0 + k1);
      }
    }
    float r0, u0x, u0y, u0z, r1, u1x, u1y, u1z;
    collide<FORCE>(d0, a.omega, a.kf, F0x, F0y, F0z, r0, u0x, u0y, u0z);
    collide<FORCE>(d1, a.omega, a.kf, F1x, F1y, F1z, r1, u1x, u1y, u1z);
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      Pack16<S>::store(fout + (size_t)i * a.plane + g.row + g.x0 + k0, d0[i], d1[i]);
    });
    if constexpr (MOM) {
      if (has0) {
        LBM_ST(&a.rho[dc0 + k0], r0);
        LBM_ST(&a.u[dc0 + k0], u0x);
        LBM_ST(&a.u[a.cells + dc0 + k0], u0y);
        LBM_ST(&a.u[2 * (size_t)a.cells + dc0 + k0], u0z);
      }
      if (has1) {
        LBM_ST(&a.rho[dc0 + k1], r1);
        LBM_ST(&a.u[dc0 + k1], u1x);
        LBM_ST(&a.u[a.cells + dc0 + k1], u1y);
        LBM_ST(&a.u[2 * (size_t)a.cells + dc0 + k1], u1z);
      }
    }
  });
}

// W: 0 periodic, 1 walls (halfway bounce-back and lid). NX4: nx % 4 == 0
// (no padding nodes, no per-node choice at the row end).
template <int S, int W, bool FORCE, bool MOM, bool NX4>
__global__ void __launch_bounds__(256) k_step_x4(const StepArgs a) {
  const int x0 = 4 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = a.z0 + blockIdx.z;
  if (x0 >= a.nx || y >= a.ny) return;
  const uint32_t walls = W != 0 ? a.walls : 0u;
  const Group g = make_group(a.nx, a.ny, a.nz, a.pitch, walls, x0, y, z);
  if constexpr (W == 0) {
    x4_group<S, false, FORCE, MOM, NX4>(a, g, y, z, false);
  } else {
    const bool xw = (a.walls & LBM_WALL_X) != 0;
    // the vote covers the warp's active threads (the others have returned)
    if (__any_sync(__activemask(), g.y0 | g.y1 | g.z0 | g.z1))
      x4_group<S, true, FORCE, MOM, NX4>(a, g, y, z, xw);
    else
      x4_group<S, false, FORCE, MOM, NX4>(a, g, y, z, xw);
  }
}

template <int S, int W, bool F, bool M>
static void x4_launch(bool nx4, dim3 g, dim3 b, const StepArgs &a, cudaStream_t s) {
  if (nx4)
    k_step_x4<S, W, F, M, true><<<g, b, 0, s>>>(a);
  else
    k_step_x4<S, W, F, M, false><<<g, b, 0, s>>>(a);
}

template <int S>
static void x4_dispatch(bool moments, const StepArgs &a, dim3 g, dim3 b, cudaStream_t s) {
  const bool walls = a.walls != 0, force = a.force != nullptr, nx4 = (a.nx & 3) == 0;
  if (walls) {
    if (force)
      moments ? x4_launch<S, 1, true, true>(nx4, g, b, a, s)
              : x4_launch<S, 1, true, false>(nx4, g, b, a, s);
    else
      moments ? x4_launch<S, 1, false, true>(nx4, g, b, a, s)
              : x4_launch<S, 1, false, false>(nx4, g, b, a, s);
  } else {
    if (force)
      moments ? x4_launch<S, 0, true, true>(nx4, g, b, a, s)
              : x4_launch<S, 0, true, false>(nx4, g, b, a, s);
    else
      moments ? x4_launch<S, 0, false, true>(nx4, g, b, a, s)
              : x4_launch<S, 0, false, false>(nx4, g, b, a, s);
  }
}

cudaError_t launch_step_x4(int storage, bool moments, const StepArgs &a, int bxq, int by,
                           cudaStream_t s) {
  const int groups = (a.nx + 3) / 4;
  const dim3 g((groups + bxq - 1) / bxq, (a.ny + by - 1) / by, a.zn), b(bxq, by, 1);
  LBM_CHECK_TABLE(s, LBM_STEP_RANGES(a, elem_bytes_of(storage)));
  switch (storage) {
    case kF16: x4_dispatch<1>(moments, a, g, b, s); break;
    case kBF16: x4_dispatch<2>(moments, a, g, b, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lbm
