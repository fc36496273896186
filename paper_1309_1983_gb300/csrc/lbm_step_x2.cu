// lbm_step_x2.cu - the fused step (Alg. 3) with two x-adjacent nodes
// (x0, x0 + 1), x0 even, per thread and no data exchange between threads;
// the default step kernel for every storage type.
//
// The two nodes of a pair share what the SoA layout lets them share:
//   * the 9 directions with e_x = 0 pull (x0, x0 + 1) from the same row: one
//     aligned 8-byte (FP32) or 4-byte (16-bit) load per pair;
//   * the 10 directions with e_x != 0 pull from x0 - e_x and x0 + 1 - e_x,
//     an odd offset: two single-value loads (the misaligned-read variant of
//     Sec. 4.3.2, as in the one-node kernel);
//   * all 19 results leave as one aligned two-value store per pair (for
//     16-bit storage after one two-value conversion).
// With 16-bit values the one-node kernel is bound by instruction issue (half
// the bytes per node means twice the nodes per second, and every node still
// pays 19 loads, 19 stores, their addresses and 38 conversions): sharing
// them takes 40 instructions per node off. With FP32 the kernel is
// DRAM-bound and the pairs add about 1% of throughput.
// The arithmetic per node is that of the one-node kernel (same collision,
// same round-to-nearest-even conversions), so both produce identical bits.
// On an odd-length row the last pair's second node lies in the row padding
// (the pitch is a multiple of 32 bytes): it is loaded and stored but never
// used.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "d3q19.cuh"
#include "internal.h"
#include "onsite.cuh"
#include "pack.cuh"
#include "stream.cuh"

namespace lbm {

// Pulled values of both nodes for direction i (bounce-back by address
// selection when SEL; the e_x = 0 pulls of the pair share y, z, hence their
// wall decisions, so they stay one paired load).
//
// Two ways of forming the addresses, the same values: RAW = true (the
// periodic kernel) adds one 64-bit index i * plane + offset to the base;
// RAW = false (the kernels with walls) selects a 32-bit plane number and a
// 32-bit offset in it and adds plane * number, then the offset, to the base.
// The second form lets ptxas keep the 16-bit wall kernels at 64 registers
// instead of 70-80 (8 resident blocks of 128 threads per SM instead of 6-7):
// +3.6% for the FP16 cavity at 384^3 (81.8 against 79.0 GLUPS), +5.4% with
// on-site walls; the periodic kernels keep the first form, which the second
// slows by 0.5% (FP16), and so do the FP32 on-site kernel (0.2%) and the
// wall-node branch form (W = 2, whose registers it raises).
template <int S, bool SEL, int i, bool RAW = false>
__device__ __forceinline__ void pull_pair(const typename Store<S>::T *__restrict__ fin,
                                          uint32_t plane, const NodeIdx &n0, const NodeIdx &n1,
                                          const float (&lidc)[Q], float &v0, float &v1) {
  static_assert(!(RAW && SEL), "the selecting pull uses the plane / offset form");
  if constexpr (RAW) {
    if constexpr (kEx[i] == 0) {
      size_t idx = (size_t)i * plane + source_of<i>(n0);
      const float2 p = Pack16<S>::load(fin + idx);
      v0 = p.x;
      v1 = p.y;
    } else {
      size_t i0 = (size_t)i * plane + source_of<i>(n0);
      size_t i1 = (size_t)i * plane + source_of<i>(n1);
      v0 = Store<S>::ld(fin + i0);
      v1 = Store<S>::ld(fin + i1);
    }
  } else if constexpr (kEx[i] == 0) {
    uint32_t pl = (uint32_t)i, off = source_of<i>(n0);
    if constexpr (SEL) {
      if (bounces<i>(n0)) {
        pl = (uint32_t)kOpp_v<i>;
        off = n0.c;
      }
    }
    const float2 p = Pack16<S>::load(fin + (size_t)pl * plane + off);
    v0 = p.x;
    v1 = p.y;
  } else {
    uint32_t p0 = (uint32_t)i, o0 = source_of<i>(n0);
    uint32_t p1 = (uint32_t)i, o1 = source_of<i>(n1);
    if constexpr (SEL) {
      if (bounces<i>(n0)) {
        p0 = (uint32_t)kOpp_v<i>;
        o0 = n0.c;
      }
      if (bounces<i>(n1)) {
        p1 = (uint32_t)kOpp_v<i>;
        o1 = n1.c;
      }
    }
    v0 = Store<S>::ld(fin + (size_t)p0 * plane + o0);
    v1 = Store<S>::ld(fin + (size_t)p1 * plane + o1);
  }
  if constexpr (SEL && kEz[i] == -1) {  // the moving plane z = nz (z1 implies a bounce)
    v0 += n0.z1 ? lidc[i] : 0.0f;
    v1 += n1.z1 ? lidc[i] : 0.0f;
  }
}

// Pulled values of both nodes in a warp whose only wall nodes lie on the x
// faces: the e_x = 0 pulls cannot bounce there, an e_x = +1 pull bounces only
// on the x = 0 node and an e_x = -1 pull only on the x = nx - 1 node (no lid
// term: the lid is the z = nz plane).
template <int S, int i>
__device__ __forceinline__ void pull_pair_xwall(const typename Store<S>::T *__restrict__ fin,
                                                uint32_t plane, const NodeIdx &n0,
                                                const NodeIdx &n1, float &v0, float &v1) {
  if constexpr (kEx[i] == 0) {
    const float2 p = Pack16<S>::load(fin + (size_t)i * plane + source_of<i>(n0));
    v0 = p.x;
    v1 = p.y;
  } else {
    constexpr uint32_t io = kOpp_v<i>;
    const bool b0 = kEx[i] == 1 ? n0.x0 : n0.x1;
    const bool b1 = kEx[i] == 1 ? n1.x0 : n1.x1;
    const uint32_t p0 = b0 ? io : (uint32_t)i, o0 = b0 ? n0.c : source_of<i>(n0);
    const uint32_t p1 = b1 ? io : (uint32_t)i, o1 = b1 ? n1.c : source_of<i>(n1);
    v0 = Store<S>::ld(fin + (size_t)p0 * plane + o0);
    v1 = Store<S>::ld(fin + (size_t)p1 * plane + o1);
  }
}

// Launch bounds: by default only the block size is fixed (64 registers for
// the 16-bit kernels with halfway or on-site walls and without, 72 for the
// periodic FP32 kernel, up to 80 with walls, force or fused moments);
// LBM_X2_MIN_BLOCKS asks for that
// many resident 256-thread blocks per SM instead (tuning experiments).
#ifdef LBM_X2_MIN_BLOCKS
#define LBM_X2_BOUNDS __launch_bounds__(256, LBM_X2_MIN_BLOCKS)
#else
#define LBM_X2_BOUNDS __launch_bounds__(256)
#endif

// W: 0 periodic, 1 walls by address selection in the warps that hold a wall
// node (warp votes pick, per warp, full selection where a y or z wall node
// is present, selection of the ten e_x != 0 pulls where only x wall nodes
// are, and the plain pulls elsewhere: no divergence; 5-14% faster than
// selecting in every warp, and the x-only path another 0.6-1.4%), 2 walls by
// the wall-node branch (the one-node kernel's face fix-ups, per node of the
// pair), 3 on-site velocity walls (plain pulls, then the rule of onsite.cuh
// on each wall node of the pair).
template <int S, int W, bool FORCE, bool MOM>
__global__ void LBM_X2_BOUNDS k_step_x2(const StepArgs a) {
  using T = typename Store<S>::T;
  const int x0 = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = a.z0 + blockIdx.z;
  if (x0 >= a.nx || y >= a.ny) return;
  const bool has1 = x0 + 1 < a.nx;
  const T *__restrict__ fin = static_cast<const T *>(a.fin);
  T *__restrict__ fout = static_cast<T *>(a.fout);
  const uint32_t walls = W != 0 ? a.walls : 0u;
  const NodeIdx n0 = node_index(a.nx, a.ny, a.nz, a.pitch, walls, x0, y, z);
  // the padding node of an odd row pulls what node 0 pulls (in bounds, unused)
  const NodeIdx n1 = node_index(a.nx, a.ny, a.nz, a.pitch, walls, has1 ? x0 + 1 : x0, y, z);

  float d0[Q], d1[Q];
  if constexpr (W == 1) {
    // the votes cover the warp's active threads (the others have returned);
    // the pair shares y and z, so n0 decides the y / z faces for both
    const unsigned m = __activemask();
    if (__any_sync(m, n0.y0 | n0.y1 | n0.z0 | n0.z1)) {
      static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        pull_pair<S, true, i>(fin, a.plane, n0, n1, a.lidc, d0[i], d1[i]);
      });
    } else if (__any_sync(m, n0.x0 | n0.x1 | n1.x1)) {
      static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        pull_pair_xwall<S, i>(fin, a.plane, n0, n1, d0[i], d1[i]);
      });
    } else {
      static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        pull_pair<S, false, i>(fin, a.plane, n0, n1, a.lidc, d0[i], d1[i]);
      });
    }
  } else {
    // the periodic kernel, the wall-node branch form and the FP32 on-site
    // kernel keep the 64-bit index form (see pull_pair)
    constexpr bool RAW = W == 0 || W == 2 || (W == 3 && S == 0);
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      pull_pair<S, false, i, RAW>(fin, a.plane, n0, n1, a.lidc, d0[i], d1[i]);
    });
  }
  if constexpr (W == 2) {
    bounce_fixup<S>(fin, a.plane, n0, a.lidc, d0);
    if (has1) bounce_fixup<S>(fin, a.plane, n1, a.lidc, d1);
  }
  const uint32_t dc = ((uint32_t)z * a.ny + y) * a.nx + x0;
  float F0x = 0.f, F0y = 0.f, F0z = 0.f, F1x = 0.f, F1y = 0.f, F1z = 0.f;
  if constexpr (FORCE) {
    F0x = LBM_LDG(a.force + dc);
    F0y = LBM_LDG(a.force + a.cells + dc);
    F0z = LBM_LDG(a.force + 2 * (size_t)a.cells + dc);
    if (has1) {
      F1x = LBM_LDG(a.force + dc + 1);
      F1y = LBM_LDG(a.force + a.cells + dc + 1);
      F1z = LBM_LDG(a.force + 2 * (size_t)a.cells + dc + 1);
    }
  }
  if constexpr (W == 3) {
    if (on_wall(n0)) onsite_apply<S>(fin, a, n0, F0x, F0y, F0z, d0);
    if (has1 && on_wall(n1)) onsite_apply<S>(fin, a, n1, F1x, F1y, F1z, d1);
  }
  float r0, u0x, u0y, u0z, r1, u1x, u1y, u1z;
  collide<FORCE>(d0, a.omega, a.kf, F0x, F0y, F0z, r0, u0x, u0y, u0z);
  collide<FORCE>(d1, a.omega, a.kf, F1x, F1y, F1z, r1, u1x, u1y, u1z);
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    Pack16<S>::store(fout + (size_t)i * a.plane + n0.c, d0[i], d1[i]);
  });
  if constexpr (MOM) {
    LBM_ST(&a.rho[dc], r0);
    LBM_ST(&a.u[dc], u0x);
    LBM_ST(&a.u[a.cells + dc], u0y);
    LBM_ST(&a.u[2 * (size_t)a.cells + dc], u0z);
    if (has1) {
      LBM_ST(&a.rho[dc + 1], r1);
      LBM_ST(&a.u[dc + 1], u1x);
      LBM_ST(&a.u[a.cells + dc + 1], u1y);
      LBM_ST(&a.u[2 * (size_t)a.cells + dc + 1], u1z);
    }
  }
}

template <int S>
static void x2_dispatch(bool moments, const StepArgs &a, dim3 g, dim3 b, cudaStream_t s) {
  const int walls = a.walls == 0 ? 0 : a.onsite ? 3 : a.wall_select ? 1 : 2;
  const bool force = a.force != nullptr;
#define LBM_X2_CASE(W, F, M)                                    \
  if (walls == W && force == F && moments == M) {               \
    k_step_x2<S, W, F, M><<<g, b, 0, s>>>(a);                   \
    return;                                                     \
  }
  LBM_X2_CASE(0, false, false)
  LBM_X2_CASE(0, false, true)
  LBM_X2_CASE(0, true, false)
  LBM_X2_CASE(0, true, true)
  LBM_X2_CASE(1, false, false)
  LBM_X2_CASE(1, false, true)
  LBM_X2_CASE(1, true, false)
  LBM_X2_CASE(1, true, true)
  LBM_X2_CASE(2, false, false)
  LBM_X2_CASE(2, false, true)
  LBM_X2_CASE(2, true, false)
  LBM_X2_CASE(2, true, true)
  LBM_X2_CASE(3, false, false)
  LBM_X2_CASE(3, false, true)
  LBM_X2_CASE(3, true, false)
  LBM_X2_CASE(3, true, true)
#undef LBM_X2_CASE
}

cudaError_t launch_step_x2(int storage, bool moments, const StepArgs &a, int bxp, int by,
                           cudaStream_t s) {
  const int pairs = (a.nx + 1) / 2;
  const dim3 g((pairs + bxp - 1) / bxp, (a.ny + by - 1) / by, a.zn), b(bxp, by, 1);
  LBM_CHECK_TABLE(s, LBM_STEP_RANGES(a, elem_bytes_of(storage)));
  switch (storage) {
    case kF32: x2_dispatch<0>(moments, a, g, b, s); break;
    case kF16: x2_dispatch<1>(moments, a, g, b, s); break;
    case kBF16: x2_dispatch<2>(moments, a, g, b, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lbm
