// lbm_step16.cu - the fused step for 16-bit storage (FP16 / BF16 of f_i - w_i)
// with two x-adjacent nodes per thread.
//
// Every direction plane is read and written as 32-bit pairs (x0, x0 + 1),
// x0 even: one 128-byte request per warp instead of two 64-byte ones, and
// twice the bytes in flight per load register. The pulls with e_x = +1 need
// (x0 - 1, x0) and those with e_x = -1 need (x0 + 1, x0 + 2): each lane
// loads the aligned pair of its own position in the source row and takes the
// missing half from its neighbour lane with a warp shuffle (the intra-warp
// propagation of Sec. 4.3.2, here applied to packed 16-bit pairs); lanes 0
// and 31 load the pair across the warp edge themselves. The arithmetic per
// node is exactly that of the one-node-per-thread kernel (same FP32
// collision, same round-to-nearest-even stores), so both produce identical
// bits.
#include "d3q19.cuh"
#include "internal.h"
#include "stream.cuh"

namespace lbm {

template <int S>
struct Pair16;

template <>
struct Pair16<1> {
  static __device__ __forceinline__ float lo(uint32_t v) {
    return __half2float(__ushort_as_half((unsigned short)(v & 0xffffu)));
  }
  static __device__ __forceinline__ float hi(uint32_t v) {
    return __half2float(__ushort_as_half((unsigned short)(v >> 16)));
  }
  static __device__ __forceinline__ float one(unsigned short v) {
    return __half2float(__ushort_as_half(v));
  }
  static __device__ __forceinline__ uint32_t bits(float f) {
    return (uint32_t)__half_as_ushort(__float2half_rn(f));
  }
};

template <>
struct Pair16<2> {
  static __device__ __forceinline__ float lo(uint32_t v) {
    return __bfloat162float(__ushort_as_bfloat16((unsigned short)(v & 0xffffu)));
  }
  static __device__ __forceinline__ float hi(uint32_t v) {
    return __bfloat162float(__ushort_as_bfloat16((unsigned short)(v >> 16)));
  }
  static __device__ __forceinline__ float one(unsigned short v) {
    return __bfloat162float(__ushort_as_bfloat16(v));
  }
  static __device__ __forceinline__ uint32_t bits(float f) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(f));
  }
};

constexpr unsigned kFull = 0xffffffffu;

// One node of the pair: gathered values from half `H` (0 = lo = x0,
// 1 = hi = x0 + 1) of the packed pulls, bounce-back fix-ups for walled faces,
// collision, and the result written back into the same half.
template <int S, bool WALLS, bool FORCE, bool MOM, int H>
__device__ __forceinline__ void pair_node(uint32_t (&V)[Q], const unsigned short *fin,
                                          const StepArgs &a, const NodeIdx &n, int x, int y,
                                          int z) {
  float d[Q];
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    d[i] = H == 0 ? Pair16<S>::lo(V[i]) : Pair16<S>::hi(V[i]);
  });
  if constexpr (WALLS) {
    if (on_wall(n)) {
      static_for<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if (bounces<i>(n)) {
          float v = Pair16<S>::one(LBM_LDG(fin + (size_t)kOpp_v<i> * a.plane + n.c));
          if constexpr (kEz[i] == -1) v += n.z1 ? a.lidc[i] : 0.0f;
          d[i] = v;
        }
      });
    }
  }
  const uint32_t dc = ((uint32_t)z * a.ny + y) * a.nx + x;
  float Fx = 0.f, Fy = 0.f, Fz = 0.f;
  if constexpr (FORCE) {
    Fx = LBM_LDG(a.force + dc);
    Fy = LBM_LDG(a.force + a.cells + dc);
    Fz = LBM_LDG(a.force + 2 * (size_t)a.cells + dc);
  }
  float rho, ux, uy, uz;
  collide<FORCE>(d, a.omega, a.kf, Fx, Fy, Fz, rho, ux, uy, uz);
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const uint32_t b = Pair16<S>::bits(d[i]);
    V[i] = H == 0 ? ((V[i] & 0xffff0000u) | b) : ((V[i] & 0x0000ffffu) | (b << 16));
  });
  if constexpr (MOM) {
    LBM_ST(&a.rho[dc], rho);
    LBM_ST(&a.u[dc], ux);
    LBM_ST(&a.u[a.cells + dc], uy);
    LBM_ST(&a.u[2 * (size_t)a.cells + dc], uz);
  }
}

#ifdef LBM_PAIR_MIN_BLOCKS
#define LBM_PAIR_BOUNDS __launch_bounds__(256, LBM_PAIR_MIN_BLOCKS)
#else
#define LBM_PAIR_BOUNDS __launch_bounds__(256)
#endif

template <int S, bool WALLS, bool FORCE, bool MOM>
__global__ void LBM_PAIR_BOUNDS k_step_pair(const StepArgs a) {
  const int lane = threadIdx.x & 31;
  const int x0 = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (y >= a.ny) return;  // uniform per warp: a warp lies in one row
  const int nx = a.nx, pitch = a.pitch;
  // pair offsets clamped into the padded row, so lanes past the row end and
  // the warp-edge loads stay in bounds (their values are never used)
  const int xc = min(x0, pitch - 2);
  const int xl = max(min(x0 - 2, pitch - 2), 0);
  const int xr = min(x0 + 2, pitch - 2);
  const unsigned short *fin = static_cast<const unsigned short *>(a.fin);
  unsigned short *fout = static_cast<unsigned short *>(a.fout);
  const NodeIdx n0 = node_index(nx, a.ny, a.nz, pitch, a.walls, min(x0, nx - 1), y, z);

  uint32_t V[Q];
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int ex = kEx[i], jy = 1 + kEy[i], jz = 1 + kEz[i];
    const unsigned short *row = fin + (size_t)i * a.plane + n0.zo[jz] + n0.yo[jy];
    const uint32_t P = LBM_LDG(reinterpret_cast<const unsigned int *>(row + xc));
    if constexpr (ex == 0) {
      V[i] = P;
    } else if constexpr (ex == 1) {
      // (x0 - 1, x0): high half of the pair at x0 - 2, low half of P
      uint32_t Pp = __shfl_up_sync(kFull, P, 1);
      if (lane == 0)
        Pp = x0 >= 2 ? LBM_LDG(reinterpret_cast<const unsigned int *>(row + xl))
                     : ((uint32_t)LBM_LDG(row + nx - 1) << 16);  // periodic: x = -1
      V[i] = __byte_perm(Pp, P, 0x5432);
    } else {
      // (x0 + 1, x0 + 2): high half of P, low half of the pair at x0 + 2
      uint32_t Pn = __shfl_down_sync(kFull, P, 1);
      if (lane == 31) Pn = LBM_LDG(reinterpret_cast<const unsigned int *>(row + xr));
      uint32_t v = __byte_perm(P, Pn, 0x5432);
      if (x0 + 2 == nx) v = (v & 0x0000ffffu) | ((uint32_t)LBM_LDG(row) << 16);  // x = nx
      if (x0 + 1 == nx) v = (v & 0xffff0000u) | (uint32_t)LBM_LDG(row);          // x = nx
      V[i] = v;
    }
  });

  if (x0 >= nx) return;
  pair_node<S, WALLS, FORCE, MOM, 0>(V, fin, a, n0, x0, y, z);
  if (x0 + 1 < nx) {
    const NodeIdx n1 = node_index(nx, a.ny, a.nz, pitch, a.walls, x0 + 1, y, z);
    pair_node<S, WALLS, FORCE, MOM, 1>(V, fin, a, n1, x0 + 1, y, z);
  }
  // the high half of the last pair of an odd-length row lands in the padding
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    LBM_ST(reinterpret_cast<unsigned int *>(fout + (size_t)i * a.plane + n0.c - n0.xo[1] + x0),
           V[i]);
  });
}

template <int S>
static void pair_dispatch(bool moments, const StepArgs &a, dim3 g, dim3 b, cudaStream_t s) {
  const bool walls = a.walls != 0, force = a.force != nullptr;
#define LBM_PAIR_CASE(W, F, M)                                  \
  if (walls == W && force == F && moments == M) {               \
    k_step_pair<S, W, F, M><<<g, b, 0, s>>>(a);                 \
    return;                                                     \
  }
  LBM_PAIR_CASE(false, false, false)
  LBM_PAIR_CASE(false, false, true)
  LBM_PAIR_CASE(false, true, false)
  LBM_PAIR_CASE(false, true, true)
  LBM_PAIR_CASE(true, false, false)
  LBM_PAIR_CASE(true, false, true)
  LBM_PAIR_CASE(true, true, false)
  LBM_PAIR_CASE(true, true, true)
#undef LBM_PAIR_CASE
}

cudaError_t launch_step_pair16(int storage, bool moments, const StepArgs &a, int bxp, int by,
                               cudaStream_t s) {
  const int pairs = (a.nx + 1) / 2;
  const dim3 g((pairs + bxp - 1) / bxp, (a.ny + by - 1) / by, a.nz), b(bxp, by, 1);
  LBM_CHECK_TABLE(s, LBM_STEP_RANGES(a, elem_bytes_of(storage)));
  switch (storage) {
    case kF16: pair_dispatch<1>(moments, a, g, b, s); break;
    case kBF16: pair_dispatch<2>(moments, a, g, b, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lbm
