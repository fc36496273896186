// lbm_push.cu - the streaming-order ablation of Sec. 4.2-4.3: the push
// iteration (Alg. 2) next to the pull iteration (Alg. 3) used everywhere
// else, and streaming alone in either form.
//
// Push keeps the POST-STREAMING distributions g as its state: each node reads
// its own 19 values (aligned), collides, and scatters f*_i to x + e_i
// (misaligned writes for e_x != 0); when x + e_i lies outside a walled axis
// the value comes back as direction ibar at x, plus 6 w_ibar (e_ibar . u_w)
// with u_w the lid velocity if that outside node lies on the plane z = nz.
// Every element of the output is written exactly once. With g^0 = P f^0 the
// push states are g^n = P f^n, P the pull streaming with bounce-back.
//
// k_stream applies P alone: form 0 gathers (misaligned reads, aligned
// writes), form 1 scatters (aligned reads, misaligned writes); form 2 is an
// unshifted copy of the 19 planes, the bandwidth reference; form 3 gathers
// with L2-only loads (no L1 or read-only cache: the paper's measurement of
// misaligned reads without the read-only data cache).
#include "d3q19.cuh"
#include "internal.h"
#include "stream.cuh"

namespace lbm {

// Target of the push of direction i from node n: plane index and position.
template <int i>
__device__ __forceinline__ void push_target(const NodeIdx &n, uint32_t plane, size_t &idx,
                                            bool &bounced) {
  // x + e_i is the pull source of x for the opposite direction
  bounced = bounces<kOpp_v<i>>(n);
  idx = bounced ? (size_t)kOpp_v<i> * plane + n.c
                : (size_t)i * plane + source_of<kOpp_v<i>>(n);
}

template <int S, bool WALLS, bool FORCE>
__global__ void __launch_bounds__(256) k_step_push(const StepArgs a) {
  using T = typename Store<S>::T;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= a.nx || y >= a.ny) return;
  const T *__restrict__ gin = static_cast<const T *>(a.fin);
  T *__restrict__ gout = static_cast<T *>(a.fout);
  const NodeIdx n = node_index(a.nx, a.ny, a.nz, a.pitch, a.walls, x, y, z);
  float d[Q];
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    d[i] = Store<S>::ld(gin + (size_t)i * a.plane + n.c);
  });
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
    if constexpr (WALLS) {
      size_t idx;
      bool bb;
      push_target<i>(n, a.plane, idx, bb);
      float v = d[i];
      // the bounced value is direction ibar at x; its source x - e_ibar = x + e_i
      // lies on the moving plane when e_i.z = +1 at the top face
      if constexpr (kEz[i] == 1) v += (bb && n.z1) ? a.lidc[kOpp_v<i>] : 0.0f;
      Store<S>::st(gout + idx, v);
    } else {
      Store<S>::st(gout + (size_t)i * a.plane + source_of<kOpp_v<i>>(n), d[i]);
    }
  });
}

template <int S>
__global__ void __launch_bounds__(256) k_stream(const StepArgs a, int form) {
  using T = typename Store<S>::T;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= a.nx || y >= a.ny) return;
  const T *__restrict__ fin = static_cast<const T *>(a.fin);
  T *__restrict__ fout = static_cast<T *>(a.fout);
  const NodeIdx n = node_index(a.nx, a.ny, a.nz, a.pitch, a.walls, x, y, z);
  if (form == 0 || form == 3) {  // gather: misaligned reads, aligned writes
    float d[Q];
    if (form == 3) {  // through L2 only
      if (a.walls)
        gather_walled<S, true>(fin, a.plane, n, a.lidc, d);
      else
        gather<S, true>(fin, a.plane, n, d);
    } else if (a.walls) {
      gather_walled<S>(fin, a.plane, n, a.lidc, d);
    } else {
      gather<S>(fin, a.plane, n, d);
    }
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      Store<S>::st(fout + (size_t)i * a.plane + n.c, d[i]);
    });
  } else if (form == 1) {  // scatter: aligned reads, misaligned writes
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      float v = Store<S>::ld(fin + (size_t)i * a.plane + n.c);
      size_t idx;
      bool bb;
      push_target<i>(n, a.plane, idx, bb);
      if constexpr (kEz[i] == 1) v += (bb && n.z1) ? a.lidc[kOpp_v<i>] : 0.0f;
      Store<S>::st(fout + idx, v);
    });
  } else {  // unshifted copy (bandwidth reference)
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      Store<S>::st(fout + (size_t)i * a.plane + n.c,
                   Store<S>::ld(fin + (size_t)i * a.plane + n.c));
    });
  }
}

template <int S>
static void push_dispatch(const StepArgs &a, dim3 g, dim3 b, cudaStream_t s) {
  const bool walls = a.walls != 0, force = a.force != nullptr;
  if (walls && force) k_step_push<S, true, true><<<g, b, 0, s>>>(a);
  else if (walls) k_step_push<S, true, false><<<g, b, 0, s>>>(a);
  else if (force) k_step_push<S, false, true><<<g, b, 0, s>>>(a);
  else k_step_push<S, false, false><<<g, b, 0, s>>>(a);
}

cudaError_t launch_step_push(int storage, const StepArgs &a, int bx, int by, cudaStream_t s) {
  const dim3 g((a.nx + bx - 1) / bx, (a.ny + by - 1) / by, a.nz), b(bx, by, 1);
  LBM_CHECK_TABLE(s, LBM_STEP_RANGES(a, elem_bytes_of(storage)));
  switch (storage) {
    case kF32: push_dispatch<0>(a, g, b, s); break;
    case kF16: push_dispatch<1>(a, g, b, s); break;
    case kBF16: push_dispatch<2>(a, g, b, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_stream(int storage, const StepArgs &a, int form, int bx, int by,
                          cudaStream_t s) {
  const dim3 g((a.nx + bx - 1) / bx, (a.ny + by - 1) / by, a.nz), b(bx, by, 1);
  LBM_CHECK_TABLE(s, LBM_STEP_RANGES(a, elem_bytes_of(storage)));
  switch (storage) {
    case kF32: k_stream<0><<<g, b, 0, s>>>(a, form); break;
    case kF16: k_stream<1><<<g, b, 0, s>>>(a, form); break;
    case kBF16: k_stream<2><<<g, b, 0, s>>>(a, form); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lbm
