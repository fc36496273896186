// lbm_step.cu - the forward kernels of liblbm:
//   k_step     fused pull stream + boundary rule + collide + store (Alg. 3)
//   k_init     f = f^eq(rho0, u0) (Eq. 5)
//   k_moments  rho, u of a stored state (Eqs. 6-7) + FP64 mass partials
//   k_finalize FP64 sum of the partials
//
// Design for sm_103a: one thread per lattice node, x-dominant blocks
// (coalesced rows, Sec. 4.3.2 and Sec. 6), all 19 loads issued before any
// use (ILP across the f_i, Sec. 4.3), misaligned pulls for e_x != 0 served
// from L1/L2 with no shared-memory or shuffle staging (the DRAM-misaligned
// variant the paper found fastest, Sec. 4.3.2), streaming (evict-first)
// stores so the destination copy does not displace the source lines that
// neighbouring warps still pull.
#include "d3q19.cuh"
#include "internal.h"
#include "onsite.cuh"
#include "stream.cuh"

namespace lbm {

// Launch bounds of the step kernel. By default only the block size is fixed
// and ptxas picks the register budget (40 registers for the periodic FP32
// kernel); defining LBM_STEP_MIN_BLOCKS asks for that many resident 256-thread
// blocks per SM instead (tuning experiments).
#ifdef LBM_STEP_MIN_BLOCKS
#define LBM_STEP_BOUNDS __launch_bounds__(256, LBM_STEP_MIN_BLOCKS)
#else
#define LBM_STEP_BOUNDS __launch_bounds__(256)
#endif

// W: 0 periodic, 1 walls by address selection, 2 walls by the wall-node
// branch (separate kernels: compiling both wall forms into one kernel cost
// ~50 instructions per node even though only one runs), 3 on-site velocity
// walls (plain pull, then the rule of onsite.cuh on wall nodes).
template <int S, int W, bool FORCE, bool MOM>
__global__ void LBM_STEP_BOUNDS k_step(const StepArgs a) {
  using T = typename Store<S>::T;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = a.z0 + blockIdx.z;
  if (x >= a.nx || y >= a.ny) return;
  if constexpr (W == 3) {
    const T *__restrict__ fin = static_cast<const T *>(a.fin);
    T *__restrict__ fout = static_cast<T *>(a.fout);
    const NodeIdx n = node_index(a.nx, a.ny, a.nz, a.pitch, a.walls, x, y, z);
    float d[Q];
    gather<S>(fin, a.plane, n, d);
    const uint32_t dc = ((uint32_t)z * a.ny + y) * a.nx + x;
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    if constexpr (FORCE) {
      Fx = LBM_LDG(a.force + dc);
      Fy = LBM_LDG(a.force + a.cells + dc);
      Fz = LBM_LDG(a.force + 2 * (size_t)a.cells + dc);
    }
    if (on_wall(n)) onsite_apply<S>(fin, a, n, Fx, Fy, Fz, d);
    float rho, ux, uy, uz;
    collide<FORCE>(d, a.omega, a.kf, Fx, Fy, Fz, rho, ux, uy, uz);
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      Store<S>::st(fout + (size_t)i * a.plane + n.c, d[i]);
    });
    if constexpr (MOM) {
      LBM_ST(&a.rho[dc], rho);
      LBM_ST(&a.u[dc], ux);
      LBM_ST(&a.u[a.cells + dc], uy);
      LBM_ST(&a.u[2 * (size_t)a.cells + dc], uz);
    }
  } else {
    step_node<S, (W != 0), FORCE, MOM, false>(
        static_cast<const T *>(a.fin), static_cast<T *>(a.fout), a.nx, a.ny, a.nz, a.pitch,
        a.plane, a.walls, a.lidc, a.omega, a.kf, a.force, a.rho, a.u, a.cells, x, y, z,
        W == 1);
  }
}

template <int S>
__global__ void __launch_bounds__(256)
    k_init(const StepArgs a, const float *__restrict__ rho0,
           const float *__restrict__ u0) {
  using T = typename Store<S>::T;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = a.z0 + blockIdx.z;
  if (x >= a.nx || y >= a.ny) return;
  const uint32_t c = ((uint32_t)z * a.ny + y) * a.pitch + x;
  const uint32_t dc = ((uint32_t)z * a.ny + y) * a.nx + x;
  const float r = rho0 ? LBM_LD(&rho0[dc]) : 1.0f;
  float ux = 0.f, uy = 0.f, uz = 0.f;
  if (u0) {
    ux = LBM_LD(&u0[dc]);
    uy = LBM_LD(&u0[a.cells + dc]);
    uz = LBM_LD(&u0[2 * (size_t)a.cells + dc]);
  }
  float d[Q];
  shifted_equilibrium(r, ux, uy, uz, d);
  T *fout = static_cast<T *>(a.fout);
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    Store<S>::st(fout + (size_t)i * a.plane + c, d[i]);
  });
}

// Grid-stride over all nodes in dense order. Optional FP64 partial sum of
// rho - 1 per block and the non-finite flag.
template <int S, bool FORCE>
__global__ void __launch_bounds__(kReduceThreads)
    k_moments(const StepArgs a, const void *fv, float *__restrict__ rho,
              float *__restrict__ u, double *__restrict__ partials,
              int *__restrict__ err) {
  using T = typename Store<S>::T;
  const T *__restrict__ f = static_cast<const T *>(fv);
  double acc = 0.0;
  bool bad = false;
  const uint32_t plane_nodes = (uint32_t)a.nx * a.ny;
  const uint32_t dc_end = (uint32_t)(a.z0 + a.zn) * plane_nodes;
  for (uint32_t dc = (uint32_t)a.z0 * plane_nodes + blockIdx.x * blockDim.x + threadIdx.x;
       dc < dc_end; dc += gridDim.x * blockDim.x) {
    const uint32_t x = dc % a.nx;
    const uint32_t t = dc / a.nx;
    const uint32_t y = t % a.ny, z = t / a.ny;
    const uint32_t c = (z * a.ny + y) * a.pitch + x;
    float d[Q];
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      d[i] = Store<S>::ld(f + (size_t)i * a.plane + c);
    });
    float dr, jx, jy, jz;
    shifted_moments(d, dr, jx, jy, jz);
    const float r = 1.0f + dr;
    if constexpr (FORCE) {
      jx = fmaf(-0.5f, LBM_LDG(a.force + dc), jx);
      jy = fmaf(-0.5f, LBM_LDG(a.force + a.cells + dc), jy);
      jz = fmaf(-0.5f, LBM_LDG(a.force + 2 * (size_t)a.cells + dc), jz);
    }
    const float rinv = __frcp_rn(r);
    if (rho) LBM_ST(&rho[dc], r);
    if (u) {
      LBM_ST(&u[dc], jx * rinv);
      LBM_ST(&u[a.cells + dc], jy * rinv);
      LBM_ST(&u[2 * (size_t)a.cells + dc], jz * rinv);
    }
    acc += (double)dr;
    bad |= !isfinite(r);
  }
  if (!partials) return;
  // block reduction of acc (warp shuffles, then one warp over the warps)
  __shared__ double red[kReduceThreads / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = acc;
  if (__syncthreads_or(bad) && threadIdx.x == 0) LBM_ATOMIC_OR(err, (int)kErrNonFinite);
  if (wid == 0) {
    acc = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) LBM_ST(&partials[blockIdx.x], acc);
  }
}

__global__ void __launch_bounds__(1024)
    k_finalize(const double *__restrict__ partials, int n, double offset,
               double *__restrict__ out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) acc += LBM_LD(&partials[k]);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (wid == 0) {
    acc = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) LBM_ST(out, offset + acc);
  }
}

// ---- launchers ---------------------------------------------------------------

static dim3 node_grid(const StepArgs &a, int bx, int by) {
  return dim3((a.nx + bx - 1) / bx, (a.ny + by - 1) / by, a.zn);
}

template <int S>
static void step_dispatch(bool moments, const StepArgs &a, dim3 g, dim3 b,
                          cudaStream_t s) {
  const int walls = a.walls == 0 ? 0 : a.onsite ? 3 : a.wall_select ? 1 : 2;
  const bool force = a.force != nullptr;
#define LBM_STEP_CASE(W, F, M)                                  \
  if (walls == W && force == F && moments == M) {               \
    k_step<S, W, F, M><<<g, b, 0, s>>>(a);                      \
    return;                                                     \
  }
  LBM_STEP_CASE(0, false, false)
  LBM_STEP_CASE(0, false, true)
  LBM_STEP_CASE(0, true, false)
  LBM_STEP_CASE(0, true, true)
  LBM_STEP_CASE(1, false, false)
  LBM_STEP_CASE(1, false, true)
  LBM_STEP_CASE(1, true, false)
  LBM_STEP_CASE(1, true, true)
  LBM_STEP_CASE(2, false, false)
  LBM_STEP_CASE(2, false, true)
  LBM_STEP_CASE(2, true, false)
  LBM_STEP_CASE(2, true, true)
  LBM_STEP_CASE(3, false, false)
  LBM_STEP_CASE(3, false, true)
  LBM_STEP_CASE(3, true, false)
  LBM_STEP_CASE(3, true, true)
#undef LBM_STEP_CASE
}

cudaError_t launch_step(int storage, bool moments, const StepArgs &a, int bx,
                        int by, cudaStream_t s) {
  const dim3 g = node_grid(a, bx, by), b(bx, by, 1);
  LBM_CHECK_TABLE(s, LBM_STEP_RANGES(a, elem_bytes_of(storage)));
  switch (storage) {
    case kF32: step_dispatch<0>(moments, a, g, b, s); break;
    case kF16: step_dispatch<1>(moments, a, g, b, s); break;
    case kBF16: step_dispatch<2>(moments, a, g, b, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_init(int storage, const StepArgs &a, const float *rho0,
                        const float *u0, int bx, int by, cudaStream_t s) {
  const dim3 g = node_grid(a, bx, by), b(bx, by, 1);
  LBM_CHECK_TABLE(s, chk_w(a.fout, 19 * (size_t)a.plane * elem_bytes_of(storage)),
                  chk_r(rho0, (size_t)a.cells * sizeof(float)),
                  chk_r(u0, 3 * (size_t)a.cells * sizeof(float)));
  switch (storage) {
    case kF32: k_init<0><<<g, b, 0, s>>>(a, rho0, u0); break;
    case kF16: k_init<1><<<g, b, 0, s>>>(a, rho0, u0); break;
    case kBF16: k_init<2><<<g, b, 0, s>>>(a, rho0, u0); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int S>
static void moments_dispatch(const StepArgs &a, const void *f, float *rho,
                             float *u, double *partials, int *err, int nb,
                             cudaStream_t s) {
  if (a.force)
    k_moments<S, true><<<nb, kReduceThreads, 0, s>>>(a, f, rho, u, partials, err);
  else
    k_moments<S, false><<<nb, kReduceThreads, 0, s>>>(a, f, rho, u, partials, err);
}

cudaError_t launch_moments(int storage, const StepArgs &a, const void *f,
                           float *rho, float *u, const Scratch *scr,
                           cudaStream_t s) {
  const uint32_t nodes = (uint32_t)a.zn * a.nx * a.ny;
  int nb = (int)((nodes + kReduceThreads - 1) / kReduceThreads);
  if (nb > kReduceBlocks) nb = kReduceBlocks;
  if (nb < 1) nb = 1;
  double *partials = scr ? scr->partials : nullptr;
  int *err = scr ? scr->err : nullptr;
  LBM_CHECK_TABLE(s, chk_r(f, 19 * (size_t)a.plane * elem_bytes_of(storage)),
                  chk_w(rho, (size_t)a.cells * sizeof(float)),
                  chk_w(u, 3 * (size_t)a.cells * sizeof(float)),
                  chk_r(a.force, 3 * (size_t)a.cells * sizeof(float)),
                  chk_w(partials, (size_t)nb * sizeof(double)), chk_rw(err, sizeof(int)));
  switch (storage) {
    case kF32: moments_dispatch<0>(a, f, rho, u, partials, err, nb, s); break;
    case kF16: moments_dispatch<1>(a, f, rho, u, partials, err, nb, s); break;
    case kBF16: moments_dispatch<2>(a, f, rho, u, partials, err, nb, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int moments_blocks(uint32_t cells) {
  int nb = (int)((cells + kReduceThreads - 1) / kReduceThreads);
  if (nb > kReduceBlocks) nb = kReduceBlocks;
  return nb < 1 ? 1 : nb;
}

cudaError_t launch_finalize_sum(const Scratch &scr, int nparts, double offset,
                                double *out, cudaStream_t s) {
  LBM_CHECK_TABLE(s, chk_r(scr.partials, (size_t)nparts * sizeof(double)),
                  chk_w(out, sizeof(double)));
  k_finalize<<<1, 1024, 0, s>>>(scr.partials, nparts, offset, out);
  return cudaGetLastError();
}

}  // namespace lbm
