// lbm_adjoint.cu - kernels of the discrete adjoint for a single lattice
// (per-node mathematics in adjoint.cuh): reverse step, loss seed, and the
// gradient with respect to the initial velocity.
#include "adjoint.cuh"

namespace lbm {

struct AdjArgs {
  StepArgs g;             // geometry, tau, walls, lid terms, force (fin = f_n)
  const float *rho_n;     // moments form: rho^n, u^n of the forward collision
  const float *u_n;
  const float *lam_in;    // lambda^{n+1}, FP32, pitched like f
  float *lam_out;         // lambda^n
  float *grad_force;      // dense [3][cells] accumulated, or null
  const float *u_target;  // seed only
  double *partials;       // seed only: per-block FP64 loss partials
};

// Extents for the LBM_CHECK tables: an FP32 state or lambda buffer (19
// values per node of the pitched layout), and a dense [3][cells] field.
static inline size_t adj_lambda_bytes(const StepArgs &g) {
  return 19 * (size_t)g.plane * sizeof(float);
}
static inline size_t adj_field_bytes(const StepArgs &g) {
  return 3 * (size_t)g.cells * sizeof(float);
}

// Minimum resident 256-thread blocks per SM for the adjoint step: 3 caps it
// at 80 registers, which measured 7% faster than the unconstrained 102 (more
// resident warps for the three 76 B/node streams), while 4 (64 registers)
// spills.
#ifndef LBM_ADJ_MIN_BLOCKS
#define LBM_ADJ_MIN_BLOCKS 3
#endif

// W: 0 periodic, 1 walls by address selection, 2 walls by the wall-node
// branch (one kernel per form: a runtime choice compiles both into one).
template <int W, bool FORCE, bool GRADF>
__global__ void __launch_bounds__(256, LBM_ADJ_MIN_BLOCKS) k_adjoint_step(const AdjArgs a) {
  const StepArgs &g = a.g;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  adjoint_node<(W != 0), FORCE, GRADF>(static_cast<const float *>(g.fin), a.lam_in, a.lam_out,
                                       g.force, a.grad_force, g.nx, g.ny, g.nz, g.pitch,
                                       g.plane, g.walls, g.lidc, g.omega, g.kf, g.cells, x, y,
                                       z, W == 1);
}

// The reverse step from stored moments (no gather of f^n): 16 + 152 bytes
// per node plus the force terms, and no 19-value state in registers.
template <int W, bool FORCE, bool GRADF>
__global__ void __launch_bounds__(256) k_adjoint_step_mom(const AdjArgs a) {
  const StepArgs &g = a.g;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  adjoint_node_mom<(W != 0), FORCE, GRADF>(a.rho_n, a.u_n, a.lam_in, a.lam_out, g.force,
                                           a.grad_force, g.nx, g.ny, g.nz, g.pitch, g.plane,
                                           g.walls, g.omega, g.kf, g.cells, x, y, z, W == 1);
}

// Seed over all nodes (grid stride), FP64 loss partials per block.
template <bool FORCE>
__global__ void __launch_bounds__(kReduceThreads) k_adjoint_seed(const AdjArgs a) {
  const StepArgs &g = a.g;
  const float *__restrict__ f = static_cast<const float *>(g.fin);
  double acc = 0.0;
  for (uint32_t dc = blockIdx.x * blockDim.x + threadIdx.x; dc < g.cells;
       dc += gridDim.x * blockDim.x) {
    const uint32_t x = dc % g.nx;
    const uint32_t t = dc / g.nx;
    const uint32_t y = t % g.ny, z = t / g.ny;
    acc += seed_node<FORCE>(f, a.u_target, a.lam_out, a.grad_force, g.force, g.nx, g.ny,
                            g.pitch, g.plane, g.cells, x, y, z);
  }
  if (!a.partials) return;
  block_sum_to<kReduceThreads>(acc, a.partials + blockIdx.x);
}

__global__ void __launch_bounds__(256)
    k_adjoint_u0(const StepArgs g, const float *__restrict__ lam0,
                 const float *__restrict__ u0, float *__restrict__ grad) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  u0grad_node(lam0, u0, grad, g.nx, g.ny, g.pitch, g.plane, g.cells, x, y, z);
}

// ---- launchers ------------------------------------------------------------

cudaError_t launch_adjoint_step(const StepArgs &g, const float *lam_in,
                                float *lam_out, float *grad_force, int bx,
                                int by, cudaStream_t s) {
  AdjArgs a;
  a.g = g;
  a.rho_n = a.u_n = nullptr;
  a.lam_in = lam_in;
  a.lam_out = lam_out;
  a.grad_force = grad_force;
  a.u_target = nullptr;
  a.partials = nullptr;
  LBM_CHECK_TABLE(s, chk_r(g.fin, adj_lambda_bytes(g)), chk_r(lam_in, adj_lambda_bytes(g)),
                  chk_w(lam_out, adj_lambda_bytes(g)), chk_rw(grad_force, adj_field_bytes(g)),
                  chk_r(g.force, adj_field_bytes(g)));
  const dim3 grid((g.nx + bx - 1) / bx, (g.ny + by - 1) / by, g.nz), blk(bx, by, 1);
  const int w = g.walls == 0 ? 0 : g.wall_select ? 1 : 2;
  const bool F = g.force != nullptr, G = grad_force != nullptr;
#define LBM_ADJ_CASE(W_, F_, G_)                                 \
  if (w == W_ && F == F_ && G == G_) {                           \
    k_adjoint_step<W_, F_, G_><<<grid, blk, 0, s>>>(a);          \
    return cudaGetLastError();                                   \
  }
  LBM_ADJ_CASE(0, false, false)
  LBM_ADJ_CASE(0, false, true)
  LBM_ADJ_CASE(0, true, false)
  LBM_ADJ_CASE(0, true, true)
  LBM_ADJ_CASE(1, false, false)
  LBM_ADJ_CASE(1, false, true)
  LBM_ADJ_CASE(1, true, false)
  LBM_ADJ_CASE(1, true, true)
  LBM_ADJ_CASE(2, false, false)
  LBM_ADJ_CASE(2, false, true)
  LBM_ADJ_CASE(2, true, false)
  LBM_ADJ_CASE(2, true, true)
#undef LBM_ADJ_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_adjoint_step_mom(const StepArgs &g, const float *rho_n, const float *u_n,
                                    const float *lam_in, float *lam_out, float *grad_force,
                                    int bx, int by, cudaStream_t s) {
  AdjArgs a;
  a.g = g;
  a.rho_n = rho_n;
  a.u_n = u_n;
  a.lam_in = lam_in;
  a.lam_out = lam_out;
  a.grad_force = grad_force;
  a.u_target = nullptr;
  a.partials = nullptr;
  LBM_CHECK_TABLE(s, chk_r(rho_n, adj_field_bytes(g) / 3), chk_r(u_n, adj_field_bytes(g)),
                  chk_r(lam_in, adj_lambda_bytes(g)), chk_w(lam_out, adj_lambda_bytes(g)),
                  chk_rw(grad_force, adj_field_bytes(g)), chk_r(g.force, adj_field_bytes(g)));
  const dim3 grid((g.nx + bx - 1) / bx, (g.ny + by - 1) / by, g.nz), blk(bx, by, 1);
  const int w = g.walls == 0 ? 0 : g.wall_select ? 1 : 2;
  const bool F = g.force != nullptr, G = grad_force != nullptr;
#define LBM_ADJ_CASE(W_, F_, G_)                                 \
  if (w == W_ && F == F_ && G == G_) {                           \
    k_adjoint_step_mom<W_, F_, G_><<<grid, blk, 0, s>>>(a);      \
    return cudaGetLastError();                                   \
  }
  LBM_ADJ_CASE(0, false, false)
  LBM_ADJ_CASE(0, false, true)
  LBM_ADJ_CASE(0, true, false)
  LBM_ADJ_CASE(0, true, true)
  LBM_ADJ_CASE(1, false, false)
  LBM_ADJ_CASE(1, false, true)
  LBM_ADJ_CASE(1, true, false)
  LBM_ADJ_CASE(1, true, true)
  LBM_ADJ_CASE(2, false, false)
  LBM_ADJ_CASE(2, false, true)
  LBM_ADJ_CASE(2, true, false)
  LBM_ADJ_CASE(2, true, true)
#undef LBM_ADJ_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_adjoint_seed(const StepArgs &g, const float *u_target,
                                float *lam_out, float *grad_force,
                                double *partials, cudaStream_t s) {
  AdjArgs a;
  a.g = g;
  a.rho_n = a.u_n = nullptr;
  a.lam_in = nullptr;
  a.lam_out = lam_out;
  a.grad_force = grad_force;
  a.u_target = u_target;
  a.partials = partials;
  const int nb = moments_blocks(g.cells);
  LBM_CHECK_TABLE(s, chk_r(g.fin, adj_lambda_bytes(g)), chk_r(u_target, adj_field_bytes(g)),
                  chk_w(lam_out, adj_lambda_bytes(g)), chk_w(grad_force, adj_field_bytes(g)),
                  chk_r(g.force, adj_field_bytes(g)),
                  chk_w(partials, (size_t)nb * sizeof(double)));
  if (g.force) k_adjoint_seed<true><<<nb, kReduceThreads, 0, s>>>(a);
  else k_adjoint_seed<false><<<nb, kReduceThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_u0(const StepArgs &g, const float *lam0,
                              const float *u0, float *grad, int bx, int by,
                              cudaStream_t s) {
  const dim3 grid((g.nx + bx - 1) / bx, (g.ny + by - 1) / by, g.nz), blk(bx, by, 1);
  LBM_CHECK_TABLE(s, chk_r(lam0, adj_lambda_bytes(g)), chk_r(u0, adj_field_bytes(g)),
                  chk_w(grad, adj_field_bytes(g)));
  k_adjoint_u0<<<grid, blk, 0, s>>>(g, lam0, u0, grad);
  return cudaGetLastError();
}

}  // namespace lbm
