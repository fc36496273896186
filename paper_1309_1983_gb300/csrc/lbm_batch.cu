// lbm_batch.cu - many independent lattices (uneven sizes, own tau and lid)
// advanced together.
//
// Layout: the domains' pitched SoA regions are concatenated in one pair of
// f buffers, each region starting on a 256-byte boundary. Work: the dense
// cell range of every domain is cut into tiles of blockDim.x consecutive
// nodes; a tile table {domain, first node} covers all domains.
//
// k_batch_persistent runs n whole time steps in ONE cooperative launch:
// every block walks the tile table with a grid stride, then all blocks meet
// at a grid barrier before the next step. The barrier spins with a wall-clock
// limit (%globaltimer); when the limit passes it sets an error bit, and every
// block leaves the kernel at its next barrier, so a wrong participant count
// ends the launch with LBM_ETIMEOUT instead of hanging the GPU. Loads of f go
// through L2 only (ld.global.cg): other blocks rewrite the buffers between
// barriers, so the non-coherent read-only path must not be used here.
#include "adjoint.cuh"
#include "d3q19.cuh"
#include "internal.h"
#include "stream.cuh"

#ifdef LBM_CHECK
#include <vector>
#endif

namespace lbm {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Exact q = n / d for n < 2^22 and 1 <= d < 2^20 with M = ceil(2^42 / d).
__device__ __forceinline__ uint32_t magic_div(uint32_t n, uint64_t M) {
  return (uint32_t)(((uint64_t)n * M) >> 42);
}

__device__ __forceinline__ void decode(const BatchDom &D, uint32_t k, int &x, int &y,
                                       int &z) {
  const uint32_t nxy = (uint32_t)D.nx * D.ny;
  const uint32_t zz = magic_div(k, D.m_nxy);
  const uint32_t r = k - zz * nxy;
  const uint32_t yy = magic_div(r, D.m_nx);
  x = (int)(r - yy * D.nx);
  y = (int)yy;
  z = (int)zz;
}

// Grid barrier with a bounded wait. Returns false (and sets the timeout bit)
// if the other blocks did not all arrive within timeout_ns, or if another
// block already gave up.
__device__ bool grid_barrier(const BatchArgs &a) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g0 = LBM_LDV(a.bar_gen);
    __threadfence();
    const unsigned arrived = LBM_ATOMIC_ADD(a.bar_count, 1u) + 1u;
    int good = 1;
    if (arrived == a.expected) {
      LBM_ST(a.bar_count, 0u);  // nobody re-arrives before gen moves
      __threadfence();
      LBM_ATOMIC_ADD(a.bar_gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (LBM_LDV(a.bar_gen) == g0) {
        if (global_ns() - t0 > a.timeout_ns) {
          LBM_ATOMIC_OR(a.err, (int)kErrTimeout);
          good = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    if (LBM_LDV(a.err) & kErrTimeout) good = 0;
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// The domain table is copied into shared memory once per launch (it is read
// for every tile), and the next tile's descriptor is fetched while the
// current tile is processed, so no tile starts with a chain of dependent
// global loads.
template <bool WALLS>
__global__ void __launch_bounds__(256) k_batch_persistent(const BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BatchDom *sdoms = reinterpret_cast<BatchDom *>(smem_raw);
  {
    const uint32_t *src = reinterpret_cast<const uint32_t *>(a.doms);
    uint32_t *dst = reinterpret_cast<uint32_t *>(sdoms);
    const int words = a.ndom * (int)(sizeof(BatchDom) / 4);
    for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = LBM_LD(&src[k]);
    __syncthreads();
  }
  for (int s = 0; s < a.nsteps; ++s) {
    const bool odd = ((a.parity0 + s) & 1) != 0;
    // selects, not a[par] indexing: a runtime index into the parameter
    // array would move the kernel parameters to local memory
    const float *fin = odd ? a.f[1] : a.f[0];
    float *fout = odd ? a.f[0] : a.f[1];
    int t = blockIdx.x;
    int2 tile = t < a.ntiles ? LBM_LD(&a.tiles[t]) : make_int2(0, 0);
    for (; t < a.ntiles; t += gridDim.x) {
      const int tn = t + gridDim.x;
      const int2 next = tn < a.ntiles ? LBM_LD(&a.tiles[tn]) : tile;
      const BatchDom &D = sdoms[tile.x];
      const uint32_t k = (uint32_t)tile.y + threadIdx.x;
      if (k < D.cells) {
        int x, y, z;
        decode(D, k, x, y, z);
        step_node<0, WALLS, false, false, true>(fin + D.foff, fout + D.foff, D.nx, D.ny, D.nz,
                                                D.pitch, D.plane, D.walls, D.lidc, D.omega,
                                                D.kf, nullptr, nullptr, nullptr, D.cells, x,
                                                y, z);
      }
      tile = next;
    }
    if (s + 1 < a.nsteps && !grid_barrier(a)) return;
  }
}

// Copy the domain table into shared memory (once per persistent launch).
__device__ __forceinline__ BatchDom *stage_domains(const BatchArgs &a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BatchDom *sdoms = reinterpret_cast<BatchDom *>(smem_raw);
  const uint32_t *src = reinterpret_cast<const uint32_t *>(a.doms);
  uint32_t *dst = reinterpret_cast<uint32_t *>(sdoms);
  const int words = a.ndom * (int)(sizeof(BatchDom) / 4);
  for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = LBM_LD(&src[k]);
  __syncthreads();
  return sdoms;
}

// A sequence of q.n steps, each from its own input buffer into its own
// output buffer (and, with MOM, writing the collision's rho and u), in one
// persistent launch: the forward segments and the segment recompute of the
// checkpointed adjoint. Tiles, prefetch, L2-only loads and the bounded grid
// barrier as in k_batch_persistent. The step table is a __grid_constant__
// parameter, so indexing it by the step number needs no local copy.
template <bool WALLS, bool MOM>
__global__ void __launch_bounds__(256) k_batch_fwd_seq(const BatchArgs a,
                                                       const __grid_constant__ BatchFwdSeq q) {
  const BatchDom *sdoms = stage_domains(a);
  for (int s = 0; s < q.n; ++s) {
    const float *fin = q.fin[s];
    float *fout = q.fout[s];
    float *rho = MOM ? q.rho[s] : nullptr;
    float *u = MOM ? q.u[s] : nullptr;
    int t = blockIdx.x;
    int2 tile = t < a.ntiles ? LBM_LD(&a.tiles[t]) : make_int2(0, 0);
    for (; t < a.ntiles; t += gridDim.x) {
      const int tn = t + gridDim.x;
      const int2 next = tn < a.ntiles ? LBM_LD(&a.tiles[tn]) : tile;
      const BatchDom &D = sdoms[tile.x];
      const uint32_t k = (uint32_t)tile.y + threadIdx.x;
      if (k < D.cells) {
        int x, y, z;
        decode(D, k, x, y, z);
        step_node<0, WALLS, false, MOM, true, true>(
            fin + D.foff, fout + D.foff, D.nx, D.ny, D.nz, D.pitch, D.plane, D.walls, D.lidc,
            D.omega, D.kf, nullptr, MOM ? rho + D.coff : nullptr,
            MOM ? u + 3 * (size_t)D.coff : nullptr, D.cells, x, y, z);
      }
      tile = next;
    }
    if (s + 1 < q.n && !grid_barrier(a)) return;
  }
}

// q.n reverse steps from stored moments in one persistent launch: step s
// reads lambda from q.lam[s & 1] (through L2: other blocks scattered it
// before the barrier) and writes q.lam[(s & 1) ^ 1]; the force gradient of
// a node is always accumulated by the same thread (tile t stays on block
// t mod gridDim in every step). Four resident blocks per SM (64 registers,
// a few spilled bytes) and the bounce-back scatter chosen per warp by a
// vote: 0.396 ms per step on the 64-cavity batch against 0.433 ms with
// 80 registers and per-node selection (5.51 against 5.04 TB/s of 192 B
// per node).
template <bool GRADF>
__global__ void __launch_bounds__(256, 4) k_batch_adj_seq(const BatchArgs a,
                                                       const __grid_constant__ BatchAdjSeq q) {
  const BatchDom *sdoms = stage_domains(a);
  for (int s = 0; s < q.n; ++s) {
    const float *lam_in = q.lam[s & 1];
    float *lam_out = q.lam[(s & 1) ^ 1];
    const float *rho = q.rho[s];
    const float *u = q.u[s];
    int t = blockIdx.x;
    int2 tile = t < a.ntiles ? LBM_LD(&a.tiles[t]) : make_int2(0, 0);
    for (; t < a.ntiles; t += gridDim.x) {
      const int tn = t + gridDim.x;
      const int2 next = tn < a.ntiles ? LBM_LD(&a.tiles[tn]) : tile;
      const BatchDom &D = sdoms[tile.x];
      const uint32_t k = (uint32_t)tile.y + threadIdx.x;
      if (k < D.cells) {
        int x, y, z;
        decode(D, k, x, y, z);
        adjoint_node_mom<true, false, GRADF, true>(
            rho + D.coff, u + 3 * (size_t)D.coff, lam_in + D.foff, lam_out + D.foff, nullptr,
            GRADF ? q.gF + 3 * (size_t)D.coff : nullptr, D.nx, D.ny, D.nz, D.pitch, D.plane,
            D.walls, D.omega, D.kf, D.cells, x, y, z, false);
      }
      tile = next;
    }
    if (s + 1 < q.n && !grid_barrier(a)) return;
  }
}

// One step over all domains without a grid barrier (one launch per step):
// the comparison path, and what the adjoint recompute uses.
template <bool WALLS>
__global__ void __launch_bounds__(256) k_batch_step(const BatchArgs a, const float *fin,
                                                    float *fout) {
  const int2 tile = LBM_LD(&a.tiles[blockIdx.x]);
  if (!LBM_VALID(&a.doms[tile.x])) return;
  const BatchDom &D = a.doms[tile.x];
  const uint32_t k = (uint32_t)tile.y + threadIdx.x;
  if (k >= D.cells) return;
  int x, y, z;
  decode(D, k, x, y, z);
  step_node<0, WALLS, false, false, false>(fin + D.foff, fout + D.foff, D.nx, D.ny, D.nz,
                                           D.pitch, D.plane, D.walls, D.lidc, D.omega, D.kf,
                                           nullptr, nullptr, nullptr, D.cells, x, y, z);
}

// The same step also writing the collision's rho and u into the dense
// per-domain fields (rho at coff, u at 3 coff of each domain).
template <bool WALLS>
__global__ void __launch_bounds__(256) k_batch_step_mom(const BatchArgs a, const float *fin,
                                                        float *fout, float *rho, float *u) {
  const int2 tile = LBM_LD(&a.tiles[blockIdx.x]);
  if (!LBM_VALID(&a.doms[tile.x])) return;
  const BatchDom &D = a.doms[tile.x];
  const uint32_t k = (uint32_t)tile.y + threadIdx.x;
  if (k >= D.cells) return;
  int x, y, z;
  decode(D, k, x, y, z);
  step_node<0, WALLS, false, true, false>(fin + D.foff, fout + D.foff, D.nx, D.ny, D.nz,
                                          D.pitch, D.plane, D.walls, D.lidc, D.omega, D.kf,
                                          nullptr, rho + D.coff, u + 3 * (size_t)D.coff,
                                          D.cells, x, y, z);
}

// f = w_i (shifted value 0) on every node of every domain.
__global__ void __launch_bounds__(256) k_batch_rest(const BatchArgs a, float *f) {
  const int2 tile = LBM_LD(&a.tiles[blockIdx.x]);
  if (!LBM_VALID(&a.doms[tile.x])) return;
  const BatchDom &D = a.doms[tile.x];
  const uint32_t k = (uint32_t)tile.y + threadIdx.x;
  if (k >= D.cells) return;
  int x, y, z;
  decode(D, k, x, y, z);
  const uint32_t c = ((uint32_t)z * D.ny + y) * D.pitch + x;
  for (int i = 0; i < Q; ++i) LBM_ST(&f[D.foff + (size_t)i * D.plane + c], 0.0f);
}

// rho and u of every node into dense per-domain blocks:
// rho[coff + k], u[3 * coff + comp * cells + k].
__global__ void __launch_bounds__(256) k_batch_moments(const BatchArgs a, const float *f,
                                                       float *rho, float *u) {
  const int2 tile = LBM_LD(&a.tiles[blockIdx.x]);
  if (!LBM_VALID(&a.doms[tile.x])) return;
  const BatchDom &D = a.doms[tile.x];
  const uint32_t k = (uint32_t)tile.y + threadIdx.x;
  if (k >= D.cells) return;
  int x, y, z;
  decode(D, k, x, y, z);
  const uint32_t c = ((uint32_t)z * D.ny + y) * D.pitch + x;
  float d[Q];
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    d[i] = LBM_LDG(f + D.foff + (size_t)i * D.plane + c);
  });
  float dr, jx, jy, jz;
  shifted_moments(d, dr, jx, jy, jz);
  const float r = 1.0f + dr, rinv = __frcp_rn(r);
  if (rho) LBM_ST(&rho[D.coff + k], r);
  if (u) {
    float *ud = u + 3 * (size_t)D.coff;
    LBM_ST(&ud[k], jx * rinv);
    LBM_ST(&ud[D.cells + k], jy * rinv);
    LBM_ST(&ud[2 * (size_t)D.cells + k], jz * rinv);
  }
}

// f = f^eq(1, u0) on every node of every domain (u0 null: rest). u0 holds
// dense per-domain blocks: u0[3 * coff + comp * cells + node].
__global__ void __launch_bounds__(256) k_batch_init_eq(const BatchArgs a, float *f,
                                                       const float *u0) {
  const int2 tile = LBM_LD(&a.tiles[blockIdx.x]);
  if (!LBM_VALID(&a.doms[tile.x])) return;
  const BatchDom &D = a.doms[tile.x];
  const uint32_t k = (uint32_t)tile.y + threadIdx.x;
  if (k >= D.cells) return;
  int x, y, z;
  decode(D, k, x, y, z);
  const uint32_t c = ((uint32_t)z * D.ny + y) * D.pitch + x;
  float ux = 0.f, uy = 0.f, uz = 0.f;
  if (u0) {
    const float *ud = u0 + 3 * (size_t)D.coff;
    ux = LBM_LD(&ud[k]);
    uy = LBM_LD(&ud[D.cells + k]);
    uz = LBM_LD(&ud[2 * (size_t)D.cells + k]);
  }
  float d[Q];
  shifted_equilibrium(1.0f, ux, uy, uz, d);
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    LBM_ST(&f[D.foff + (size_t)i * D.plane + c], d[i]);
  });
}

// ---- batched adjoint (one launch per reverse step over the tile table) ----

// Minimum resident 256-thread blocks per SM of the batched adjoint step (3:
// 80 registers with a few spilled bytes, measured 14% faster than 2 blocks
// at 128 registers without spills).
#ifndef LBM_BATCH_ADJ_MIN_BLOCKS
#define LBM_BATCH_ADJ_MIN_BLOCKS 3
#endif

template <bool GRADF>
__global__ void __launch_bounds__(256, LBM_BATCH_ADJ_MIN_BLOCKS)
    k_batch_adjoint_step(const BatchArgs a, const float *fn, const float *lam_in,
                         float *lam_out, float *gF) {
  const int2 tile = LBM_LD(&a.tiles[blockIdx.x]);
  if (!LBM_VALID(&a.doms[tile.x])) return;
  const BatchDom &D = a.doms[tile.x];
  const uint32_t k = (uint32_t)tile.y + threadIdx.x;
  if (k >= D.cells) return;
  int x, y, z;
  decode(D, k, x, y, z);
  // small domains: wall nodes in most warps, so bounce-back by address
  // selection (measured 5% faster here than the wall-node branch)
  adjoint_node<true, false, GRADF>(fn + D.foff, lam_in + D.foff, lam_out + D.foff, nullptr,
                                   GRADF ? gF + 3 * (size_t)D.coff : nullptr, D.nx, D.ny, D.nz,
                                   D.pitch, D.plane, D.walls, D.lidc, D.omega, D.kf, D.cells,
                                   x, y, z, true);
}

// The batched reverse step from stored moments (no gather of f^n).
template <bool GRADF>
__global__ void __launch_bounds__(256)
    k_batch_adjoint_step_mom(const BatchArgs a, const float *rho, const float *u,
                             const float *lam_in, float *lam_out, float *gF) {
  const int2 tile = LBM_LD(&a.tiles[blockIdx.x]);
  if (!LBM_VALID(&a.doms[tile.x])) return;
  const BatchDom &D = a.doms[tile.x];
  const uint32_t k = (uint32_t)tile.y + threadIdx.x;
  if (k >= D.cells) return;
  int x, y, z;
  decode(D, k, x, y, z);
  adjoint_node_mom<true, false, GRADF>(rho + D.coff, u + 3 * (size_t)D.coff, lam_in + D.foff,
                                       lam_out + D.foff, nullptr,
                                       GRADF ? gF + 3 * (size_t)D.coff : nullptr, D.nx, D.ny,
                                       D.nz, D.pitch, D.plane, D.walls, D.omega, D.kf, D.cells,
                                       x, y, z, true);
}

// Seed per node, FP64 loss partial per tile (block) into partials[tile].
__global__ void __launch_bounds__(256)
    k_batch_adjoint_seed(const BatchArgs a, const float *fT, const float *ut, float *lam,
                         float *gF, double *partials) {
  const int2 tile = LBM_LD(&a.tiles[blockIdx.x]);
  if (!LBM_VALID(&a.doms[tile.x])) return;
  const BatchDom &D = a.doms[tile.x];
  const uint32_t k = (uint32_t)tile.y + threadIdx.x;
  double acc = 0.0;
  if (k < D.cells) {
    int x, y, z;
    decode(D, k, x, y, z);
    acc = seed_node<false>(fT + D.foff, ut + 3 * (size_t)D.coff, lam + D.foff,
                           gF ? gF + 3 * (size_t)D.coff : nullptr, nullptr, D.nx, D.ny,
                           D.pitch, D.plane, D.cells, x, y, z);
  }
  if (partials) block_sum_to<256>(acc, partials + blockIdx.x);
}

__global__ void __launch_bounds__(256)
    k_batch_adjoint_u0(const BatchArgs a, const float *lam0, const float *u0, float *grad) {
  const int2 tile = LBM_LD(&a.tiles[blockIdx.x]);
  if (!LBM_VALID(&a.doms[tile.x])) return;
  const BatchDom &D = a.doms[tile.x];
  const uint32_t k = (uint32_t)tile.y + threadIdx.x;
  if (k >= D.cells) return;
  int x, y, z;
  decode(D, k, x, y, z);
  u0grad_node(lam0 + D.foff, u0 ? u0 + 3 * (size_t)D.coff : nullptr,
              grad + 3 * (size_t)D.coff, D.nx, D.ny, D.pitch, D.plane, D.cells, x, y, z);
}

// ---- launchers ------------------------------------------------------------

const void *batch_persistent_kernel(bool walls) {
  return walls ? (const void *)k_batch_persistent<true>
               : (const void *)k_batch_persistent<false>;
}

size_t batch_persistent_smem(int ndom) { return sizeof(BatchDom) * (size_t)ndom; }

cudaError_t launch_batch_persistent(const BatchArgs &a, int grid, int threads,
                                    cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = batch_persistent_smem(a.ndom);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  LBM_CHECK_TABLE(s, LBM_BATCH_RANGES(a), chk_rw(a.f[0], LBM_BATCH_F(a)),
                  chk_rw(a.f[1], LBM_BATCH_F(a)));
  if (a.walls_any)
    return cudaLaunchKernelEx(&cfg, k_batch_persistent<true>, a);
  return cudaLaunchKernelEx(&cfg, k_batch_persistent<false>, a);
}

const void *batch_fwd_seq_kernel(bool walls, bool moments) {
  if (walls)
    return moments ? (const void *)k_batch_fwd_seq<true, true>
                   : (const void *)k_batch_fwd_seq<true, false>;
  return moments ? (const void *)k_batch_fwd_seq<false, true>
                 : (const void *)k_batch_fwd_seq<false, false>;
}

const void *batch_adj_seq_kernel(bool gradf) {
  return gradf ? (const void *)k_batch_adj_seq<true> : (const void *)k_batch_adj_seq<false>;
}

static cudaLaunchConfig_t coop_config(int grid, int threads, size_t smem, cudaStream_t s,
                                      cudaLaunchAttribute *attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

cudaError_t launch_batch_fwd_seq(const BatchArgs &a, const BatchFwdSeq &q, int grid, int threads,
                                 cudaStream_t s) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = coop_config(grid, threads, batch_persistent_smem(a.ndom), s, attr);
  const bool mom = q.rho[0] != nullptr;
#ifdef LBM_CHECK
  {
    std::vector<CheckRange> r = {LBM_BATCH_RANGES(a)};
    for (int k = 0; k < q.n; ++k) {
      r.push_back(chk_r(q.fin[k], LBM_BATCH_F(a)));
      r.push_back(chk_w(q.fout[k], LBM_BATCH_F(a)));
      if (mom) {
        r.push_back(chk_w(q.rho[k], LBM_BATCH_FIELD(a, 1)));
        r.push_back(chk_w(q.u[k], LBM_BATCH_FIELD(a, 3)));
      }
    }
    const cudaError_t ce = check_table(s, r.data(), (int)r.size());
    if (ce != cudaSuccess) return ce;
  }
#endif
  if (a.walls_any)
    return mom ? cudaLaunchKernelEx(&cfg, k_batch_fwd_seq<true, true>, a, q)
               : cudaLaunchKernelEx(&cfg, k_batch_fwd_seq<true, false>, a, q);
  return mom ? cudaLaunchKernelEx(&cfg, k_batch_fwd_seq<false, true>, a, q)
             : cudaLaunchKernelEx(&cfg, k_batch_fwd_seq<false, false>, a, q);
}

cudaError_t launch_batch_adj_seq(const BatchArgs &a, const BatchAdjSeq &q, int grid, int threads,
                                 cudaStream_t s) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = coop_config(grid, threads, batch_persistent_smem(a.ndom), s, attr);
#ifdef LBM_CHECK
  {
    std::vector<CheckRange> r = {LBM_BATCH_RANGES(a), chk_rw(q.lam[0], LBM_BATCH_F(a)),
                                 chk_rw(q.lam[1], LBM_BATCH_F(a)),
                                 chk_rw(q.gF, LBM_BATCH_FIELD(a, 3))};
    for (int k = 0; k < q.n; ++k) {
      r.push_back(chk_r(q.rho[k], LBM_BATCH_FIELD(a, 1)));
      r.push_back(chk_r(q.u[k], LBM_BATCH_FIELD(a, 3)));
    }
    const cudaError_t ce = check_table(s, r.data(), (int)r.size());
    if (ce != cudaSuccess) return ce;
  }
#endif
  if (q.gF) return cudaLaunchKernelEx(&cfg, k_batch_adj_seq<true>, a, q);
  return cudaLaunchKernelEx(&cfg, k_batch_adj_seq<false>, a, q);
}

cudaError_t launch_batch_step(const BatchArgs &a, const float *fin, float *fout,
                              int threads, cudaStream_t s) {
  LBM_CHECK_TABLE(s, LBM_BATCH_RANGES(a), chk_r(fin, LBM_BATCH_F(a)),
                  chk_w(fout, LBM_BATCH_F(a)));
  if (a.walls_any)
    k_batch_step<true><<<a.ntiles, threads, 0, s>>>(a, fin, fout);
  else
    k_batch_step<false><<<a.ntiles, threads, 0, s>>>(a, fin, fout);
  return cudaGetLastError();
}

cudaError_t launch_batch_step_mom(const BatchArgs &a, const float *fin, float *fout, float *rho,
                                  float *u, int threads, cudaStream_t s) {
  LBM_CHECK_TABLE(s, LBM_BATCH_RANGES(a), chk_r(fin, LBM_BATCH_F(a)), chk_w(fout, LBM_BATCH_F(a)),
                  chk_w(rho, LBM_BATCH_FIELD(a, 1)), chk_w(u, LBM_BATCH_FIELD(a, 3)));
  if (a.walls_any)
    k_batch_step_mom<true><<<a.ntiles, threads, 0, s>>>(a, fin, fout, rho, u);
  else
    k_batch_step_mom<false><<<a.ntiles, threads, 0, s>>>(a, fin, fout, rho, u);
  return cudaGetLastError();
}

cudaError_t launch_batch_adjoint_step_mom(const BatchArgs &a, const float *rho, const float *u,
                                          const float *lam_in, float *lam_out, float *gF,
                                          int threads, cudaStream_t s) {
  LBM_CHECK_TABLE(s, LBM_BATCH_RANGES(a), chk_r(rho, LBM_BATCH_FIELD(a, 1)),
                  chk_r(u, LBM_BATCH_FIELD(a, 3)), chk_r(lam_in, LBM_BATCH_F(a)),
                  chk_w(lam_out, LBM_BATCH_F(a)), chk_rw(gF, LBM_BATCH_FIELD(a, 3)));
  if (gF)
    k_batch_adjoint_step_mom<true><<<a.ntiles, threads, 0, s>>>(a, rho, u, lam_in, lam_out, gF);
  else
    k_batch_adjoint_step_mom<false><<<a.ntiles, threads, 0, s>>>(a, rho, u, lam_in, lam_out,
                                                                 gF);
  return cudaGetLastError();
}

cudaError_t launch_batch_rest(const BatchArgs &a, float *f, int threads, cudaStream_t s) {
  LBM_CHECK_TABLE(s, LBM_BATCH_RANGES(a), chk_w(f, LBM_BATCH_F(a)));
  k_batch_rest<<<a.ntiles, threads, 0, s>>>(a, f);
  return cudaGetLastError();
}

cudaError_t launch_batch_moments(const BatchArgs &a, const float *f, float *rho, float *u,
                                 int threads, cudaStream_t s) {
  LBM_CHECK_TABLE(s, LBM_BATCH_RANGES(a), chk_r(f, LBM_BATCH_F(a)),
                  chk_w(rho, LBM_BATCH_FIELD(a, 1)), chk_w(u, LBM_BATCH_FIELD(a, 3)));
  k_batch_moments<<<a.ntiles, threads, 0, s>>>(a, f, rho, u);
  return cudaGetLastError();
}

cudaError_t launch_batch_init_eq(const BatchArgs &a, float *f, const float *u0, int threads,
                                 cudaStream_t s) {
  LBM_CHECK_TABLE(s, LBM_BATCH_RANGES(a), chk_w(f, LBM_BATCH_F(a)),
                  chk_r(u0, LBM_BATCH_FIELD(a, 3)));
  k_batch_init_eq<<<a.ntiles, threads, 0, s>>>(a, f, u0);
  return cudaGetLastError();
}

cudaError_t launch_batch_adjoint_step(const BatchArgs &a, const float *fn, const float *lam_in,
                                      float *lam_out, float *gF, int threads, cudaStream_t s) {
  LBM_CHECK_TABLE(s, LBM_BATCH_RANGES(a), chk_r(fn, LBM_BATCH_F(a)),
                  chk_r(lam_in, LBM_BATCH_F(a)), chk_w(lam_out, LBM_BATCH_F(a)),
                  chk_rw(gF, LBM_BATCH_FIELD(a, 3)));
  if (gF)
    k_batch_adjoint_step<true><<<a.ntiles, threads, 0, s>>>(a, fn, lam_in, lam_out, gF);
  else
    k_batch_adjoint_step<false><<<a.ntiles, threads, 0, s>>>(a, fn, lam_in, lam_out, gF);
  return cudaGetLastError();
}

cudaError_t launch_batch_adjoint_seed(const BatchArgs &a, const float *fT, const float *ut,
                                      float *lam, float *gF, double *partials, int threads,
                                      cudaStream_t s) {
  LBM_CHECK_TABLE(s, LBM_BATCH_RANGES(a), chk_r(fT, LBM_BATCH_F(a)),
                  chk_r(ut, LBM_BATCH_FIELD(a, 3)), chk_w(lam, LBM_BATCH_F(a)),
                  chk_w(gF, LBM_BATCH_FIELD(a, 3)),
                  chk_w(partials, (size_t)a.ntiles * sizeof(double)));
  k_batch_adjoint_seed<<<a.ntiles, threads, 0, s>>>(a, fT, ut, lam, gF, partials);
  return cudaGetLastError();
}

cudaError_t launch_batch_adjoint_u0(const BatchArgs &a, const float *lam0, const float *u0,
                                    float *grad, int threads, cudaStream_t s) {
  LBM_CHECK_TABLE(s, LBM_BATCH_RANGES(a), chk_r(lam0, LBM_BATCH_F(a)),
                  chk_r(u0, LBM_BATCH_FIELD(a, 3)), chk_w(grad, LBM_BATCH_FIELD(a, 3)));
  k_batch_adjoint_u0<<<a.ntiles, threads, 0, s>>>(a, lam0, u0, grad);
  return cudaGetLastError();
}

}  // namespace lbm
