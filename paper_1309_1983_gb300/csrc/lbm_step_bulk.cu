// lbm_step_bulk.cu - the fused step with the pulled rows staged in shared
// memory by the bulk-copy (TMA) engine.
//
// Why: the one-node-per-thread kernel keeps every pulled value in a register
// from the load until it is used, so the bytes it can have in flight per SM
// are bounded by the register file; with 16-bit storage (2 bytes per 32-bit
// register) that bound is about half of what HBM3e needs to stay busy.
// Bulk copies write shared memory directly, so the in-flight bytes are bounded
// by the shared-memory pipeline instead.
//
// Structure (persistent, warp-specialised): a tile is TX = 128 consecutive
// nodes of TY rows in one z plane. For every direction i and row r, the
// source row (y + r - e_y, z - e_z), periodically wrapped, is copied for
// x in [x0 - H, x0 + TX + H) (H = 16 bytes of halo, clamped to the padded row)
// into one shared-memory row: one cp.async.bulk per (i, r), completing on the
// stage's mbarrier. One producer thread fills STAGES stages ahead; 128
// consumer threads take node x0 + tid of each row, read the 19 values at
// x - e_x from the staged rows, and run the same collision as the other
// kernels. Sources outside the copied span (the periodic wrap at the two row
// ends) and bounce-back replacements on walled faces are read from global
// memory directly. Every mbarrier wait is bounded: on timeout the thread sets
// the error word and the block stops issuing and returns after waiting
// (bounded) for the copies it started.
#include "d3q19.cuh"
#include "internal.h"
#include "stream.cuh"
#include "tma.cuh"

namespace lbm {

namespace bulk {

constexpr int TX = 128;
constexpr int kConsumers = TX;
constexpr int kThreads = TX + 32;  // + one producer warp

struct TileCoord {
  int x0, y0, z;
};

__device__ __forceinline__ TileCoord tile_coord(int t, int nxs, int nys, int TY) {
  TileCoord c;
  const int xs = t % nxs;
  const int r = t / nxs;
  c.x0 = xs * TX;
  c.y0 = (r % nys) * TY;
  c.z = r / nys;
  return c;
}

}  // namespace bulk

struct BulkArgs {
  StepArgs g;
  int *err;
  int nxs, nys, ntiles;
};

template <int S, bool WALLS, bool FORCE, int TY, int STAGES>
__global__ void __launch_bounds__(bulk::kThreads) k_step_bulk(const BulkArgs A) {
  using T = typename Store<S>::T;
  constexpr int EB = (int)sizeof(T);
  constexpr int H = 16 / EB;                  // halo elements (16 bytes)
  constexpr int TXH = bulk::TX + 2 * H;       // staged row length
  constexpr int STAGE_ELEMS = Q * TY * TXH;
  extern __shared__ __align__(128) unsigned char smem[];
  T *rows = reinterpret_cast<T *>(smem);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)STAGES * STAGE_ELEMS * EB);
  uint64_t *empty = full + STAGES;

  const StepArgs &a = A.g;
  const T *__restrict__ fin = static_cast<const T *>(a.fin);
  T *__restrict__ fout = static_cast<T *>(a.fout);
  const int tid = threadIdx.x;
  const bool producer = tid >= bulk::kConsumers;

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tma::mbar_init(&full[s], 1);
      tma::mbar_init(&empty[s], bulk::kConsumers);
    }
    tma::fence_barrier_init();
  }
  __syncthreads();

  const uint32_t row = (uint32_t)a.ny * a.pitch;
  if (producer) {
    if (tid != bulk::kConsumers) return;  // one producer thread
    int k = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < A.ntiles && ok; t += gridDim.x, ++k) {
      const int s = k % STAGES;
      if (k >= STAGES && !tma::mbar_wait(&empty[s], ((k / STAGES) - 1) & 1)) {
        LBM_ATOMIC_OR(A.err, (int)kErrTimeout);
        ok = false;
        break;
      }
      const bulk::TileCoord tc = bulk::tile_coord(t, A.nxs, A.nys, TY);
      const int lo = max(tc.x0 - H, 0);
      const int hi = min(tc.x0 + bulk::TX + H, a.pitch);
      const int nrows = min(TY, a.ny - tc.y0);
      const uint32_t bytes = (uint32_t)(Q * nrows * (hi - lo) * EB);
      tma::mbar_expect_tx(&full[s], bytes);
      T *st = rows + (size_t)s * STAGE_ELEMS;
      const int zm = tc.z == 0 ? a.nz - 1 : tc.z - 1, zp = tc.z == a.nz - 1 ? 0 : tc.z + 1;
      for (int r = 0; r < nrows; ++r) {
        const int y = tc.y0 + r;
        const int ym = y == 0 ? a.ny - 1 : y - 1, yp = y == a.ny - 1 ? 0 : y + 1;
        static_for<0, Q>([&](auto I) {
          constexpr int i = decltype(I)::value;
          constexpr int ey = kEy[i], ez = kEz[i];
          const int sy = ey == 1 ? ym : (ey == -1 ? yp : y);
          const int sz = ez == 1 ? zm : (ez == -1 ? zp : tc.z);
          const T *src = fin + (size_t)i * a.plane + (uint32_t)sz * row + (uint32_t)sy * a.pitch + lo;
          T *dst = st + ((size_t)i * TY + r) * TXH + (lo - (tc.x0 - H));
          // a refused copy (check build) leaves the stage incomplete: the
          // consumers' bounded wait then reports kErrTimeout
          if (LBM_CHK(src, (uint32_t)((hi - lo) * EB), 16u, kChkRead))
            tma::bulk_copy(dst, src, (uint32_t)((hi - lo) * EB), &full[s]);
        });
      }
    }
    // drain: wait (bounded) for every stage this block armed, so no copy is
    // still writing shared memory when the block exits
    const int last = k;
    for (int j = max(0, last - STAGES); j < last; ++j)
      tma::mbar_wait(&full[j % STAGES], (j / STAGES) & 1);
    return;
  }

  // consumers
  int k = 0;
  for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x, ++k) {
    const int s = k % STAGES;
    if (!tma::mbar_wait(&full[s], (k / STAGES) & 1)) {
      LBM_ATOMIC_OR(A.err, (int)kErrTimeout);
      return;
    }
    const bulk::TileCoord tc = bulk::tile_coord(t, A.nxs, A.nys, TY);
    const T *st = rows + (size_t)s * STAGE_ELEMS;
    const int x = tc.x0 + tid;
    for (int r = 0; r < TY; ++r) {
      const int y = tc.y0 + r;
      if (x >= a.nx || y >= a.ny) continue;
      const NodeIdx n = node_index(a.nx, a.ny, a.nz, a.pitch, a.walls, x, y, tc.z);
      float d[Q];
      static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int ex = kEx[i];
        const int sx = x - ex;
        if (ex != 0 && (sx < 0 || sx >= a.nx))
          d[i] = Store<S>::ld(fin + (size_t)i * a.plane + source_of<i>(n));  // wrap
        else
          d[i] = Store<S>::ld_smem(st + ((size_t)i * TY + r) * TXH + (tid + H - ex));
      });
      if constexpr (WALLS) {
        if (on_wall(n)) {
          static_for<1, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            if (bounces<i>(n)) {
              float v = Store<S>::ld(fin + (size_t)kOpp_v<i> * a.plane + n.c);
              if constexpr (kEz[i] == -1) v += n.z1 ? a.lidc[i] : 0.0f;
              d[i] = v;
            }
          });
        }
      }
      const uint32_t dc = ((uint32_t)tc.z * a.ny + y) * a.nx + x;
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
        Store<S>::st(fout + (size_t)i * a.plane + n.c, d[i]);
      });
    }
    tma::mbar_arrive(&empty[s]);
  }
}

template <int S, int TY, int STAGES>
static size_t bulk_smem_bytes() {
  using T = typename Store<S>::T;
  constexpr int H = 16 / (int)sizeof(T);
  return (size_t)STAGES * Q * TY * (bulk::TX + 2 * H) * sizeof(T) + 2 * STAGES * sizeof(uint64_t);
}

template <int S, int TY, int STAGES>
static cudaError_t bulk_launch(const StepArgs &g, int *err, int sms, cudaStream_t s) {
  BulkArgs A;
  A.g = g;
  A.err = err;
  A.nxs = (g.nx + bulk::TX - 1) / bulk::TX;
  A.nys = (g.ny + TY - 1) / TY;
  A.ntiles = A.nxs * A.nys * g.nz;
  const size_t smem = bulk_smem_bytes<S, TY, STAGES>();
  const bool walls = g.walls != 0, force = g.force != nullptr;
  const void *fn = walls ? (force ? (const void *)k_step_bulk<S, true, true, TY, STAGES>
                                  : (const void *)k_step_bulk<S, true, false, TY, STAGES>)
                         : (force ? (const void *)k_step_bulk<S, false, true, TY, STAGES>
                                  : (const void *)k_step_bulk<S, false, false, TY, STAGES>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, bulk::kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int grid = per_sm * sms;
  if (grid > A.ntiles) grid = A.ntiles;
  void *args[] = {&A};
  return cudaLaunchKernel(fn, dim3(grid), dim3(bulk::kThreads), args, smem, s);
}

cudaError_t launch_step_bulk(int storage, const StepArgs &a, int *err, int variant, int sms,
                             cudaStream_t s) {
  LBM_CHECK_TABLE(s, LBM_STEP_RANGES(a, elem_bytes_of(storage)), chk_rw(err, sizeof(int)));
  switch (storage) {
    case kF32:
      return variant == 1 ? bulk_launch<0, 1, 6>(a, err, sms, s) : bulk_launch<0, 2, 3>(a, err, sms, s);
    case kF16:
      return variant == 1 ? bulk_launch<1, 1, 8>(a, err, sms, s) : bulk_launch<1, 2, 4>(a, err, sms, s);
    case kBF16:
      return variant == 1 ? bulk_launch<2, 1, 8>(a, err, sms, s) : bulk_launch<2, 2, 4>(a, err, sms, s);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace lbm
