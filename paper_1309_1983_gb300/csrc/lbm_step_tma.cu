// lbm_step_tma.cu - the fused step (Alg. 3) for 16-bit storage with every
// pulled value staged in shared memory by tensor copies (TMA); a measured
// alternative to the two-node kernel, selected with LBM_KERNEL_TMA.
//
// The idea: the two-node kernel (lbm_step_x2.cu) keeps each pulled value in
// a register from its load until its use, so the bytes a thread has in
// flight are bounded by its registers: with 16-bit values 76 bytes per
// thread, about 70 KB per SM at 64 registers, against about 110 KB for the
// FP32 kernel, and ncu shows the 16-bit kernel keeping DRAM 77% busy where
// the FP32 one reaches 85%. Tensor copies write shared memory directly: the
// bytes in flight are bounded by the shared memory given to the pipeline
// (up to about 170 KB per SM here) and cost no registers, and the consumers
// read the staged values with 32-bit shared loads at constant offsets.
//
// Measured on GB300 (384^3, FP16): 69.8 GLUPS periodic and 63.3 GLUPS in
// the cavity, against 83.2 and 81.7 for the two-node kernel. ncu at 256^3:
// the 8-value x halos of neighbouring tiles are fetched from DRAM a second
// time (47.5 read bytes per node against 38), DRAM is 52% busy (cavity
// 41%), and the consumer warps wait on the stage barriers (long-scoreboard
// stalls) and, in the warps on a lattice face, on their global loads. The
// variants tried (the tile seams read from global memory instead of halos,
// the face values written into the stage by the producer warp, face loads
// issued before the stage wait, a 64-register cap with 6 blocks per SM, 2
// or 4 stages, L2 promotion of 128 or 256 bytes, 16-value halos) were all
// slower or no faster; the
// two-node kernel stays the default. (A two-node kernel taking two pairs
// per thread in two rows, loads of both issued first, 152 bytes in flight a
// thread, measured no faster either: 82.1 against 83.3 GLUPS.)
//
// Tiles: 64 x-consecutive nodes (32 pairs) of TY rows in one z plane, or
// 128 nodes of 2 rows. For each direction i one tensor copy brings the
// source rows (y - e_y, z - e_z) of the tile: x from x0 over TX values
// (e_x = 0), from x0 over TX + 8 values (e_x = -1) or from x0 - 8 over
// TX + 8 values (e_x = +1; a copy's first x must be a multiple of 8
// values, 16 bytes). The copy engine fills positions outside the lattice
// with zeros. On a periodic z axis the source plane is wrapped (one plane
// per tile); x and y sources are not: the nodes whose source lies outside
// the lattice along x or y, or along a walled z, take that value from
// global memory instead -- the periodic wrap, or the halfway bounce-back
// with the moving-lid term -- in the warps that hold such a node only (a
// tile touching an x face, a row on a y face, a plane on a walled z face).
//
// Roles: one producer thread per block issues a tile's 19 copies onto the
// tile's pipeline stage; the consumer warps, each holding 32 pairs of one
// row of the tile (lane p the nodes x0 + 2p and x0 + 2p + 1), wait for the
// stage, read their 38 values, free the stage, complete the pulls at the
// lattice faces, collide, and store one aligned two-value word per
// direction. The arithmetic is that of the two-node kernel (same collision,
// same conversions), so both produce the same values. Persistent blocks
// walk the tiles in x, y, z order with a stride of the grid size. Every
// wait is bounded (tma.cuh): on timeout the thread sets kErrTimeout in the
// error word and stops; the producer then waits (bounded) for the copies it
// started before the block exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <string.h>

#include "d3q19.cuh"
#include "internal.h"
#include "pack.cuh"
#include "step_tma.h"
#include "stream.cuh"
#include "tma.cuh"

namespace lbm {

namespace tile {

constexpr int kHalo = 8;  // extra x values of the e_x != 0 copies (16 bytes)

// A tile: TX x-consecutive nodes (TX / 2 pairs, TX / 64 warps per row) of TY
// rows. Staged rows: TX values (e_x = 0) or TX + 8 values (e_x != 0).
template <int TX, int TY>
struct Geom {
  static constexpr int kRowA = TX * 2;
  static constexpr int kRowB = (TX + kHalo) * 2;
  static constexpr int kWarpsPerRow = TX / 64;
  static constexpr int kConsumerWarps = TY * kWarpsPerRow;
  static constexpr int kThreads = 32 * (kConsumerWarps + 1);  // + the producer warp
  static __host__ __device__ constexpr int box_bytes(int i) {
    return kEx[i] == 0 ? TY * kRowA : TY * kRowB;
  }
  // boxes start on 128-byte boundaries of the stage
  static __host__ __device__ constexpr int box_offset(int i) {
    int o = 0;
    for (int j = 0; j < i; ++j) o += (box_bytes(j) + 127) / 128 * 128;
    return o;
  }
  static __host__ __device__ constexpr int stage_bytes() { return box_offset(Q); }
  // bytes the 19 copies of one stage complete on its barrier
  static __host__ __device__ constexpr uint32_t stage_tx() {
    uint32_t b = 0;
    for (int j = 0; j < Q; ++j) b += (uint32_t)box_bytes(j);
    return b;
  }
  // stages, their full and empty barriers, and room to align the base to 128
  static constexpr size_t smem_bytes(int stages) {
    return (size_t)stages * stage_bytes() + 2 * stages * sizeof(uint64_t) + 128;
  }
};

// Position of a block's current tile: tile t = xt + nxt (yt + nyt (z - z0)),
// advanced by the grid size without divisions (the host splits the grid
// size the same way: gx + nxt (gy + nyt gz), gx < nxt, gy < nyt).
struct Walk {
  int xt, yt, z;
  __device__ __forceinline__ void start(int t, int nxt, int nyt, int z0) {
    const int r = t / nxt;
    xt = t - r * nxt;
    yt = r % nyt;
    z = z0 + r / nyt;
  }
  __device__ __forceinline__ void next(int gx, int gy, int gz, int nxt, int nyt) {
    xt += gx;
    int c = xt >= nxt;
    xt -= c ? nxt : 0;
    yt += gy + c;
    c = yt >= nyt;
    yt -= c ? nyt : 0;
    z += gz + c;
  }
};

// True when the source x - e_i of node (x, y, z) lies outside the lattice
// along x or y, or along z when z is walled: the staged value is the copy
// engine's zero fill and the node takes the value from global memory.
template <int i>
__device__ __forceinline__ bool outside(int nx, int ny, int nz, bool zwall, int x, int y, int z) {
  bool o = false;
  if constexpr (kEx[i] == 1) o |= x == 0;
  if constexpr (kEx[i] == -1) o |= x == nx - 1;
  if constexpr (kEy[i] == 1) o |= y == 0;
  if constexpr (kEy[i] == -1) o |= y == ny - 1;
  if constexpr (kEz[i] == 1) o |= zwall && z == 0;
  if constexpr (kEz[i] == -1) o |= zwall && z == nz - 1;
  return o;
}

// The pulled value of direction i at a node whose source lies outside the
// lattice: halfway bounce-back f_ibar(x) (+ the moving-lid term for sources
// on the plane z = nz) across a walled axis, else the periodically wrapped
// source f_i(x - e_i).
template <int S, int i>
__device__ __forceinline__ float edge_pull(const typename Store<S>::T *__restrict__ fin,
                                           uint32_t plane, const NodeIdx &n,
                                           const float (&lidc)[Q]) {
  if (bounces<i>(n)) {
    float v = Store<S>::ld(fin + (size_t)kOpp_v<i> * plane + n.c);
    if constexpr (kEz[i] == -1) v += n.z1 ? lidc[i] : 0.0f;
    return v;
  }
  return Store<S>::ld(fin + (size_t)i * plane + source_of<i>(n));
}

// The staged values of row r, pair pp of the tile: nodes x0 + 2pp and
// x0 + 2pp + 1.
template <int S, class G>
__device__ __forceinline__ void pull_staged(const unsigned char *st, int r, int pp,
                                            float (&d0)[Q], float (&d1)[Q]) {
  const uint32_t *ra = reinterpret_cast<const uint32_t *>(st + r * G::kRowA) + pp;
  const uint32_t *rb = reinterpret_cast<const uint32_t *>(st + r * G::kRowB) + pp;
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int off = G::box_offset(i) / 4;  // in 32-bit words
    if constexpr (kEx[i] == 0) {
      const float2 v = Pack16<S>::unpack(ra[off]);
      d0[i] = v.x;
      d1[i] = v.y;
    } else {
      // e_x = +1 (copy from x0 - 8): sources x0 + 2pp - 1, x0 + 2pp are
      // values 2pp + 7, 2pp + 8 of the row, the high half of word pp + 3
      // and the low half of word pp + 4; e_x = -1 (copy from x0): values
      // 2pp + 1, 2pp + 2, words pp and pp + 1.
      constexpr int w = off + (kEx[i] == 1 ? 3 : 0);
      const float2 v = Pack16<S>::unpack(__byte_perm(rb[w], rb[w + 1], 0x5432));
      d0[i] = v.x;
      d1[i] = v.y;
    }
  });
}

}  // namespace tile

struct TmaArgs {
  CUtensorMap map_a;  // boxes of TX x TY values (directions with e_x = 0)
  CUtensorMap map_b;  // boxes of (TX + 8) x TY values (e_x != 0)
  StepArgs g;
  int *err;
  int nxt, nyt, ntiles;  // tiles along x, along y, in all
  int gx, gy, gz;        // the grid size as a tile step (Walk::next)
};

#ifdef LBM_CHECK
// Check build: the values a copy reads (the part of its box inside the
// lattice) must lie in the launch's input buffer; a refused copy is not
// issued, and the consumers' bounded wait then reports kErrTimeout.
template <int i>
__device__ bool box_permitted(const StepArgs &a, int xs, int bw, int ys, int ty, int zs) {
  const int xa = max(xs, 0), xb = min(xs + bw, a.nx) - 1;
  const int ya = max(ys, 0), yb = min(ys + ty, a.ny) - 1;
  if (xa > xb || ya > yb || zs < 0 || zs >= a.nz) return true;  // nothing is read
  const uint16_t *f = static_cast<const uint16_t *>(a.fin) + (size_t)i * a.plane +
                      (size_t)zs * a.ny * a.pitch;
  return LBM_CHK(f + (size_t)ya * a.pitch + xa, 2u, 2u, kChkRead) &&
         LBM_CHK(f + (size_t)yb * a.pitch + xb, 2u, 2u, kChkRead);
}
#endif

// Tile (TX x TY nodes) of one block's walk, for both roles.
template <int TX, int TY>
__device__ __forceinline__ void tile_origin(const tile::Walk &w, int &x0, int &y0) {
  x0 = w.xt * TX;
  y0 = w.yt * TY;
}

template <class G, int TX, int TY, int STAGES, bool WALLS>
__device__ __forceinline__ void tma_produce(const TmaArgs &A, uint32_t sbase, uint64_t *full,
                                            uint64_t *empty) {
  const StepArgs &a = A.g;
  const bool zwall = WALLS && (a.walls & LBM_WALL_Z) != 0;
  tma::prefetch_map(&A.map_a);
  tma::prefetch_map(&A.map_b);
  tile::Walk w;
  w.start(blockIdx.x, A.nxt, A.nyt, a.z0);
  int k = 0;
  for (int t = blockIdx.x; t < A.ntiles;
       t += gridDim.x, ++k, w.next(A.gx, A.gy, A.gz, A.nxt, A.nyt)) {
    const int s = k % STAGES;
    if (k >= STAGES && !tma::mbar_wait(&empty[s], ((k / STAGES) - 1) & 1)) {
      LBM_ATOMIC_OR(A.err, (int)kErrTimeout);
      break;
    }
    int x0, y0;
    tile_origin<TX, TY>(w, x0, y0);
    tma::mbar_expect_tx(&full[s], G::stage_tx());
    const uint32_t st = sbase + (uint32_t)s * G::stage_bytes();
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      constexpr int ex = kEx[i], ey = kEy[i], ez = kEz[i];
      constexpr uint32_t off = (uint32_t)G::box_offset(i);
      int zs = w.z - ez;
      if (!zwall) zs = zs < 0 ? zs + a.nz : (zs >= a.nz ? zs - a.nz : zs);
      const int xs = ex == 1 ? x0 - tile::kHalo : x0;
      const int ys = y0 - ey;
#ifdef LBM_CHECK
      if (!box_permitted<i>(a, xs, ex == 0 ? TX : TX + tile::kHalo, ys, TY, zs)) return;
#endif
      tma::tensor_load_4d(st + off, ex == 0 ? &A.map_a : &A.map_b, xs, ys, zs, i, &full[s]);
    });
  }
  // wait (bounded) for every stage this thread armed, so that no copy still
  // writes shared memory when the block exits
  for (int j = k - STAGES < 0 ? 0 : k - STAGES; j < k; ++j)
    tma::mbar_wait(&full[j % STAGES], (j / STAGES) & 1);
}

template <int S, class G, int TX, int TY, int STAGES, bool WALLS, bool FORCE, bool MOM>
__device__ __forceinline__ void tma_consume(const TmaArgs &A, const unsigned char *sgen,
                                            uint64_t *full, uint64_t *empty, int warp, int lane) {
  using T = typename Store<S>::T;
  const StepArgs &a = A.g;
  const T *__restrict__ fin = static_cast<const T *>(a.fin);
  T *__restrict__ fout = static_cast<T *>(a.fout);
  const bool zwall = WALLS && (a.walls & LBM_WALL_Z) != 0;
  const uint32_t row = (uint32_t)a.ny * a.pitch;
  const int r = warp / G::kWarpsPerRow;                   // the warp's row of the tile
  const int pp = (warp % G::kWarpsPerRow) * 32 + lane;  // the thread's pair in the row
  tile::Walk w;
  w.start(blockIdx.x, A.nxt, A.nyt, a.z0);
  int k = 0;
  for (int t = blockIdx.x; t < A.ntiles;
       t += gridDim.x, ++k, w.next(A.gx, A.gy, A.gz, A.nxt, A.nyt)) {
    const int s = k % STAGES;
    if (!tma::mbar_wait(&full[s], (k / STAGES) & 1)) {
      LBM_ATOMIC_OR(A.err, (int)kErrTimeout);
      return;
    }
    float d0[Q], d1[Q];
    tile::pull_staged<S, G>(sgen + s * G::stage_bytes(), r, pp, d0, d1);
    // the warp's reads of the stage are ordered before lane 0's release
    // arrival, after which the producer may refill it
    __syncwarp();
    if (lane == 0) tma::mbar_arrive(&empty[s]);

    int tx0, ty0;
    tile_origin<TX, TY>(w, tx0, ty0);
    const int x0 = tx0 + 2 * pp, y = ty0 + r, z = w.z;
    if (x0 >= a.nx || y >= a.ny) continue;
    const bool has1 = x0 + 1 < a.nx;
    // the padding node of an odd row completes its pulls as node x0 (in
    // bounds; its result lands in the row padding, unused)
    const int x1 = has1 ? x0 + 1 : x0;
    // warp-uniform: the tile's x faces and plane, the warp's row
    if (tx0 == 0 || tx0 + TX >= a.nx || y == 0 || y == a.ny - 1 ||
        (zwall && (z == 0 || z == a.nz - 1))) {
      const uint32_t walls = WALLS ? a.walls : 0u;
      const NodeIdx n0 = node_index(a.nx, a.ny, a.nz, a.pitch, walls, x0, y, z);
      const NodeIdx n1 = node_index(a.nx, a.ny, a.nz, a.pitch, walls, x1, y, z);
      static_for<1, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if (tile::outside<i>(a.nx, a.ny, a.nz, zwall, x0, y, z))
          d0[i] = tile::edge_pull<S, i>(fin, a.plane, n0, a.lidc);
        if (tile::outside<i>(a.nx, a.ny, a.nz, zwall, x1, y, z))
          d1[i] = tile::edge_pull<S, i>(fin, a.plane, n1, a.lidc);
      });
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
    float r0, u0x, u0y, u0z, r1, u1x, u1y, u1z;
    collide<FORCE>(d0, a.omega, a.kf, F0x, F0y, F0z, r0, u0x, u0y, u0z);
    collide<FORCE>(d1, a.omega, a.kf, F1x, F1y, F1z, r1, u1x, u1y, u1z);
    const uint32_t c = (uint32_t)z * row + (uint32_t)y * a.pitch + (uint32_t)x0;
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      Pack16<S>::store(fout + (size_t)i * a.plane + c, d0[i], d1[i]);
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
}

template <int S, int TX, int TY, int STAGES, bool WALLS, bool FORCE, bool MOM>
__global__ void __launch_bounds__(tile::Geom<TX, TY>::kThreads)
    k_step_tma(const __grid_constant__ TmaArgs A) {
  using G = tile::Geom<TX, TY>;
  extern __shared__ unsigned char smem_raw[];
  // stage base aligned to 128 bytes (the boxes' alignment)
  const uint32_t raw = tma::smem_addr(smem_raw);
  const uint32_t sbase = (raw + 127u) & ~127u;
  unsigned char *sgen = smem_raw + (sbase - raw);
  uint64_t *full = reinterpret_cast<uint64_t *>(sgen + STAGES * G::stage_bytes());
  uint64_t *empty = full + STAGES;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tma::mbar_init(&full[s], 1);
      tma::mbar_init(&empty[s], G::kConsumerWarps);  // one arrival per consumer warp
    }
    tma::fence_barrier_init();
  }
  __syncthreads();
  if (warp == G::kConsumerWarps) {
    if (lane == 0) tma_produce<G, TX, TY, STAGES, WALLS>(A, sbase, full, empty);
    return;
  }
  tma_consume<S, G, TX, TY, STAGES, WALLS, FORCE, MOM>(A, sgen, full, empty, warp, lane);
}

// ---- host side ----------------------------------------------------------------

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime (no
// link against the driver library).
EncodeTiled encode_tiled() {
  static const EncodeTiled fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (EncodeTiled) nullptr;
    }
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// no L2 promotion: 128- and 256-byte promotion measured 1-13% slower
constexpr CUtensorMapL2promotion kPromotion = CU_TENSOR_MAP_L2_PROMOTION_NONE;

// The 19 planes of a 16-bit f buffer as a 4-D tensor (x, y, z, i), boxes of
// bx x ty x 1 x 1 values.
cudaError_t encode_map(CUtensorMap *m, const StepArgs &a, int bx, int ty) {
  const EncodeTiled enc = encode_tiled();
  if (enc == nullptr) return cudaErrorNotSupported;
  const cuuint64_t dims[4] = {(cuuint64_t)a.nx, (cuuint64_t)a.ny, (cuuint64_t)a.nz,
                              (cuuint64_t)Q};
  const cuuint64_t strides[3] = {(cuuint64_t)a.pitch * 2, (cuuint64_t)a.pitch * a.ny * 2,
                                 (cuuint64_t)a.plane * 2};
  const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)ty, 1u, 1u};
  const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, const_cast<void *>(a.fin), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, kPromotion, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int S, int TX, int TY, int STAGES, bool WALLS, bool FORCE, bool MOM>
cudaError_t tma_launch(TmaArgs &A, int sms, cudaStream_t s) {
  using G = tile::Geom<TX, TY>;
  const void *fn = (const void *)k_step_tma<S, TX, TY, STAGES, WALLS, FORCE, MOM>;
  constexpr size_t smem = G::smem_bytes(STAGES);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, G::kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long want = (long long)per_sm * sms;
  const int grid = (int)(want < A.ntiles ? want : A.ntiles);
  A.gx = grid % A.nxt;
  A.gy = (grid / A.nxt) % A.nyt;
  A.gz = grid / (A.nxt * A.nyt);
  k_step_tma<S, TX, TY, STAGES, WALLS, FORCE, MOM><<<grid, G::kThreads, smem, s>>>(A);
  return cudaGetLastError();
}

template <int S, int TX, int TY, int STAGES>
cudaError_t tma_dispatch(bool mom, TmaArgs &A, int sms, cudaStream_t s) {
  const bool walls = A.g.walls != 0, force = A.g.force != nullptr;
#define LBM_TMA_CASE(W, F, M)                 \
  if (walls == W && force == F && mom == M) \
    return tma_launch<S, TX, TY, STAGES, W, F, M>(A, sms, s);
  LBM_TMA_CASE(false, false, false)
  LBM_TMA_CASE(false, false, true)
  LBM_TMA_CASE(false, true, false)
  LBM_TMA_CASE(false, true, true)
  LBM_TMA_CASE(true, false, false)
  LBM_TMA_CASE(true, false, true)
  LBM_TMA_CASE(true, true, false)
  LBM_TMA_CASE(true, true, true)
#undef LBM_TMA_CASE
  return cudaErrorInvalidValue;
}

// Tile shapes (nodes along x, rows) by the `by` of the launch: 1 -> 128 x 2,
// 8 -> 64 x 8, else (the default pair block's 2 included) 64 x 4, the
// fastest measured; three pipeline stages each.
struct Shape {
  int tx, ty;
};
Shape tma_shape(int by) {
  return by == 1 ? Shape{128, 2} : by == 8 ? Shape{64, 8} : Shape{64, 4};
}

template <int S>
cudaError_t tma_rows(const Shape &sh, bool mom, TmaArgs &A, int sms, cudaStream_t s) {
  if (sh.tx == 128) return tma_dispatch<S, 128, 2, 3>(mom, A, sms, s);
  if (sh.ty == 8) return tma_dispatch<S, 64, 8, 3>(mom, A, sms, s);
  return tma_dispatch<S, 64, 4, 3>(mom, A, sms, s);
}

}  // namespace

cudaError_t launch_step_tma(int storage, bool moments, const StepArgs &a, int *err, int by,
                            int sms, cudaStream_t s) {
  if ((storage != kF16 && storage != kBF16) || a.onsite) return cudaErrorInvalidValue;
  const Shape sh = tma_shape(by);
  TmaArgs A;
  memset(&A, 0, sizeof(A));
  A.g = a;
  A.err = err;
  A.nxt = (a.nx + sh.tx - 1) / sh.tx;
  A.nyt = (a.ny + sh.ty - 1) / sh.ty;
  A.ntiles = A.nxt * A.nyt * a.zn;
  if (A.ntiles == 0) return cudaSuccess;
  cudaError_t e = encode_map(&A.map_a, a, sh.tx, sh.ty);
  if (e == cudaSuccess) e = encode_map(&A.map_b, a, sh.tx + tile::kHalo, sh.ty);
  if (e != cudaSuccess) return e;
  LBM_CHECK_TABLE(s, LBM_STEP_RANGES(a, 2), chk_rw(err, sizeof(int)));
  return storage == kF16 ? tma_rows<1>(sh, moments, A, sms, s)
                         : tma_rows<2>(sh, moments, A, sms, s);
}

}  // namespace lbm
