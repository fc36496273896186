// lbm_batch_capi.cu - extern "C" entry points of the batched path
// (lbm_batch_*): domain table and tiles, buffer binding, the persistent
// cooperative launch captured in a CUDA graph, and host exchange.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "d3q19.cuh"
#include "internal.h"
#include "tune.h"

using lbm::BatchArgs;
using lbm::BatchDom;

struct lbm_batch {
  int ndom = 0;
  uint32_t flags = 0;
  std::vector<BatchDom> doms;
  std::vector<int2> tiles;
  size_t f_elems = 0;  // FP32 elements per f buffer
  size_t cells = 0;    // total nodes
  BatchDom *d_doms = nullptr;
  int2 *d_tiles = nullptr;
  double *d_partials = nullptr;  // one FP64 partial per tile (adjoint loss)
  double *d_loss_sum = nullptr;
  unsigned *d_bar = nullptr;  // [0] count, [1] generation
  int *d_err = nullptr;
  bool tiles_dirty = true;
  float *f[2] = {nullptr, nullptr};
  int cur = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t capture = nullptr;
  bool bound = false;
  int device = -1;
  int threads = 256;
  int blocks_per_sm = 0;  // 0: as many as fit
  double timeout_s = 1.0;
  int inject_extra = 0;
  bool use_graph = true;
  bool graph_ok = true;
  std::map<std::tuple<int, int, int, int, unsigned, unsigned long long>, cudaGraphExec_t>
      graphs;
  // graphs of the step-sequence launches (lbm_batch_run, lbm_batch_adjoint_run),
  // keyed by kind, grid, expected blocks, timeout and a hash of the step table
  std::map<std::tuple<int, int, int, unsigned, unsigned long long, unsigned long long>,
           cudaGraphExec_t>
      seq_graphs;
};

namespace {

int bfail(int code, const char *what) { return lbm::set_error(code, what); }

int bcuda(cudaError_t e, const char *where) { return lbm::set_cuda_error(e, where); }

#define BCUDA(call, where)                               \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return bcuda(e_, where);      \
  } while (0)

uint64_t magic42(uint32_t d) { return ((1ull << 42) + d - 1) / d; }

void build_tiles(lbm_batch *b) {
  b->tiles.clear();
  for (int k = 0; k < b->ndom; ++k)
    for (uint32_t c0 = 0; c0 < b->doms[k].cells; c0 += (uint32_t)b->threads)
      b->tiles.push_back(make_int2(k, (int)c0));
}

void drop_graphs(lbm_batch *b) {
  for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
  for (auto &kv : b->seq_graphs) cudaGraphExecDestroy(kv.second);
  b->seq_graphs.clear();
}

// FNV-1a over a byte range (keys the graph cache of step-sequence launches).
unsigned long long fnv1a(const void *p, size_t n, unsigned long long h = 1469598103934665603ull) {
  const unsigned char *c = static_cast<const unsigned char *>(p);
  for (size_t k = 0; k < n; ++k) h = (h ^ c[k]) * 1099511628211ull;
  return h;
}

// Persistent grid of `kernel`: resident blocks per SM (capped by
// blocks_per_sm) times the SM count.
int coop_grid(lbm_batch *b, const void *kernel, int *grid) {
  int per_sm = 0;
  BCUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, b->threads,
                                                      lbm::batch_persistent_smem(b->ndom)),
        "occupancy query");
  if (b->blocks_per_sm > 0 && b->blocks_per_sm < per_sm) per_sm = b->blocks_per_sm;
  int sms = 0;
  BCUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device), "SM count");
  if (per_sm < 1) return bfail(LBM_EINVAL, "persistent kernel does not fit on an SM");
  *grid = per_sm * sms;
  return LBM_OK;
}

bool aligned_to(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Graphs kept for step-sequence launches: a checkpointed adjoint uses a few
// per checkpoint; past this many distinct step tables the cache is emptied.
constexpr size_t kMaxSeqGraphs = 512;

// One cooperative launch through `launch(stream)` (barrier words reset
// first), replayed from a CUDA graph cached under `key` when CUDA can
// capture it; waits for the launch and reports a barrier timeout.
template <class Launch>
int coop_run(lbm_batch *b,
             const std::tuple<int, int, int, unsigned, unsigned long long, unsigned long long> &key,
             Launch &&launch) {
  bool launched = false;
  if (b->use_graph && b->graph_ok) {
    auto it = b->seq_graphs.find(key);
    if (it == b->seq_graphs.end() && b->seq_graphs.size() >= kMaxSeqGraphs) {
      for (auto &kv : b->seq_graphs) cudaGraphExecDestroy(kv.second);
      b->seq_graphs.clear();
      it = b->seq_graphs.end();
    }
    if (it == b->seq_graphs.end()) {
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned), b->capture);
        cudaMemsetAsync(b->d_err, 0, sizeof(int), b->capture);
        launch(b->capture);
        e = cudaStreamEndCapture(b->capture, &g);
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        cudaGetLastError();
        b->graph_ok = false;
      } else {
        it = b->seq_graphs.emplace(key, ge).first;
      }
    }
    if (b->graph_ok) {
      BCUDA(cudaGraphLaunch(it->second, b->stream), "graph launch");
      launched = true;
    }
  }
  if (!launched) {
    BCUDA(cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned), b->stream), "barrier reset");
    BCUDA(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream), "error reset");
    BCUDA(launch(b->stream), "persistent launch");
  }
  int err = 0;
  BCUDA(cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream),
        "error word copy");
  BCUDA(cudaStreamSynchronize(b->stream), "stream sync");
  if (err & lbm::kErrTimeout) return bfail(LBM_ETIMEOUT, "grid barrier timed out");
  return LBM_OK;
}

int upload_tables(lbm_batch *b) {
  if (!b->tiles_dirty) return LBM_OK;
  build_tiles(b);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->d_partials) cudaFree(b->d_partials);
  b->d_tiles = nullptr;
  b->d_partials = nullptr;
  BCUDA(cudaMalloc(&b->d_tiles, sizeof(int2) * b->tiles.size()), "cudaMalloc tiles");
  BCUDA(cudaMalloc(&b->d_partials, sizeof(double) * b->tiles.size()), "cudaMalloc partials");
  BCUDA(cudaMemcpy(b->d_tiles, b->tiles.data(), sizeof(int2) * b->tiles.size(),
                   cudaMemcpyHostToDevice), "tile upload");
  b->tiles_dirty = false;
  drop_graphs(b);
  return LBM_OK;
}

BatchArgs make_args(const lbm_batch *b) {
  BatchArgs a;
  memset(&a, 0, sizeof(a));
  a.f[0] = b->f[0];
  a.f[1] = b->f[1];
#ifdef LBM_CHECK
  a.f_elems = b->f_elems;
  a.cells = (uint32_t)b->cells;
#endif
  a.doms = b->d_doms;
  a.tiles = b->d_tiles;
  a.ntiles = (int)b->tiles.size();
  a.ndom = b->ndom;
  a.walls_any = (b->flags & (LBM_WALL_X | LBM_WALL_Y | LBM_WALL_Z)) != 0;
  a.bar_count = b->d_bar;
  a.bar_gen = b->d_bar + 1;
  a.err = b->d_err;
  a.timeout_ns = (unsigned long long)(b->timeout_s * 1e9);
  return a;
}

int persistent_grid(lbm_batch *b, int *grid) {
  int per_sm = 0;
  BCUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, lbm::batch_persistent_kernel(
                         (b->flags & (LBM_WALL_X | LBM_WALL_Y | LBM_WALL_Z)) != 0),
            b->threads, lbm::batch_persistent_smem(b->ndom)),
        "occupancy query");
  if (b->blocks_per_sm > 0 && b->blocks_per_sm < per_sm) per_sm = b->blocks_per_sm;
  int sms = 0;
  BCUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device), "SM count");
  if (per_sm < 1) return bfail(LBM_EINVAL, "persistent kernel does not fit on an SM");
  *grid = per_sm * sms;
  return LBM_OK;
}

// Alignment the kernels' accesses need (lbm.h conventions); NULL passes here
// (each call judges NULL itself), and it is checked before the handle.
constexpr size_t kAlignF = 256, kAlignField = 4, kAlignF64 = 8;

#define LBM_BREQUIRE_ALIGNED(cond) \
  do {                             \
    if (!(cond)) return bfail(LBM_EINVAL, "misaligned device buffer"); \
  } while (0)

int check_b(const lbm_batch *b) {
  if (!b) return bfail(LBM_EINVAL, "NULL handle");
  if (!b->bound) return bfail(LBM_EUNBOUND, "no buffers bound");
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(int ndom, const int *dims, const float *tau, const float *lid_ux,
                     uint32_t flags, lbm_batch_t **out) {
  if (!out) return bfail(LBM_EINVAL, "out is NULL");
  *out = nullptr;
#ifdef LBM_CHECK
  if (!lbm::check_record()) return bfail(LBM_ENOMEM, "check record allocation failed");
#endif
  if (ndom < 1 || !dims || !tau) return bfail(LBM_EINVAL, "need ndom >= 1, dims, tau");
  if (ndom > lbm::kMaxBatchDomains) return bfail(LBM_ERANGE, "at most 256 domains per batch");
  const uint32_t known = LBM_WALL_X | LBM_WALL_Y | LBM_WALL_Z | LBM_LID;
  if (flags & ~known) return bfail(LBM_EINVAL, "batch supports walls and lid, FP32 only");
  if ((flags & LBM_LID) && !(flags & LBM_WALL_Z)) return bfail(LBM_EINVAL, "LBM_LID needs LBM_WALL_Z");
  lbm_batch *b = new (std::nothrow) lbm_batch();
  if (!b) return bfail(LBM_ENOMEM, "host allocation failed");
  b->ndom = ndom;
  b->flags = flags;
  size_t foff = 0, coff = 0;
  for (int k = 0; k < ndom; ++k) {
    const int nx = dims[3 * k], ny = dims[3 * k + 1], nz = dims[3 * k + 2];
    const float t = tau[k];
    if (nx < 1 || ny < 1 || nz < 1 || !(t > 0.5f) || !isfinite(t)) {
      delete b;
      return bfail(LBM_EINVAL, "bad domain size or tau");
    }
    const size_t cells = (size_t)nx * ny * nz;
    if (cells > (1u << 22) || (size_t)nx * ny >= (1u << 20)) {
      delete b;
      return bfail(LBM_ERANGE, "a batch domain may hold at most 2^22 nodes");
    }
    BatchDom D;
    memset(&D, 0, sizeof(D));
    D.nx = nx;
    D.ny = ny;
    D.nz = nz;
    // Unpadded rows: the batch kernels walk each domain's nodes in dense
    // order, so with pitch = nx every z plane is one contiguous run and no
    // 32-byte sector is ever partly written (a padded row end would leave a
    // partial sector that L2 must complete from DRAM on eviction).
    D.pitch = nx;
    D.plane = (uint32_t)((size_t)D.pitch * ny * nz);
    D.cells = (uint32_t)cells;
    D.foff = foff;
    D.coff = (uint32_t)coff;
    D.walls = flags & (LBM_WALL_X | LBM_WALL_Y | LBM_WALL_Z);
    D.m_nx = magic42((uint32_t)nx);
    D.m_nxy = magic42((uint32_t)(nx * ny));
    D.omega = lbm::relaxation_rate(t);
    D.kf = 1.0f - 0.5f * D.omega;
    const double ux = (lid_ux && (flags & LBM_LID)) ? (double)lid_ux[k] : 0.0;
    for (int i = 0; i < lbm::Q; ++i)
      D.lidc[i] = (flags & LBM_LID) && lbm::kEz[i] == -1
                      ? (float)(6.0 * lbm::weight_d(i) * lbm::kEx[i] * ux)
                      : 0.0f;
    b->doms.push_back(D);
    foff += ((size_t)lbm::Q * D.plane + 63) / 64 * 64;  // 256-byte aligned regions
    coff += cells;
  }
  b->f_elems = foff;
  b->cells = coff;
  if (coff >= (1ull << 32)) {
    delete b;
    return bfail(LBM_ERANGE, "too many nodes in one batch");
  }
  *out = b;
  return LBM_OK;
}

int lbm_batch_destroy(lbm_batch_t *b) {
  if (!b) return LBM_OK;
  drop_graphs(b);
  if (b->d_doms) cudaFree(b->d_doms);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->d_partials) cudaFree(b->d_partials);
  if (b->d_bar) cudaFree(b->d_bar);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
  return LBM_OK;
}

int lbm_batch_layout(const lbm_batch_t *b, size_t *f_bytes, size_t *cells,
                     size_t *f_offsets, size_t *cell_offsets) {
  if (!b) return bfail(LBM_EINVAL, "NULL handle");
  if (f_bytes) *f_bytes = b->f_elems * sizeof(float);
  if (cells) *cells = b->cells;
  for (int k = 0; k < b->ndom; ++k) {
    if (f_offsets) f_offsets[k] = (size_t)b->doms[k].foff;
    if (cell_offsets) cell_offsets[k] = b->doms[k].coff;
  }
  return LBM_OK;
}

int lbm_batch_bind(lbm_batch_t *b, void *f_a, void *f_b, void *stream) {
  if (!b) return bfail(LBM_EINVAL, "NULL handle");
  if (!f_a || !f_b || f_a == f_b) return bfail(LBM_EINVAL, "need two distinct f buffers");
  if (((uintptr_t)f_a % 256) || ((uintptr_t)f_b % 256))
    return bfail(LBM_EINVAL, "f buffers must be 256-byte aligned");
  int dev = 0;
  BCUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (!b->d_doms || dev != b->device) {
    drop_graphs(b);
    if (b->d_doms) cudaFree(b->d_doms);
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->d_partials) cudaFree(b->d_partials);
    if (b->d_bar) cudaFree(b->d_bar);
    if (b->capture) cudaStreamDestroy(b->capture);
    b->d_doms = nullptr;
    b->d_tiles = nullptr;
    b->d_partials = nullptr;
    b->d_bar = nullptr;
    b->capture = nullptr;
    b->device = dev;
    BCUDA(cudaMalloc(&b->d_doms, sizeof(BatchDom) * b->doms.size()), "cudaMalloc domains");
    BCUDA(cudaMemcpy(b->d_doms, b->doms.data(), sizeof(BatchDom) * b->doms.size(),
                     cudaMemcpyHostToDevice), "domain upload");
    BCUDA(cudaMalloc(&b->d_bar, 64), "cudaMalloc barrier");
    BCUDA(cudaMemset(b->d_bar, 0, 64), "barrier clear");
    b->d_err = reinterpret_cast<int *>(b->d_bar + 2);
    BCUDA(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking), "capture stream");
    b->tiles_dirty = true;
  }
  int rc = upload_tables(b);
  if (rc) return rc;
  b->f[0] = static_cast<float *>(f_a);
  b->f[1] = static_cast<float *>(f_b);
  b->cur = 0;
  b->stream = static_cast<cudaStream_t>(stream);
  b->bound = true;
  drop_graphs(b);
  return LBM_OK;
}

int lbm_batch_set_tiling(lbm_batch_t *b, int threads, int blocks_per_sm) {
  if (!b) return bfail(LBM_EINVAL, "NULL handle");
  if (threads < 32 || threads > 256 || threads % 32 || blocks_per_sm < 0)
    return bfail(LBM_EINVAL, "threads in {32..256} step 32, blocks_per_sm >= 0");
  if (threads != b->threads) b->tiles_dirty = true;
  b->threads = threads;
  b->blocks_per_sm = blocks_per_sm;
  drop_graphs(b);
  if (b->bound) return upload_tables(b);
  return LBM_OK;
}

int lbm_batch_set_timeout(lbm_batch_t *b, double seconds) {
  if (!b || !(seconds > 0.0) || seconds > 60.0) return bfail(LBM_EINVAL, "timeout in (0, 60] s");
  b->timeout_s = seconds;
  drop_graphs(b);
  return LBM_OK;
}

int lbm_batch_inject_barrier_fault(lbm_batch_t *b, int extra) {
  if (!b || extra < 0) return bfail(LBM_EINVAL, "extra must be >= 0");
  b->inject_extra = extra;
  drop_graphs(b);
  return LBM_OK;
}

int lbm_batch_use_graph(lbm_batch_t *b, int on) {
  if (!b) return bfail(LBM_EINVAL, "NULL handle");
  b->use_graph = on != 0;
  return LBM_OK;
}

int lbm_batch_info(const lbm_batch_t *b, int *grid, int *threads, int *ntiles,
                   int *graph_used) {
  if (!b) return bfail(LBM_EINVAL, "NULL handle");
  if (grid) {
    int g = 0;
    if (b->bound) {
      int rc = persistent_grid(const_cast<lbm_batch *>(b), &g);
      if (rc) return rc;
    }
    *grid = g;
  }
  if (threads) *threads = b->threads;
  if (ntiles) *ntiles = (int)b->tiles.size();
  if (graph_used) *graph_used = b->use_graph && b->graph_ok;
  return LBM_OK;
}

int lbm_batch_current(const lbm_batch_t *b, void **f_cur, void **f_other) {
  int rc = check_b(b);
  if (rc) return rc;
  if (f_cur) *f_cur = b->f[b->cur];
  if (f_other) *f_other = b->f[1 - b->cur];
  return LBM_OK;
}

int lbm_batch_init_rest(lbm_batch_t *b) {
  int rc = check_b(b);
  if (rc) return rc;
  cudaError_t e = lbm::launch_batch_rest(make_args(b), b->f[b->cur], b->threads, b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch init launch");
  return LBM_OK;
}

int lbm_batch_step(lbm_batch_t *b, int n) {
  int rc = check_b(b);
  if (rc) return rc;
  if (n < 0) return bfail(LBM_EINVAL, "n must be >= 0");
  if (n == 0) return LBM_OK;
  int grid = 0;
  rc = persistent_grid(b, &grid);
  if (rc) return rc;
  BatchArgs a = make_args(b);
  a.nsteps = n;
  a.parity0 = b->cur;
  a.expected = (unsigned)(grid + b->inject_extra);
  const auto key = std::make_tuple(n, b->cur, grid, b->threads, a.expected, a.timeout_ns);
  bool launched = false;
  if (b->use_graph && b->graph_ok) {
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned), b->capture);
        cudaMemsetAsync(b->d_err, 0, sizeof(int), b->capture);
        lbm::launch_batch_persistent(a, grid, b->threads, b->capture);
        e = cudaStreamEndCapture(b->capture, &g);
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        cudaGetLastError();
        b->graph_ok = false;  // this driver cannot capture the cooperative launch
      } else {
        it = b->graphs.emplace(key, ge).first;
      }
    }
    if (b->graph_ok) {
      BCUDA(cudaGraphLaunch(it->second, b->stream), "graph launch");
      launched = true;
    }
  }
  if (!launched) {
    BCUDA(cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned), b->stream), "barrier reset");
    BCUDA(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream), "error reset");
    BCUDA(lbm::launch_batch_persistent(a, grid, b->threads, b->stream), "persistent launch");
  }
  int err = 0;
  BCUDA(cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream),
        "error word copy");
  BCUDA(cudaStreamSynchronize(b->stream), "stream sync");
  b->cur ^= (n & 1);
  if (err & lbm::kErrTimeout) return bfail(LBM_ETIMEOUT, "grid barrier timed out");
  return LBM_OK;
}

int lbm_batch_step_launches(lbm_batch_t *b, int n) {
  int rc = check_b(b);
  if (rc) return rc;
  if (n < 0) return bfail(LBM_EINVAL, "n must be >= 0");
  BatchArgs a = make_args(b);
  for (int k = 0; k < n; ++k) {
    BCUDA(lbm::launch_batch_step(a, b->f[b->cur], b->f[1 - b->cur], b->threads, b->stream),
          "batch step launch");
    b->cur ^= 1;
  }
  return LBM_OK;
}

int lbm_batch_moments(lbm_batch_t *b, float *rho, float *u) {
  LBM_BREQUIRE_ALIGNED(aligned_to(rho, kAlignField) && aligned_to(u, kAlignField));
  int rc = check_b(b);
  if (rc) return rc;
  BCUDA(lbm::launch_batch_moments(make_args(b), b->f[b->cur], rho, u, b->threads, b->stream),
        "batch moments launch");
  return LBM_OK;
}

int lbm_batch_get_f(lbm_batch_t *b, int dom, double *host_f) {
  int rc = check_b(b);
  if (rc) return rc;
  if (dom < 0 || dom >= b->ndom || !host_f) return bfail(LBM_EINVAL, "bad domain or buffer");
  const BatchDom &D = b->doms[dom];
  std::vector<float> stage((size_t)lbm::Q * D.plane);
  BCUDA(cudaMemcpyAsync(stage.data(), b->f[b->cur] + D.foff, stage.size() * sizeof(float),
                        cudaMemcpyDeviceToHost, b->stream), "state copy");
  BCUDA(cudaStreamSynchronize(b->stream), "stream sync");
  for (int i = 0; i < lbm::Q; ++i)
    for (int z = 0; z < D.nz; ++z)
      for (int y = 0; y < D.ny; ++y)
        for (int x = 0; x < D.nx; ++x)
          host_f[(size_t)i * D.cells + ((size_t)z * D.ny + y) * D.nx + x] =
              (double)stage[(size_t)i * D.plane + ((size_t)z * D.ny + y) * D.pitch + x] +
              lbm::weight_d(i);
  return LBM_OK;
}

int lbm_batch_set_f(lbm_batch_t *b, int dom, const double *host_f) {
  int rc = check_b(b);
  if (rc) return rc;
  if (dom < 0 || dom >= b->ndom || !host_f) return bfail(LBM_EINVAL, "bad domain or buffer");
  const BatchDom &D = b->doms[dom];
  std::vector<float> stage((size_t)lbm::Q * D.plane, 0.0f);
  for (int i = 0; i < lbm::Q; ++i)
    for (int z = 0; z < D.nz; ++z)
      for (int y = 0; y < D.ny; ++y)
        for (int x = 0; x < D.nx; ++x)
          stage[(size_t)i * D.plane + ((size_t)z * D.ny + y) * D.pitch + x] =
              (float)(host_f[(size_t)i * D.cells + ((size_t)z * D.ny + y) * D.nx + x] -
                      lbm::weight_d(i));
  BCUDA(cudaMemcpyAsync(b->f[b->cur] + D.foff, stage.data(), stage.size() * sizeof(float),
                        cudaMemcpyHostToDevice, b->stream), "state copy");
  BCUDA(cudaStreamSynchronize(b->stream), "stream sync");
  return LBM_OK;
}

int lbm_batch_init_equilibrium(lbm_batch_t *b, const float *u0) {
  LBM_BREQUIRE_ALIGNED(aligned_to(u0, kAlignField));
  int rc = check_b(b);
  if (rc) return rc;
  BCUDA(lbm::launch_batch_init_eq(make_args(b), b->f[b->cur], u0, b->threads, b->stream),
        "batch init launch");
  return LBM_OK;
}

int lbm_batch_step_to(lbm_batch_t *b, const void *f_in, void *f_out) {
  LBM_BREQUIRE_ALIGNED(aligned_to(f_in, kAlignF) && aligned_to(f_out, kAlignF));
  int rc = check_b(b);
  if (rc) return rc;
  if (!f_in || !f_out || f_in == f_out) return bfail(LBM_EINVAL, "bad buffers");
  BCUDA(lbm::launch_batch_step(make_args(b), static_cast<const float *>(f_in),
                               static_cast<float *>(f_out), b->threads, b->stream),
        "batch step launch");
  return LBM_OK;
}

int lbm_batch_step_to_moments(lbm_batch_t *b, const void *f_in, void *f_out, float *rho,
                              float *u) {
  LBM_BREQUIRE_ALIGNED(aligned_to(f_in, kAlignF) && aligned_to(f_out, kAlignF) &&
                       aligned_to(rho, kAlignField) && aligned_to(u, kAlignField));
  int rc = check_b(b);
  if (rc) return rc;
  if (!f_in || !f_out || f_in == f_out || !rho || !u) return bfail(LBM_EINVAL, "bad buffers");
  BCUDA(lbm::launch_batch_step_mom(make_args(b), static_cast<const float *>(f_in),
                                   static_cast<float *>(f_out), rho, u, b->threads, b->stream),
        "batch step launch");
  return LBM_OK;
}

int lbm_batch_adjoint_seed(lbm_batch_t *b, const void *f_T, const float *u_target,
                           float *lambda_T, float *grad_force, double *loss) {
  LBM_BREQUIRE_ALIGNED(aligned_to(f_T, kAlignF) && aligned_to(u_target, kAlignField) &&
                       aligned_to(lambda_T, kAlignField) && aligned_to(grad_force, kAlignField) &&
                       aligned_to(loss, kAlignF64));
  int rc = check_b(b);
  if (rc) return rc;
  if (!f_T || !u_target || !lambda_T) return bfail(LBM_EINVAL, "NULL buffer");
  BatchArgs a = make_args(b);
  BCUDA(lbm::launch_batch_adjoint_seed(a, static_cast<const float *>(f_T), u_target, lambda_T,
                                       grad_force, loss ? b->d_partials : nullptr, b->threads,
                                       b->stream),
        "batch seed launch");
  if (loss) {
    lbm::Scratch scr;
    scr.partials = b->d_partials;
    BCUDA(lbm::launch_finalize_sum(scr, a.ntiles, 0.0, loss, b->stream), "loss reduction");
  }
  return LBM_OK;
}

int lbm_batch_adjoint_step(lbm_batch_t *b, const void *f_n, const float *lambda_in,
                           float *lambda_out, float *grad_force) {
  LBM_BREQUIRE_ALIGNED(aligned_to(f_n, kAlignF) && aligned_to(lambda_in, kAlignField) &&
                       aligned_to(lambda_out, kAlignField) && aligned_to(grad_force, kAlignField));
  int rc = check_b(b);
  if (rc) return rc;
  if (!f_n || !lambda_in || !lambda_out || lambda_in == lambda_out)
    return bfail(LBM_EINVAL, "bad buffers");
  BCUDA(lbm::launch_batch_adjoint_step(make_args(b), static_cast<const float *>(f_n),
                                       lambda_in, lambda_out, grad_force, b->threads,
                                       b->stream),
        "batch adjoint step launch");
  return LBM_OK;
}

int lbm_batch_adjoint_step_moments(lbm_batch_t *b, const float *rho_n, const float *u_n,
                                   const float *lambda_in, float *lambda_out,
                                   float *grad_force) {
  LBM_BREQUIRE_ALIGNED(aligned_to(rho_n, kAlignField) && aligned_to(u_n, kAlignField) &&
                       aligned_to(lambda_in, kAlignField) && aligned_to(lambda_out, kAlignField) &&
                       aligned_to(grad_force, kAlignField));
  int rc = check_b(b);
  if (rc) return rc;
  if (!rho_n || !u_n || !lambda_in || !lambda_out || lambda_in == lambda_out)
    return bfail(LBM_EINVAL, "bad buffers");
  BCUDA(lbm::launch_batch_adjoint_step_mom(make_args(b), rho_n, u_n, lambda_in, lambda_out,
                                           grad_force, b->threads, b->stream),
        "batch adjoint step launch");
  return LBM_OK;
}

int lbm_batch_run(lbm_batch_t *b, int n, const void *const *f_in, void *const *f_out,
                  float *const *rho, float *const *u) {
  int rc = check_b(b);
  if (rc) return rc;
  if (n < 1 || n > lbm::kMaxSeqSteps || !f_in || !f_out)
    return bfail(LBM_EINVAL, "need 1 <= n <= 64 and the f_in, f_out arrays");
  if ((rho == nullptr) != (u == nullptr)) return bfail(LBM_EINVAL, "give both rho and u or neither");
  lbm::BatchFwdSeq q;
  memset(&q, 0, sizeof(q));
  q.n = n;
  for (int k = 0; k < n; ++k) {
    if (!f_in[k] || !f_out[k] || f_in[k] == f_out[k]) return bfail(LBM_EINVAL, "bad f buffers");
    if (!aligned_to(f_in[k], 256) || !aligned_to(f_out[k], 256))
      return bfail(LBM_EINVAL, "f buffers must be 256-byte aligned");
    q.fin[k] = static_cast<const float *>(f_in[k]);
    q.fout[k] = static_cast<float *>(f_out[k]);
    if (rho) {
      if (!rho[k] || !u[k]) return bfail(LBM_EINVAL, "NULL rho or u buffer");
      if (!aligned_to(rho[k], 4) || !aligned_to(u[k], 4))
        return bfail(LBM_EINVAL, "rho/u misaligned");
      q.rho[k] = rho[k];
      q.u[k] = u[k];
    }
  }
  const bool walls = (b->flags & (LBM_WALL_X | LBM_WALL_Y | LBM_WALL_Z)) != 0;
  int grid = 0;
  rc = coop_grid(b, lbm::batch_fwd_seq_kernel(walls, rho != nullptr), &grid);
  if (rc) return rc;
  BatchArgs a = make_args(b);
  a.expected = (unsigned)(grid + b->inject_extra);
  const auto key = std::make_tuple(rho ? 1 : 0, grid, b->threads, a.expected, a.timeout_ns,
                                   fnv1a(&q, sizeof(q)));
  return coop_run(b, key, [&](cudaStream_t s) {
    return lbm::launch_batch_fwd_seq(a, q, grid, b->threads, s);
  });
}

int lbm_batch_adjoint_run(lbm_batch_t *b, int n, const float *const *rho, const float *const *u,
                          float *lambda_a, float *lambda_b, float *grad_force) {
  int rc = check_b(b);
  if (rc) return rc;
  if (n < 1 || n > lbm::kMaxSeqSteps || !rho || !u)
    return bfail(LBM_EINVAL, "need 1 <= n <= 64 and the rho, u arrays");
  if (!lambda_a || !lambda_b || lambda_a == lambda_b)
    return bfail(LBM_EINVAL, "need two distinct lambda buffers");
  if (!aligned_to(lambda_a, 256) || !aligned_to(lambda_b, 256) ||
      (grad_force && !aligned_to(grad_force, 4)))
    return bfail(LBM_EINVAL, "lambda buffers must be 256-byte aligned");
  lbm::BatchAdjSeq q;
  memset(&q, 0, sizeof(q));
  q.n = n;
  q.lam[0] = lambda_a;
  q.lam[1] = lambda_b;
  q.gF = grad_force;
  for (int k = 0; k < n; ++k) {
    if (!rho[k] || !u[k]) return bfail(LBM_EINVAL, "NULL rho or u buffer");
    if (!aligned_to(rho[k], 4) || !aligned_to(u[k], 4))
      return bfail(LBM_EINVAL, "rho/u misaligned");
    q.rho[k] = rho[k];
    q.u[k] = u[k];
  }
  int grid = 0;
  rc = coop_grid(b, lbm::batch_adj_seq_kernel(grad_force != nullptr), &grid);
  if (rc) return rc;
  BatchArgs a = make_args(b);
  a.expected = (unsigned)(grid + b->inject_extra);
  const auto key = std::make_tuple(2 + (grad_force ? 1 : 0), grid, b->threads, a.expected,
                                   a.timeout_ns, fnv1a(&q, sizeof(q)));
  return coop_run(b, key, [&](cudaStream_t s) {
    return lbm::launch_batch_adj_seq(a, q, grid, b->threads, s);
  });
}

int lbm_batch_adjoint_u0(lbm_batch_t *b, const float *lambda0, const float *u0,
                         float *grad_u0) {
  LBM_BREQUIRE_ALIGNED(aligned_to(lambda0, kAlignField) && aligned_to(u0, kAlignField) &&
                       aligned_to(grad_u0, kAlignField));
  int rc = check_b(b);
  if (rc) return rc;
  if (!lambda0 || !grad_u0) return bfail(LBM_EINVAL, "NULL buffer");
  BCUDA(lbm::launch_batch_adjoint_u0(make_args(b), lambda0, u0, grad_u0, b->threads, b->stream),
        "batch u0 gradient launch");
  return LBM_OK;
}

int lbm_batch_autotune(lbm_batch_t *b, const char *cache_path, int steps, int *threads_out,
                       int *blocks_per_sm_out, float *ms_out) {
  int rc = check_b(b);
  if (rc) return rc;
  if (steps < 1 || steps > 100000) return bfail(LBM_EINVAL, "steps in [1, 100000]");
  steps += steps & 1;  // even: the timed call replays the graph the untimed one captured
  // key: GPU, the domain list (FNV-1a over dims and walls) and the flags
  uint64_t hsh = 1469598103934665603ull;
  auto mix = [&](uint64_t v) {
    for (int k = 0; k < 8; ++k) {
      hsh ^= (v >> (8 * k)) & 0xffu;
      hsh *= 1099511628211ull;
    }
  };
  for (const BatchDom &D : b->doms) {
    mix((uint64_t)D.nx);
    mix((uint64_t)D.ny);
    mix((uint64_t)D.nz);
    mix((uint64_t)D.walls);
  }
  char geo[96];
  snprintf(geo, sizeof geo, "batch/%d/%016llx/flags%u", b->ndom, (unsigned long long)hsh,
           b->flags);
  const std::string key = lbm::device_key(b->device) + "/" + geo;
  int t = 0, bps = 0;
  float best_ms = 0.f;
  if (lbm::tune_cache_lookup(cache_path, key, &t, &bps, &best_ms) &&
      lbm_batch_set_tiling(b, t, bps) == LBM_OK) {
    if (threads_out) *threads_out = t;
    if (blocks_per_sm_out) *blocks_per_sm_out = bps;
    if (ms_out) *ms_out = best_ms;
    return LBM_OK;
  }
  // tile sizes x resident blocks per SM (0 = as many as fit) of the
  // persistent launch; the untimed first call also captures its graph
  static const int kThreads[] = {64, 128, 256};
  static const int kBps[] = {0, 2, 4, 6, 8};
  int best_t = 0, best_b = 0;
  for (int tt : kThreads) {
    for (int bb : kBps) {
      rc = lbm_batch_set_tiling(b, tt, bb);
      if (rc) return rc;
      float ms = 0.f;
      rc = lbm::time_calls(b->stream, 1, [&]() { return lbm_batch_step(b, steps); }, &ms);
      if (rc) return rc;
      ms /= steps;
      if (!best_t || ms < best_ms) {
        best_t = tt;
        best_b = bb;
        best_ms = ms;
      }
    }
  }
  rc = lbm_batch_set_tiling(b, best_t, best_b);
  if (rc) return rc;
  if (lbm::tune_cache_store(cache_path, key, best_t, best_b, best_ms))
    return bfail(LBM_EINVAL, "autotune cache not writable");
  if (threads_out) *threads_out = best_t;
  if (blocks_per_sm_out) *blocks_per_sm_out = best_b;
  if (ms_out) *ms_out = best_ms;
  return LBM_OK;
}

}  // extern "C"
