// lbm_capi.cu - the extern "C" entry points of liblbm.so declared in lbm.h:
// handle management, argument checks, the ping-pong buffer swap of Sec. 4.1
// (footnote), host exchange of states, and the launch of the kernels in
// lbm_step.cu.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <new>

#include "d3q19.cuh"
#include "internal.h"
#include "step_tma.h"

using lbm::StepArgs;

namespace lbm {

float relaxation_rate(float tau) {
  // c = omega/12 on a grid of 22 significant bits, so that 12 c needs at
  // most 24 bits and is an exact FP32 value, and of multiples of 2^-26, so
  // that omega = 12 c is a multiple of 2^-24 and 1 - omega is exact too
  // (this coarsens omega below 1/2, i.e. tau > 2, to 2^-24 absolute). Among
  // the grid points nearest to 1/(12 tau), take one that the kernels'
  // product omega * (1/12) reproduces exactly.
  const double c0 = 1.0 / (12.0 * (double)tau);
  int e = 0;
  frexp(c0, &e);  // c0 in [2^(e-1), 2^e)
  const double q = fmax(ldexp(1.0, e - 22), ldexp(1.0, -26));
  const double cr = nearbyint(c0 / q) * q;
  for (int k = 0; k < 64; ++k) {
    const double cand = cr + (k % 2 ? -1.0 : 1.0) * (double)((k + 1) / 2) * q;
    if (!(cand > 0.0)) continue;
    volatile float c = (float)cand;
    volatile float om = 12.0f * c;
    volatile float back = om * (1.0f / 12.0f);
    volatile float keep = 1.0f - om;
    if ((double)c == cand && (double)om == 12.0 * cand && back == c &&
        (double)keep == 1.0 - 12.0 * cand)
      return om;
  }
  return (float)(1.0 / (double)tau);  // tau beyond ~4e6: no such value
}

}  // namespace lbm

namespace {

thread_local char g_last_error[256] = "";

int fail(int code, const char *what) {
  snprintf(g_last_error, sizeof(g_last_error), "%s", what);
  return code;
}

int cuda_fail(cudaError_t e, const char *where) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where,
           cudaGetErrorString(e));
  return LBM_ECUDA;
}

#define LBM_CUDA(call, where)                    \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

constexpr uint32_t kKnownFlags = LBM_WALL_X | LBM_WALL_Y | LBM_WALL_Z |
                                 LBM_LID | LBM_STORE_F16 | LBM_STORE_BF16 |
                                 LBM_FORCE | LBM_ADJOINT | LBM_WALLS_ONSITE;

// On-site walls on a handle that has a walled axis.
bool onsite(const lbm_t *h) {
  return (h->flags & LBM_WALLS_ONSITE) && (h->flags & (LBM_WALL_X | LBM_WALL_Y | LBM_WALL_Z));
}

StepArgs make_args(const lbm_t *h, const void *fin, void *fout) {
  StepArgs a;
  memset(&a, 0, sizeof(a));
  a.fin = fin;
  a.fout = fout;
  a.force = (h->flags & LBM_FORCE) ? h->force : nullptr;
  a.nx = h->nx;
  a.ny = h->ny;
  a.nz = h->nz;
  a.pitch = h->pitch;
  a.plane = (uint32_t)h->plane;
  a.cells = (uint32_t)((size_t)h->nx * h->ny * h->nz);
  a.omega = lbm::relaxation_rate(h->tau);
  a.kf = 1.0f - 0.5f * a.omega;
  a.walls = h->flags & (LBM_WALL_X | LBM_WALL_Y | LBM_WALL_Z);
  a.z0 = 0;
  a.zn = h->nz;
  // The one-node kernel with 16-bit storage is issue-bound: there the branch
  // form's shorter common path wins once wall nodes are rare in every warp
  // (long rows). FP32 is bandwidth-bound and the divergence-free select form
  // is never slower; the two-node kernel selects only in the warps that hold
  // a wall node and is fastest so.
  a.onsite = onsite(h) ? 1 : 0;
  a.onsite_lid = (h->flags & LBM_LID) ? 1 : 0;
  for (int k = 0; k < 3; ++k) a.lid[k] = h->lid[k];
  a.wall_select = h->wall_mode == LBM_WALLS_SELECT ||
                  (h->wall_mode == LBM_WALLS_AUTO &&
                   (h->storage == lbm::kF32 || h->nx < 256 || h->kernel == LBM_KERNEL_X2 ||
                    h->kernel == LBM_KERNEL_X4));
  for (int i = 0; i < lbm::Q; ++i) {
    a.lidc[i] = 0.0f;
    if ((h->flags & LBM_LID) && lbm::kEz[i] == -1)
      a.lidc[i] = (float)(6.0 * lbm::weight_d(i) *
                          (lbm::kEx[i] * (double)h->lid[0] +
                           lbm::kEy[i] * (double)h->lid[1] +
                           lbm::kEz[i] * (double)h->lid[2]));
  }
  return a;
}

int check_bound(const lbm_t *h) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  if (!h->bound) return fail(LBM_EUNBOUND, "no buffers bound");
  return LBM_OK;
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Alignment the kernels' accesses need (lbm.h conventions); NULL passes here
// (each call judges NULL itself). Checked before the handle's state, so a
// misaligned buffer is reported as such whatever the handle.
constexpr size_t kAlignF = 256, kAlignField = 4, kAlignF64 = 8;

#define LBM_REQUIRE_ALIGNED(cond) \
  do {                            \
    if (!(cond)) return fail(LBM_EINVAL, "misaligned device buffer"); \
  } while (0)

int ensure_scratch(lbm_t *h) {
  int dev = 0;
  LBM_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (h->scr.partials && h->device == dev) return LBM_OK;
  if (h->scr.partials) {
    cudaFree(h->scr.partials);
    h->scr = lbm::Scratch();
  }
  // one allocation: partials | sum | err
  const size_t bytes = sizeof(double) * (lbm::kReduceBlocks + 1) + 64;
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(LBM_ENOMEM, "cudaMalloc of the handle scratch failed");
  }
  h->scr.partials = static_cast<double *>(p);
  h->scr.sum = h->scr.partials + lbm::kReduceBlocks;
  h->scr.err = reinterpret_cast<int *>(h->scr.sum + 1);
  h->scr.nblocks = lbm::kReduceBlocks;
  h->device = dev;
  LBM_CUDA(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  LBM_CUDA(cudaMemset(h->scr.err, 0, sizeof(int)), "cudaMemset");
  return LBM_OK;
}

cudaError_t launch_one_step(const lbm_t *h, bool mom, const StepArgs &a, cudaStream_t s) {
  if (h->kernel == LBM_KERNEL_PAIR && h->storage != lbm::kF32)
    return lbm::launch_step_pair16(h->storage, mom, a, h->pbx, h->pby, s);
  if (h->kernel == LBM_KERNEL_X2)
    return lbm::launch_step_x2(h->storage, mom, a, h->pbx, h->pby, s);
  if (h->kernel == LBM_KERNEL_X4)
    return lbm::launch_step_x4(h->storage, mom, a, h->pbx, h->pby, s);
  if (h->kernel == LBM_KERNEL_TMA)
    return lbm::launch_step_tma(h->storage, mom, a, h->scr.err, h->pby, h->sms, s);
  if ((h->kernel == LBM_KERNEL_BULK || h->kernel == LBM_KERNEL_BULK1) && !mom)
    return lbm::launch_step_bulk(h->storage, a, h->scr.err,
                                 h->kernel == LBM_KERNEL_BULK1 ? 1 : 0, h->sms, s);
  return lbm::launch_step(h->storage, mom, a, h->bx, h->by, s);
}
cudaError_t launch_one_step(const lbm_t *h, bool mom, const StepArgs &a) {
  return launch_one_step(h, mom, a, h->stream);
}

void drop_graphs(lbm_t *h) {
  for (int p = 0; p < 2; ++p) {
    if (h->gexec[p]) cudaGraphExecDestroy(h->gexec[p]);
    h->gexec[p] = nullptr;
  }
}

// The graph of graph_steps steps starting from buffer p (captured on a
// private stream on first use or after a configuration change).
int step_graph(lbm_t *h, int p, cudaGraphExec_t *out) {
  if (h->gexec[p] && h->gexec_version[p] == h->config_version) {
    *out = h->gexec[p];
    return LBM_OK;
  }
  if (h->gexec[p]) cudaGraphExecDestroy(h->gexec[p]);
  h->gexec[p] = nullptr;
  if (!h->gcap)
    LBM_CUDA(cudaStreamCreateWithFlags(&h->gcap, cudaStreamNonBlocking), "stream create");
  LBM_CUDA(cudaStreamBeginCapture(h->gcap, cudaStreamCaptureModeThreadLocal), "graph capture");
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < h->graph_steps && e == cudaSuccess; ++k) {
    const int c = p ^ (k & 1);
    e = launch_one_step(h, false, make_args(h, h->f[c], h->f[1 - c]), h->gcap);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(h->gcap, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->gexec[p], g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->gexec[p] = nullptr;
    return cuda_fail(e, "step graph capture");
  }
  h->gexec_version[p] = h->config_version;
  *out = h->gexec[p];
  return LBM_OK;
}

// Streams, events and staging of lbm_run_host, created on first use.
int ensure_pipeline(lbm_t *h) {
  if (h->pipe_ready) return LBM_OK;
  const size_t cells = (size_t)h->nx * h->ny * h->nz;
  if (cudaMalloc(&h->stage, 7 * cells * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    h->stage = nullptr;
    return fail(LBM_ENOMEM, "cudaMalloc of the host-transfer staging failed");
  }
  LBM_CUDA(cudaStreamCreateWithFlags(&h->copy_in, cudaStreamNonBlocking), "stream create");
  LBM_CUDA(cudaStreamCreateWithFlags(&h->copy_out, cudaStreamNonBlocking), "stream create");
  LBM_CUDA(cudaEventCreateWithFlags(&h->ev_start, cudaEventDisableTiming), "event create");
  LBM_CUDA(cudaEventCreateWithFlags(&h->ev_done, cudaEventDisableTiming), "event create");
  for (int k = 0; k < lbm_lattice::kMaxSlabs; ++k) {
    LBM_CUDA(cudaEventCreateWithFlags(&h->ev_in[k], cudaEventDisableTiming), "event create");
    LBM_CUDA(cudaEventCreateWithFlags(&h->ev_out[k], cudaEventDisableTiming), "event create");
  }
  h->pipe_ready = true;
  return LBM_OK;
}

void release_pipeline(lbm_t *h) {
  if (!h->pipe_ready) {
    if (h->stage) cudaFree(h->stage);
    return;
  }
  cudaFree(h->stage);
  cudaStreamDestroy(h->copy_in);
  cudaStreamDestroy(h->copy_out);
  cudaEventDestroy(h->ev_start);
  cudaEventDestroy(h->ev_done);
  for (int k = 0; k < lbm_lattice::kMaxSlabs; ++k) {
    cudaEventDestroy(h->ev_in[k]);
    cudaEventDestroy(h->ev_out[k]);
  }
  h->pipe_ready = false;
  h->stage = nullptr;
}

int do_steps(lbm_t *h, int n, float *rho, float *u) {
  // whole graphs first (an even number of steps each, so the current buffer
  // is unchanged), then plain launches; a step writing rho, u is always plain
  const int G = h->graph_steps;
  if (G > 0 && n - (rho ? 1 : 0) >= G) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    LBM_CUDA(cudaStreamIsCapturing(h->stream, &cs), "stream query");
    if (cs == cudaStreamCaptureStatusNone) {
      cudaGraphExec_t ge = nullptr;
      int rc = step_graph(h, h->cur, &ge);
      if (rc) return rc;
      const int reps = (n - (rho ? 1 : 0)) / G;
      for (int r = 0; r < reps; ++r) LBM_CUDA(cudaGraphLaunch(ge, h->stream), "graph launch");
      n -= reps * G;
    }
  }
  for (int k = 0; k < n; ++k) {
    StepArgs a = make_args(h, h->f[h->cur], h->f[1 - h->cur]);
    const bool mom = (rho != nullptr) && (k == n - 1);
    if (mom) {
      a.rho = rho;
      a.u = u;
    }
    cudaError_t e = launch_one_step(h, mom, a);
    if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
    h->cur ^= 1;
  }
  return LBM_OK;
}

float host_to_float(const void *base, size_t k, int storage) {
  switch (storage) {
    case lbm::kF16: return __half2float(static_cast<const __half *>(base)[k]);
    case lbm::kBF16:
      return __bfloat162float(static_cast<const __nv_bfloat16 *>(base)[k]);
    default: return static_cast<const float *>(base)[k];
  }
}

void host_from_float(void *base, size_t k, int storage, float v) {
  switch (storage) {
    case lbm::kF16: static_cast<__half *>(base)[k] = __float2half_rn(v); break;
    case lbm::kBF16:
      static_cast<__nv_bfloat16 *>(base)[k] = __float2bfloat16_rn(v);
      break;
    default: static_cast<float *>(base)[k] = v;
  }
}

}  // namespace

namespace lbm {
int set_error(int code, const char *what) { return fail(code, what); }
int set_cuda_error(cudaError_t e, const char *where) { return cuda_fail(e, where); }

#ifdef LBM_CHECK
// The refused-access record of the check build: allocated and zeroed once,
// on the first handle creation (before any stream capture, during which a
// cudaMalloc is not allowed), and kept for the life of the process.
CheckRecord *check_record() {
  static CheckRecord *rec = [] {
    CheckRecord *p = nullptr;
    if (cudaMalloc(&p, sizeof(CheckRecord)) != cudaSuccess) return (CheckRecord *)nullptr;
    if (cudaMemset(p, 0, sizeof(CheckRecord)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess)
      return (CheckRecord *)nullptr;
    return p;
  }();
  return rec;
}

static std::atomic<size_t> g_check_narrow{0};
size_t check_narrow_bytes() { return g_check_narrow.load(); }
#endif
}  // namespace lbm

extern "C" {

const char *lbm_strerror(int code) {
  switch (code) {
    case LBM_OK: return "LBM_OK";
    case LBM_EINVAL: return "LBM_EINVAL: invalid argument";
    case LBM_ENOMEM: return "LBM_ENOMEM: allocation failed";
    case LBM_ECUDA: return "LBM_ECUDA: CUDA error";
    case LBM_ETIMEOUT: return "LBM_ETIMEOUT: bounded device wait gave up";
    case LBM_ENONFINITE: return "LBM_ENONFINITE: non-finite density";
    case LBM_EUNBOUND: return "LBM_EUNBOUND: no buffers bound";
    case LBM_ERANGE: return "LBM_ERANGE: size above the supported maximum";
    case LBM_ENOTSUP: return "LBM_ENOTSUP: not in this build";
    default: return "LBM: unknown status code";
  }
}

const char *lbm_last_error(void) { return g_last_error; }

int lbm_create(int nx, int ny, int nz, float tau, uint32_t flags,
               lbm_t **out) {
  if (!out) return fail(LBM_EINVAL, "out is NULL");
  *out = nullptr;
#ifdef LBM_CHECK
  if (!lbm::check_record()) return fail(LBM_ENOMEM, "check record allocation failed");
#endif
  if (nx < 1 || ny < 1 || nz < 1) return fail(LBM_EINVAL, "sizes must be >= 1");
  if (!(tau > 0.5f) || !isfinite(tau)) return fail(LBM_EINVAL, "tau must be > 1/2");
  if (flags & ~kKnownFlags) return fail(LBM_EINVAL, "unknown flag bits");
  const uint32_t st = flags & (LBM_STORE_F16 | LBM_STORE_BF16);
  if (st == (LBM_STORE_F16 | LBM_STORE_BF16))
    return fail(LBM_EINVAL, "more than one storage type");
  if ((flags & LBM_LID) && !(flags & LBM_WALL_Z))
    return fail(LBM_EINVAL, "LBM_LID needs LBM_WALL_Z");
  if ((flags & LBM_ADJOINT) && st) return fail(LBM_EINVAL, "LBM_ADJOINT needs FP32 storage");
  if (flags & LBM_WALLS_ONSITE) {
    if (((flags & LBM_WALL_X) && nx < 3) || ((flags & LBM_WALL_Y) && ny < 3) ||
        ((flags & LBM_WALL_Z) && nz < 3))
      return fail(LBM_EINVAL, "on-site walls need >= 3 nodes along every walled axis");
    if (flags & LBM_ADJOINT) return fail(LBM_EINVAL, "the adjoint supports halfway walls only");
  }
  const int storage = st == LBM_STORE_F16 ? lbm::kF16
                      : st == LBM_STORE_BF16 ? lbm::kBF16 : lbm::kF32;
  const int eb = storage == lbm::kF32 ? 4 : 2;
  const int align = 32 / eb;  // 32-byte rows
  const long long pitch = ((long long)nx + align - 1) / align * align;
  const long long plane = pitch * ny * (long long)nz;
  if (plane >= (1ll << 31)) return fail(LBM_ERANGE, "nz*ny*pitch must be < 2^31");
  lbm_t *h = new (std::nothrow) lbm_t();
  if (!h) return fail(LBM_ENOMEM, "host allocation failed");
  h->nx = nx;
  h->ny = ny;
  h->nz = nz;
  h->pitch = (int)pitch;
  h->flags = flags;
  h->storage = storage;
  h->elem_bytes = eb;
  h->plane = (size_t)plane;
  h->tau = tau;
  h->lid[0] = h->lid[1] = h->lid[2] = 0.0f;
  h->f[0] = h->f[1] = nullptr;
  h->cur = 0;
  h->force = nullptr;
  h->stream = nullptr;
  h->bound = false;
  const int bx = nx >= 128 ? 128 : ((nx + 31) / 32) * 32;
  int by = 256 / bx;
  if (by > ny) by = ny;
  h->bx = bx;
  h->by = by < 1 ? 1 : by;
  // two nodes per thread: fewer instructions per node (decisive where the
  // one-node kernel is issue-bound, 16-bit storage; about 1% with FP32)
  h->kernel = LBM_KERNEL_X2;
  h->wall_mode = LBM_WALLS_AUTO;
  h->pbx = 64;  // 64 pairs x 2 rows measured best for the two-node kernel
  h->pby = ny < 2 ? ny : 2;
  h->device = -1;
  h->stage = nullptr;
  h->pipe_ready = false;
  h->graph_steps = 32;
  h->config_version = 0;
  h->gcap = nullptr;
  h->gexec[0] = h->gexec[1] = nullptr;
  h->gexec_version[0] = h->gexec_version[1] = 0;
  *out = h;
  return LBM_OK;
}

int lbm_destroy(lbm_t *h) {
  if (!h) return LBM_OK;
  release_pipeline(h);
  drop_graphs(h);
  if (h->gcap) cudaStreamDestroy(h->gcap);
  if (h->scr.partials) cudaFree(h->scr.partials);
  delete h;
  return LBM_OK;
}

int lbm_get_layout(const lbm_t *h, lbm_layout_t *out) {
  if (!h || !out) return fail(LBM_EINVAL, "NULL argument");
  out->nx = h->nx;
  out->ny = h->ny;
  out->nz = h->nz;
  out->pitch = h->pitch;
  out->elem_bytes = h->elem_bytes;
  out->plane = h->plane;
  out->f_bytes = (size_t)lbm::Q * h->plane * h->elem_bytes;
  // adjoint buffers are FP32 on the FP32 row alignment
  const size_t pitch32 = ((size_t)h->nx + 7) / 8 * 8;
  out->lambda_bytes = (size_t)lbm::Q * pitch32 * h->ny * h->nz * 4;
  out->cells = (size_t)h->nx * h->ny * h->nz;
  return LBM_OK;
}

int lbm_buffer_bytes(const lbm_t *h, int which, size_t *bytes) {
  if (!h || !bytes) return fail(LBM_EINVAL, "NULL argument");
  lbm_layout_t L;
  lbm_get_layout(h, &L);
  switch (which) {
    case LBM_BUF_F: *bytes = L.f_bytes; break;
    case LBM_BUF_RHO: *bytes = L.cells * sizeof(float); break;
    case LBM_BUF_FORCE:
    case LBM_BUF_U:
    case LBM_BUF_GRADF: *bytes = 3 * L.cells * sizeof(float); break;
    case LBM_BUF_LAMBDA: *bytes = L.lambda_bytes; break;
    default: return fail(LBM_EINVAL, "unknown buffer kind");
  }
  return LBM_OK;
}

int lbm_bind(lbm_t *h, void *f_a, void *f_b, const float *force, void *stream) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  if (!f_a || !f_b || f_a == f_b) return fail(LBM_EINVAL, "need two distinct f buffers");
  if (!aligned(f_a, 256) || !aligned(f_b, 256))
    return fail(LBM_EINVAL, "f buffers must be 256-byte aligned");
  if ((h->flags & LBM_FORCE) && !force)
    return fail(LBM_EINVAL, "LBM_FORCE needs a force field");
  if (force && !aligned(force, 4)) return fail(LBM_EINVAL, "force misaligned");
  int rc = ensure_scratch(h);
  if (rc) return rc;
  h->f[0] = f_a;
  h->f[1] = f_b;
  h->cur = 0;
  h->force = force;
  h->stream = static_cast<cudaStream_t>(stream);
  h->bound = true;
  h->config_version++;
  return LBM_OK;
}

int lbm_set_lid(lbm_t *h, float ux, float uy, float uz) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  if (!(h->flags & LBM_LID)) return fail(LBM_EINVAL, "handle has no lid");
  if (!isfinite(ux) || !isfinite(uy) || !isfinite(uz))
    return fail(LBM_EINVAL, "lid velocity not finite");
  h->lid[0] = ux;
  h->lid[1] = uy;
  h->lid[2] = uz;
  h->config_version++;
  return LBM_OK;
}

int lbm_set_tau(lbm_t *h, float tau) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  if (!(tau > 0.5f) || !isfinite(tau)) return fail(LBM_EINVAL, "tau must be > 1/2");
  h->tau = tau;
  h->config_version++;
  return LBM_OK;
}

int lbm_set_block(lbm_t *h, int bx, int by) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  if (bx < 32 || bx % 32 != 0 || by < 1 || bx * by > 256)
    return fail(LBM_EINVAL, "block must be bx%32==0, by>=1, bx*by<=256");
  h->bx = bx;
  h->by = by;
  h->config_version++;
  return LBM_OK;
}

int lbm_set_kernel(lbm_t *h, int variant) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  if (variant != LBM_KERNEL_NODE && variant != LBM_KERNEL_PAIR && variant != LBM_KERNEL_BULK &&
      variant != LBM_KERNEL_BULK1 && variant != LBM_KERNEL_X2 && variant != LBM_KERNEL_X4 &&
      variant != LBM_KERNEL_TMA)
    return fail(LBM_EINVAL, "unknown kernel variant");
  if (variant == LBM_KERNEL_PAIR && h->storage == lbm::kF32)
    return fail(LBM_EINVAL, "the shuffle pair kernel needs 16-bit storage");
  if (variant == LBM_KERNEL_X4 && h->storage == lbm::kF32)
    return fail(LBM_EINVAL, "the four-node kernel needs 16-bit storage");
  if (variant == LBM_KERNEL_TMA && h->storage == lbm::kF32)
    return fail(LBM_EINVAL, "the tensor-copy staged kernel needs 16-bit storage");
  if (onsite(h) && variant != LBM_KERNEL_X2 && variant != LBM_KERNEL_NODE)
    return fail(LBM_EINVAL, "on-site walls run on LBM_KERNEL_X2 or LBM_KERNEL_NODE");
  h->kernel = variant;
  h->config_version++;
  return LBM_OK;
}

int lbm_set_wall_mode(lbm_t *h, int mode) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  if (mode < LBM_WALLS_AUTO || mode > LBM_WALLS_SELECT) return fail(LBM_EINVAL, "bad mode");
  h->wall_mode = mode;
  h->config_version++;
  return LBM_OK;
}

int lbm_set_graph_steps(lbm_t *h, int steps) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  if (steps < 0 || steps > 1024 || (steps & 1))
    return fail(LBM_EINVAL, "graph steps must be even, in [0, 1024]");
  h->graph_steps = steps;
  drop_graphs(h);
  return LBM_OK;
}

int lbm_set_pair_block(lbm_t *h, int bxp, int by) {
  if (!h) return fail(LBM_EINVAL, "NULL handle");
  if (bxp < 32 || bxp % 32 != 0 || by < 1 || bxp * by > 256)
    return fail(LBM_EINVAL, "pair block must be bxp%32==0, by>=1, bxp*by<=256");
  h->pbx = bxp;
  h->pby = by;
  h->config_version++;
  return LBM_OK;
}

int lbm_current(const lbm_t *h, void **f_cur, void **f_other) {
  int rc = check_bound(h);
  if (rc) return rc;
  if (f_cur) *f_cur = h->f[h->cur];
  if (f_other) *f_other = h->f[1 - h->cur];
  return LBM_OK;
}

int lbm_init_equilibrium(lbm_t *h, const float *rho, const float *u) {
  LBM_REQUIRE_ALIGNED(aligned(rho, kAlignField) && aligned(u, kAlignField));
  int rc = check_bound(h);
  if (rc) return rc;
  StepArgs a = make_args(h, nullptr, h->f[h->cur]);
  cudaError_t e = lbm::launch_init(h->storage, a, rho, u, h->bx, h->by, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "init kernel launch");
  return LBM_OK;
}

int lbm_step(lbm_t *h, int n) {
  int rc = check_bound(h);
  if (rc) return rc;
  if (n < 0) return fail(LBM_EINVAL, "n must be >= 0");
  return do_steps(h, n, nullptr, nullptr);
}

int lbm_step_moments(lbm_t *h, int n, float *rho, float *u) {
  LBM_REQUIRE_ALIGNED(aligned(rho, kAlignField) && aligned(u, kAlignField));
  int rc = check_bound(h);
  if (rc) return rc;
  if (n < 1 || !rho || !u) return fail(LBM_EINVAL, "need n >= 1 and rho, u");
  return do_steps(h, n, rho, u);
}

int lbm_step_to(lbm_t *h, const void *f_in, void *f_out) {
  LBM_REQUIRE_ALIGNED(aligned(f_in, kAlignF) && aligned(f_out, kAlignF));
  int rc = check_bound(h);
  if (rc) return rc;
  if (!f_in || !f_out || f_in == f_out) return fail(LBM_EINVAL, "bad buffers");
  StepArgs a = make_args(h, f_in, f_out);
  cudaError_t e = launch_one_step(h, false, a);
  if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
  return LBM_OK;
}

int lbm_step_to_moments(lbm_t *h, const void *f_in, void *f_out, float *rho, float *u) {
  LBM_REQUIRE_ALIGNED(aligned(f_in, kAlignF) && aligned(f_out, kAlignF) &&
                      aligned(rho, kAlignField) && aligned(u, kAlignField));
  int rc = check_bound(h);
  if (rc) return rc;
  if (!f_in || !f_out || f_in == f_out || !rho || !u) return fail(LBM_EINVAL, "bad buffers");
  StepArgs a = make_args(h, f_in, f_out);
  a.rho = rho;
  a.u = u;
  cudaError_t e = launch_one_step(h, true, a);
  if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
  return LBM_OK;
}

int lbm_step_push(lbm_t *h, const void *g_in, void *g_out) {
  LBM_REQUIRE_ALIGNED(aligned(g_in, kAlignF) && aligned(g_out, kAlignF));
  int rc = check_bound(h);
  if (rc) return rc;
  if (!g_in || !g_out || g_in == g_out) return fail(LBM_EINVAL, "bad buffers");
  if (onsite(h)) return fail(LBM_EINVAL, "the push iteration supports halfway walls only");
  StepArgs a = make_args(h, g_in, g_out);
  cudaError_t e = lbm::launch_step_push(h->storage, a, h->bx, h->by, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "push step launch");
  return LBM_OK;
}

int lbm_stream(lbm_t *h, const void *f_in, void *f_out, int form) {
  LBM_REQUIRE_ALIGNED(aligned(f_in, kAlignF) && aligned(f_out, kAlignF));
  int rc = check_bound(h);
  if (rc) return rc;
  if (!f_in || !f_out || f_in == f_out) return fail(LBM_EINVAL, "bad buffers");
  if (form < LBM_STREAM_PULL || form > LBM_STREAM_PULL_L2) return fail(LBM_EINVAL, "bad form");
  if (onsite(h)) return fail(LBM_EINVAL, "streaming alone supports halfway walls only");
  StepArgs a = make_args(h, f_in, f_out);
  cudaError_t e = lbm::launch_stream(h->storage, a, form, h->bx, h->by, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream kernel launch");
  return LBM_OK;
}

int lbm_moments(lbm_t *h, float *rho, float *u, double *mass) {
  LBM_REQUIRE_ALIGNED(aligned(rho, kAlignField) && aligned(u, kAlignField));
  int rc = check_bound(h);
  if (rc) return rc;
  StepArgs a = make_args(h, nullptr, nullptr);
  if (mass) LBM_CUDA(cudaMemsetAsync(h->scr.err, 0, sizeof(int), h->stream), "memset");
  cudaError_t e = lbm::launch_moments(h->storage, a, h->f[h->cur], rho, u,
                                      mass ? &h->scr : nullptr, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "moments kernel launch");
  if (!mass) return LBM_OK;
  e = lbm::launch_finalize_sum(h->scr, lbm::moments_blocks(a.cells),
                               (double)a.cells, h->scr.sum, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "finalize kernel launch");
  double m = 0.0;
  int err = 0;
  LBM_CUDA(cudaMemcpyAsync(&m, h->scr.sum, sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream), "mass copy");
  LBM_CUDA(cudaMemcpyAsync(&err, h->scr.err, sizeof(int), cudaMemcpyDeviceToHost,
                           h->stream), "error word copy");
  LBM_CUDA(cudaStreamSynchronize(h->stream), "stream sync");
  *mass = m;
  if (err & lbm::kErrNonFinite) return fail(LBM_ENONFINITE, "non-finite density");
  return LBM_OK;
}

int lbm_sync(lbm_t *h) {
  int rc = check_bound(h);
  if (rc) return rc;
  int err = 0;
  LBM_CUDA(cudaMemcpyAsync(&err, h->scr.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream),
           "error word copy");
  LBM_CUDA(cudaStreamSynchronize(h->stream), "stream sync");
  LBM_CUDA(cudaGetLastError(), "pending error");
  if (err & lbm::kErrTimeout) {
    LBM_CUDA(cudaMemset(h->scr.err, 0, sizeof(int)), "error word clear");
    return fail(LBM_ETIMEOUT, "a bounded wait in a step kernel gave up");
  }
  return LBM_OK;
}

int lbm_get_f(lbm_t *h, double *host_f) {
  int rc = check_bound(h);
  if (rc) return rc;
  return lbm_get_buffer(h, h->f[h->cur], host_f);
}

int lbm_get_buffer(lbm_t *h, const void *buf, double *host_f) {
  int rc = check_bound(h);
  if (rc) return rc;
  if (!host_f || !buf) return fail(LBM_EINVAL, "NULL buffer");
  const size_t bytes = (size_t)lbm::Q * h->plane * h->elem_bytes;
  void *stage = malloc(bytes);
  if (!stage) return fail(LBM_ENOMEM, "host staging allocation failed");
  cudaError_t e = cudaMemcpyAsync(stage, buf, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    free(stage);
    return cuda_fail(e, "state copy to host");
  }
  const size_t cells = (size_t)h->nx * h->ny * h->nz;
  for (int i = 0; i < lbm::Q; ++i) {
    const double w = lbm::weight_d(i);
    for (int z = 0; z < h->nz; ++z)
      for (int y = 0; y < h->ny; ++y)
        for (int x = 0; x < h->nx; ++x) {
          const size_t k = i * h->plane + ((size_t)z * h->ny + y) * h->pitch + x;
          const size_t o = i * cells + ((size_t)z * h->ny + y) * h->nx + x;
          host_f[o] = (double)host_to_float(stage, k, h->storage) + w;
        }
  }
  free(stage);
  return LBM_OK;
}

int lbm_set_f(lbm_t *h, const double *host_f) {
  int rc = check_bound(h);
  if (rc) return rc;
  if (!host_f) return fail(LBM_EINVAL, "host_f is NULL");
  const size_t bytes = (size_t)lbm::Q * h->plane * h->elem_bytes;
  void *stage = calloc(1, bytes);
  if (!stage) return fail(LBM_ENOMEM, "host staging allocation failed");
  const size_t cells = (size_t)h->nx * h->ny * h->nz;
  for (int i = 0; i < lbm::Q; ++i) {
    const double w = lbm::weight_d(i);
    for (int z = 0; z < h->nz; ++z)
      for (int y = 0; y < h->ny; ++y)
        for (int x = 0; x < h->nx; ++x) {
          const size_t k = i * h->plane + ((size_t)z * h->ny + y) * h->pitch + x;
          const size_t o = i * cells + ((size_t)z * h->ny + y) * h->nx + x;
          host_from_float(stage, k, h->storage, (float)(host_f[o] - w));
        }
  }
  cudaError_t e = cudaMemcpyAsync(h->f[h->cur], stage, bytes,
                                  cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  free(stage);
  if (e != cudaSuccess) return cuda_fail(e, "state copy to device");
  return LBM_OK;
}

int lbm_run_host(lbm_t *h, const float *u0_host, int n, float *rho_host,
                 float *u_host) {
  int rc = check_bound(h);
  if (rc) return rc;
  if (n < 1 || !rho_host || !u_host) return fail(LBM_EINVAL, "need n >= 1, rho, u");
  rc = ensure_pipeline(h);
  if (rc) return rc;
  const size_t cells = (size_t)h->nx * h->ny * h->nz;
  const size_t nxy = (size_t)h->nx * h->ny;
  const int S = h->nz < lbm_lattice::kMaxSlabs ? h->nz : lbm_lattice::kMaxSlabs;
  int zs[lbm_lattice::kMaxSlabs + 1];
  // Slabs 0..2 thin: the first outbound copy (slab 1) waits for them to be
  // copied in and initialised, and slab 0 is the last one out, so thin
  // leading slabs shorten the start and the tail of the pipeline.
  const int thin = S >= 8 ? h->nz / (4 * S) : 0;
  if (thin >= 1 && h->nz - 3 * thin >= S - 3) {
    for (int k = 0; k <= 3; ++k) zs[k] = k * thin;
    for (int k = 4; k <= S; ++k)
      zs[k] = 3 * thin + (int)((long long)(k - 3) * (h->nz - 3 * thin) / (S - 3));
  } else {
    for (int k = 0; k <= S; ++k) zs[k] = (int)((long long)k * h->nz / S);
  }
  float *u0d = h->stage;            // 3 * cells
  float *rd = h->stage + 3 * cells;  // cells
  float *ud = rd + cells;            // 3 * cells
  // the copy streams start after the work already queued on the handle's stream
  LBM_CUDA(cudaEventRecord(h->ev_start, h->stream), "event record");
  LBM_CUDA(cudaStreamWaitEvent(h->copy_in, h->ev_start, 0), "stream wait");
  LBM_CUDA(cudaStreamWaitEvent(h->copy_out, h->ev_start, 0), "stream wait");
  auto copy_in_and_init = [&](int k) -> int {
    if (u0_host) {
      const size_t off = (size_t)zs[k] * nxy, len = (size_t)(zs[k + 1] - zs[k]) * nxy;
      for (int c = 0; c < 3; ++c)
        LBM_CUDA(cudaMemcpyAsync(u0d + c * cells + off, u0_host + c * cells + off,
                                 len * sizeof(float), cudaMemcpyHostToDevice, h->copy_in),
                 "u0 copy");
    }
    LBM_CUDA(cudaEventRecord(h->ev_in[k], h->copy_in), "event record");
    LBM_CUDA(cudaStreamWaitEvent(h->stream, h->ev_in[k], 0), "stream wait");
    StepArgs a = make_args(h, nullptr, h->f[h->cur]);
    a.z0 = zs[k];
    a.zn = zs[k + 1] - zs[k];
    cudaError_t e = lbm::launch_init(h->storage, a, nullptr, u0_host ? u0d : nullptr, h->bx,
                                     h->by, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "init kernel launch");
    return LBM_OK;
  };
  auto last_step_and_copy_out = [&](int k) -> int {
    StepArgs a = make_args(h, h->f[h->cur], h->f[1 - h->cur]);
    a.z0 = zs[k];
    a.zn = zs[k + 1] - zs[k];
    cudaError_t e = lbm::launch_step(h->storage, false, a, h->bx, h->by, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
    StepArgs m = make_args(h, nullptr, nullptr);
    m.z0 = a.z0;
    m.zn = a.zn;
    e = lbm::launch_moments(h->storage, m, h->f[1 - h->cur], rd, ud, nullptr, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "moments kernel launch");
    LBM_CUDA(cudaEventRecord(h->ev_out[k], h->stream), "event record");
    LBM_CUDA(cudaStreamWaitEvent(h->copy_out, h->ev_out[k], 0), "stream wait");
    const size_t off = (size_t)zs[k] * nxy, len = (size_t)(zs[k + 1] - zs[k]) * nxy;
    LBM_CUDA(cudaMemcpyAsync(rho_host + off, rd + off, len * sizeof(float),
                             cudaMemcpyDeviceToHost, h->copy_out), "rho copy");
    for (int c = 0; c < 3; ++c)
      LBM_CUDA(cudaMemcpyAsync(u_host + c * cells + off, ud + c * cells + off,
                               len * sizeof(float), cudaMemcpyDeviceToHost, h->copy_out),
               "u copy");
    return LBM_OK;
  };
  if (n == 1 && S >= 3) {
    // One step: slab k of the step needs slabs k - 1 .. k + 1 initialised
    // (periodically), so slabs 1 .. S-2 step as soon as their upper
    // neighbour has arrived, and their results leave while later slabs are
    // still coming in; slabs S-1 and 0 (which wrap around) go last.
    rc = copy_in_and_init(0);
    if (rc) return rc;
    rc = copy_in_and_init(1);
    if (rc) return rc;
    for (int k = 1; k <= S - 2; ++k) {
      rc = copy_in_and_init(k + 1);
      if (rc) return rc;
      rc = last_step_and_copy_out(k);
      if (rc) return rc;
    }
    rc = last_step_and_copy_out(S - 1);
    if (rc) return rc;
    rc = last_step_and_copy_out(0);
    if (rc) return rc;
  } else {
    // 1. copy u0 in by z slabs; each slab is initialised as soon as it arrives
    for (int k = 0; k < S; ++k) {
      rc = copy_in_and_init(k);
      if (rc) return rc;
    }
    // 2. all but the last step over the whole lattice
    rc = do_steps(h, n - 1, nullptr, nullptr);
    if (rc) return rc;
    // 3. the last step and the moments by z slabs; each slab is copied out as
    //    soon as its moments are done
    for (int k = 0; k < S; ++k) {
      rc = last_step_and_copy_out(k);
      if (rc) return rc;
    }
  }
  h->cur ^= 1;
  LBM_CUDA(cudaEventRecord(h->ev_done, h->copy_out), "event record");
  LBM_CUDA(cudaStreamWaitEvent(h->stream, h->ev_done, 0), "stream wait");
  LBM_CUDA(cudaStreamSynchronize(h->stream), "stream sync");
  return LBM_OK;
}

// ---- discrete adjoint ---------------------------------------------------

int lbm_adjoint_seed(lbm_t *h, const void *f_T, const float *u_target,
                     float *lambda_T, float *grad_force, double *loss) {
  LBM_REQUIRE_ALIGNED(aligned(f_T, kAlignF) && aligned(u_target, kAlignField) &&
                      aligned(lambda_T, kAlignField) && aligned(grad_force, kAlignField) &&
                      aligned(loss, kAlignF64));
  int rc = check_bound(h);
  if (rc) return rc;
  if (h->storage != lbm::kF32) return fail(LBM_EINVAL, "adjoint needs FP32 storage");
  if (!f_T || !u_target || !lambda_T) return fail(LBM_EINVAL, "NULL buffer");
  StepArgs g = make_args(h, f_T, nullptr);
  cudaError_t e = lbm::launch_adjoint_seed(g, u_target, lambda_T, grad_force,
                                           loss ? h->scr.partials : nullptr, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint seed launch");
  if (loss) {
    e = lbm::launch_finalize_sum(h->scr, lbm::moments_blocks(g.cells), 0.0, loss, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "loss reduction launch");
  }
  return LBM_OK;
}

int lbm_adjoint_step(lbm_t *h, const void *f_n, const float *lambda_in,
                     float *lambda_out, float *grad_force) {
  LBM_REQUIRE_ALIGNED(aligned(f_n, kAlignF) && aligned(lambda_in, kAlignField) &&
                      aligned(lambda_out, kAlignField) && aligned(grad_force, kAlignField));
  int rc = check_bound(h);
  if (rc) return rc;
  if (h->storage != lbm::kF32) return fail(LBM_EINVAL, "adjoint needs FP32 storage");
  if (!f_n || !lambda_in || !lambda_out || lambda_in == lambda_out)
    return fail(LBM_EINVAL, "bad buffers");
  if (onsite(h)) return fail(LBM_EINVAL, "the adjoint supports halfway walls only");
  StepArgs g = make_args(h, f_n, nullptr);
  // The adjoint issues ~1.7x the forward's instructions per node: the branch
  // form (fewer instructions off the walls) wins from 64-node rows on
  // (measured at 128^3 and 256^3), and
  // 64 x 2 blocks measured best for both periodic and walled lattices.
  g.wall_select = h->wall_mode == LBM_WALLS_SELECT ||
                  (h->wall_mode == LBM_WALLS_AUTO && h->nx < 64);
  const int abx = h->nx <= 32 ? 32 : 64;
  cudaError_t e = lbm::launch_adjoint_step(g, lambda_in, lambda_out, grad_force, abx,
                                           128 / abx, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint step launch");
  return LBM_OK;
}

int lbm_adjoint_step_moments(lbm_t *h, const float *rho_n, const float *u_n,
                             const float *lambda_in, float *lambda_out, float *grad_force) {
  LBM_REQUIRE_ALIGNED(aligned(rho_n, kAlignField) && aligned(u_n, kAlignField) &&
                      aligned(lambda_in, kAlignField) && aligned(lambda_out, kAlignField) &&
                      aligned(grad_force, kAlignField));
  int rc = check_bound(h);
  if (rc) return rc;
  if (h->storage != lbm::kF32) return fail(LBM_EINVAL, "adjoint needs FP32 storage");
  if (!rho_n || !u_n || !lambda_in || !lambda_out || lambda_in == lambda_out)
    return fail(LBM_EINVAL, "bad buffers");
  if (onsite(h)) return fail(LBM_EINVAL, "the adjoint supports halfway walls only");
  StepArgs g = make_args(h, nullptr, nullptr);
  g.wall_select = h->wall_mode == LBM_WALLS_SELECT ||
                  (h->wall_mode == LBM_WALLS_AUTO && h->nx < 64);
  const int abx = h->nx <= 32 ? 32 : 64;
  cudaError_t e = lbm::launch_adjoint_step_mom(g, rho_n, u_n, lambda_in, lambda_out, grad_force,
                                               abx, 128 / abx, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint step launch");
  return LBM_OK;
}

int lbm_adjoint_u0(lbm_t *h, const float *lambda0, const float *u0,
                   float *grad_u0) {
  LBM_REQUIRE_ALIGNED(aligned(lambda0, kAlignField) && aligned(u0, kAlignField) &&
                      aligned(grad_u0, kAlignField));
  int rc = check_bound(h);
  if (rc) return rc;
  if (h->storage != lbm::kF32) return fail(LBM_EINVAL, "adjoint needs FP32 storage");
  if (!lambda0 || !grad_u0) return fail(LBM_EINVAL, "NULL buffer");
  StepArgs g = make_args(h, nullptr, nullptr);
  cudaError_t e = lbm::launch_adjoint_u0(g, lambda0, u0, grad_u0, h->bx, h->by, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint u0 launch");
  return LBM_OK;
}

int lbm_check_status(unsigned long long *refused, unsigned long long *first_addr,
                     unsigned int *first_bytes, unsigned int *first_kind) {
#ifdef LBM_CHECK
  lbm::CheckRecord r = {};
  lbm::CheckRecord *d = lbm::check_record();
  if (!d) return fail(LBM_ENOMEM, "check record allocation failed");
  LBM_CUDA(cudaDeviceSynchronize(), "check status sync");
  LBM_CUDA(cudaMemcpy(&r, d, sizeof(r), cudaMemcpyDeviceToHost), "check status copy");
  if (refused) *refused = r.count;
  if (first_addr) *first_addr = r.first;
  if (first_bytes) *first_bytes = r.first_bytes;
  if (first_kind) *first_kind = r.first_kind;
  return LBM_OK;
#else
  (void)refused, (void)first_addr, (void)first_bytes, (void)first_kind;
  return fail(LBM_ENOTSUP, "built without LBM_CHECK");
#endif
}

int lbm_check_reset(void) {
#ifdef LBM_CHECK
  lbm::CheckRecord *d = lbm::check_record();
  if (!d) return fail(LBM_ENOMEM, "check record allocation failed");
  LBM_CUDA(cudaDeviceSynchronize(), "check reset sync");
  LBM_CUDA(cudaMemset(d, 0, sizeof(lbm::CheckRecord)), "check reset");
  LBM_CUDA(cudaDeviceSynchronize(), "check reset sync");
  return LBM_OK;
#else
  return fail(LBM_ENOTSUP, "built without LBM_CHECK");
#endif
}

int lbm_check_narrow(size_t bytes) {
#ifdef LBM_CHECK
  lbm::g_check_narrow.store(bytes);
  return LBM_OK;
#else
  (void)bytes;
  return fail(LBM_ENOTSUP, "built without LBM_CHECK");
#endif
}

}  // extern "C"
