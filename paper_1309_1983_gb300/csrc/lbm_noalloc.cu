// lbm_noalloc.cu - lbm_moments_noalloc: the moment kernel with its FP64 mass
// reduction, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code whose device memory is owned in
// full by another allocator (a framework's caching pool, or an arena sized
// once at start-up), and latency-critical loops in which cudaMalloc/cudaFree
// may synchronise the device. lbm_moments needs a bound handle, and binding
// allocates the handle's scratch with cudaMalloc. This entry point takes the
// distribution buffer and the outputs as plain pointers and keeps its
// reduction scratch in the file-scope array below instead.
//
// The array exists once per GPU (it is created when the library's device code
// is loaded on that GPU) and stays until the process exits. Every call on a
// device shares it, so calls whose work overlaps on the GPU (different
// streams, or host threads racing) race on it; order them on one stream. The
// array keeps the last call's contents: the per-block partial sums are fully
// rewritten by each call before they are read. The moment kernel also sets a
// non-finite flag in the word after them; nothing reads that word here (the
// call does no non-finite check: a non-finite density makes the FP64 mass
// non-finite), so it is never cleared.
//
// In host code the array's name is only a stand-in for the device symbol: its
// device address is looked up with cudaGetSymbolAddress, once per CUDA
// context (a context created after cudaDeviceReset, or another context made
// current, gets its own lookup), and only that address is passed to kernels.
#include <string.h>

#include <mutex>

#include "d3q19.cuh"
#include "internal.h"

namespace {

// kReduceBlocks FP64 partial sums, then one int flag word (in the next
// double slot), padded to a multiple of 256 bytes: 9.75 KiB per GPU.
constexpr int kNoallocSlots = lbm::kReduceBlocks + 32;
static_assert(kNoallocSlots >= lbm::kReduceBlocks + 1,
              "partials (at most kReduceBlocks: moments_blocks clamps to it) + flag word");
static __device__ __align__(256) double g_noalloc_scratch[kNoallocSlots];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
struct ScratchAddr {
  unsigned long long ctx_id;  // cuCtxGetId of the context the address belongs to
  double *addr;
};
ScratchAddr g_scratch_addr[kMaxDevices] = {};

// Context queries through the runtime's driver entry points (no link-time
// dependency on libcuda).
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
bool g_entry_points_loaded = false;

// Unique id of the current context, 0 if there is none or it cannot be
// queried. Called with g_setup_mutex held.
unsigned long long current_context_id() {
  if (!g_entry_points_loaded) {
    g_entry_points_loaded = true;
    void *fa = nullptr, *fb = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fa, 12000, cudaEnableDefault,
                                         &qa) == cudaSuccess &&
        qa == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &fb, 12000, cudaEnableDefault, &qb) ==
            cudaSuccess &&
        qb == cudaDriverEntryPointSuccess) {
      g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(fa);
      g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(fb);
    }
    cudaGetLastError();
  }
  if (!g_ctx_get_current || !g_ctx_get_id) return 0;
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_get_current(&ctx) != 0 || !ctx) return 0;
  if (g_ctx_get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the array in the current context of device `dev`; the
// host-side symbol is only a stand-in and must never be handed to a kernel.
int scratch_address(int dev, double **out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  ScratchAddr &slot = g_scratch_addr[dev];
  const unsigned long long id = current_context_id();
  if (!slot.addr || id == 0 || slot.ctx_id != id) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return lbm::set_cuda_error(e, "cudaGetSymbolAddress");
    slot.addr = static_cast<double *>(p);
    slot.ctx_id = current_context_id();  // the lookup makes the context current
  }
  *out = slot.addr;
  return LBM_OK;
}

}  // namespace

static bool aligned_ptr(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

extern "C" int lbm_moments_noalloc(const void *f, int nx, int ny, int nz, uint32_t flags,
                                   const float *force, float *rho, float *u, double *mass,
                                   void *stream) {
  if (!f) return lbm::set_error(LBM_EINVAL, "f is NULL");
  if (!aligned_ptr(f, 256) || !aligned_ptr(force, 4) || !aligned_ptr(rho, 4) ||
      !aligned_ptr(u, 4) || !aligned_ptr(mass, 8))
    return lbm::set_error(LBM_EINVAL, "misaligned device buffer");
#ifdef LBM_CHECK
  if (!lbm::check_record()) return lbm::set_error(LBM_ENOMEM, "check record allocation failed");
#endif
  if (nx < 1 || ny < 1 || nz < 1) return lbm::set_error(LBM_EINVAL, "sizes must be >= 1");
  const uint32_t st = flags & (LBM_STORE_F16 | LBM_STORE_BF16);
  if (st == (LBM_STORE_F16 | LBM_STORE_BF16))
    return lbm::set_error(LBM_EINVAL, "more than one storage type");
  if ((flags & LBM_FORCE) && !force) return lbm::set_error(LBM_EINVAL, "LBM_FORCE needs force");
  const int storage = st == LBM_STORE_F16 ? lbm::kF16 : st == LBM_STORE_BF16 ? lbm::kBF16
                                                                             : lbm::kF32;
  const int align = storage == lbm::kF32 ? 8 : 16;
  const long long pitch = ((long long)nx + align - 1) / align * align;
  const long long plane = pitch * ny * (long long)nz;
  if (plane >= (1ll << 31))
    return lbm::set_error(LBM_ERANGE,
                          "lbm_moments_noalloc: nz * ny * pitch must be < 2^31 nodes");
  const uint32_t cells = (uint32_t)((long long)nx * ny * nz);
  const int nparts = lbm::moments_blocks(cells);  // <= kReduceBlocks by construction
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return lbm::set_cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return lbm::set_error(LBM_ERANGE, "device ordinal >= 64");
  double *scratch = nullptr;
  int rc = scratch_address(dev, &scratch);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  lbm::StepArgs a;
  memset(&a, 0, sizeof(a));
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.pitch = (int)pitch;
  a.plane = (uint32_t)plane;
  a.cells = cells;
  a.z0 = 0;
  a.zn = nz;
  a.force = (flags & LBM_FORCE) ? force : nullptr;

  lbm::Scratch scr;
  scr.partials = mass ? scratch : nullptr;
  scr.sum = nullptr;
  scr.err = reinterpret_cast<int *>(scratch + lbm::kReduceBlocks);
  scr.nblocks = lbm::kReduceBlocks;
  e = lbm::launch_moments(storage, a, f, rho, u, mass ? &scr : nullptr, s);
  if (e != cudaSuccess) return lbm::set_cuda_error(e, "moments kernel launch");
  if (mass) {
    e = lbm::launch_finalize_sum(scr, nparts, (double)cells, mass, s);
    if (e != cudaSuccess) return lbm::set_cuda_error(e, "finalize kernel launch");
  }
  return LBM_OK;
}
