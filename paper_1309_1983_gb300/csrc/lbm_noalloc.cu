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
// is loaded on that GPU) and stays until the process exits. Every call on a device
// shares it, so calls whose work overlaps on the GPU (different streams,
// or host threads racing) race on it; order them on one stream. The array
// keeps the last call's contents: the per-block partial sums are fully
// rewritten by each call before they are read, and the error word is cleared
// at the start of each call.
#include <string.h>

#include <mutex>

#include "d3q19.cuh"
#include "internal.h"

namespace {

// kReduceBlocks FP64 partial sums, then one int error word (in the next
// double slot), padded to a multiple of 256 bytes: 9.75 KiB per GPU.
constexpr int kNoallocSlots = lbm::kReduceBlocks + 32;
static __device__ __align__(256) double g_noalloc_scratch[kNoallocSlots];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the array on the current device; the host-side symbol is
// only a stand-in and must never be handed to a kernel.
int scratch_address(int dev, double **out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return lbm::set_cuda_error(e, "cudaGetSymbolAddress");
    g_scratch_addr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_addr[dev];
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_moments_noalloc(const void *f, int nx, int ny, int nz, uint32_t flags,
                                   const float *force, float *rho, float *u, double *mass,
                                   void *stream) {
  if (!f) return lbm::set_error(LBM_EINVAL, "f is NULL");
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
  const int nparts = lbm::moments_blocks(cells);
  if (nparts > lbm::kReduceBlocks)
    return lbm::set_error(LBM_ERANGE, "lbm_moments_noalloc: reduction exceeds static scratch");
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
  if (mass) {
    e = cudaMemsetAsync(scr.err, 0, sizeof(int), s);
    if (e != cudaSuccess) return lbm::set_cuda_error(e, "error word clear");
  }
  e = lbm::launch_moments(storage, a, f, rho, u, mass ? &scr : nullptr, s);
  if (e != cudaSuccess) return lbm::set_cuda_error(e, "moments kernel launch");
  if (mass) {
    e = lbm::launch_finalize_sum(scr, nparts, (double)cells, mass, s);
    if (e != cudaSuccess) return lbm::set_cuda_error(e, "finalize kernel launch");
  }
  return LBM_OK;
}
