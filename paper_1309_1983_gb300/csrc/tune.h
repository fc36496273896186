// tune.h - helpers shared by the lattice and batch autotuners: the text
// cache of tuned launch shapes and event timing on a stream.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "internal.h"

namespace lbm {

// "<GPU name>/sm<count>" of a device (spaces replaced by '_').
std::string device_key(int device);
// Shape (a, b) and time stored for `key` in the cache file; false on a miss
// or when path is null or unreadable.
bool tune_cache_lookup(const char *path, const std::string &key, int *a, int *b, float *ms);
// Replace or add the line for `key`; 0 on success (or when path is null).
int tune_cache_store(const char *path, const std::string &key, int a, int b, float ms);

// Mean time in ms of one call of `run` (which returns an LBM status) on
// stream s, timed with CUDA events over `reps` calls after one untimed call.
template <typename F>
int time_calls(cudaStream_t s, int reps, F run, float *ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return set_cuda_error(e, "autotune event");
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_cuda_error(e, "autotune event");
  }
  int rc = run();
  if (!rc) e = cudaEventRecord(e0, s);
  for (int k = 0; !rc && e == cudaSuccess && k < reps; ++k) rc = run();
  if (!rc && e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (!rc && e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (!rc && e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (e != cudaSuccess) return set_cuda_error(e, "autotune timing");
  *ms = t / reps;
  return 0;
}

}  // namespace lbm
