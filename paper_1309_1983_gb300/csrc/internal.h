// internal.h - handle layout and kernel launchers shared by the translation
// units of liblbm (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "lbm.h"

namespace lbm {

// Per-launch arguments of the fused step kernel.
struct StepArgs {
  const void *fin;
  void *fout;
  const float *force;  // dense [3][cells] or nullptr
  float *rho;          // dense outputs of the fused-moments variant
  float *u;
  int nx, ny, nz, pitch;
  uint32_t plane;      // elements per direction plane (< 2^31)
  uint32_t cells;      // nx * ny * nz
  float omega, kf;     // 1/tau and 1 - 1/(2 tau)
  uint32_t walls;      // LBM_WALL_* bits
  float lidc[19];      // 6 w_i (e_i . u_w) for sources on z = nz (else 0)
};

struct Scratch {
  double *partials = nullptr;  // per-block FP64 partial sums
  double *sum = nullptr;       // final FP64 reduction result
  int *err = nullptr;          // device error word (bit flags)
  int nblocks = 0;             // capacity of partials
};

constexpr int kReduceBlocks = 1216;  // 152 SMs x 8
constexpr int kReduceThreads = 256;

enum : int { kErrNonFinite = 1, kErrTimeout = 2 };

// storage codes
enum : int { kF32 = 0, kF16 = 1, kBF16 = 2 };

cudaError_t launch_step(int storage, bool moments, const StepArgs &a, int bx,
                        int by, cudaStream_t s);
cudaError_t launch_init(int storage, const StepArgs &a, const float *rho0,
                        const float *u0, int bx, int by, cudaStream_t s);
// Moments of a stored state into dense rho/u (either may be null); when
// scratch is given, FP64 per-block partial sums of rho - 1 and the
// non-finite flag go there.
cudaError_t launch_moments(int storage, const StepArgs &a, const void *f,
                           float *rho, float *u, const Scratch *scr,
                           cudaStream_t s);
int moments_blocks(uint32_t cells);  // partial sums written by launch_moments
cudaError_t launch_finalize_sum(const Scratch &scr, int nparts, double offset,
                                double *out, cudaStream_t s);

}  // namespace lbm

struct lbm_lattice {
  int nx, ny, nz, pitch;
  uint32_t flags;
  int storage;  // lbm::kF32 / kF16 / kBF16
  int elem_bytes;
  size_t plane;
  float tau;
  float lid[3];
  void *f[2];
  int cur;
  const float *force;
  cudaStream_t stream;
  bool bound;
  int bx, by;
  int device;
  lbm::Scratch scr;
};
