// internal.h - handle layout and kernel launchers shared by the translation
// units of liblbm (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "check.cuh"
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
  int z0, zn;          // planes [z0, z0 + zn) processed by a launch (0, nz: all)
  int wall_select;     // 1: per-direction address select, 0: branch on wall nodes
  int onsite;          // 1: walled axes use the on-site velocity rule (onsite.cuh)
  int onsite_lid;      // 1: the top plane's interior moves with lid[] (on-site)
  float lid[3];        // lid velocity u_w
};

// Buffers of a launch over StepArgs, for the LBM_CHECK tables (check.cuh;
// not evaluated in the normal build): f in (read) and f out (write) of
// `elem` bytes per value, the force field (read), the moment outputs
// (write). 19 directions per node.
#define LBM_STEP_RANGES(a, elem)                                          \
  ::lbm::chk_r((a).fin, 19 * (size_t)(a).plane * (elem)),                 \
      ::lbm::chk_w((a).fout, 19 * (size_t)(a).plane * (elem)),            \
      ::lbm::chk_r((a).force, 3 * (size_t)(a).cells * sizeof(float)),     \
      ::lbm::chk_w((a).rho, (size_t)(a).cells * sizeof(float)),           \
      ::lbm::chk_w((a).u, 3 * (size_t)(a).cells * sizeof(float))

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
constexpr int elem_bytes_of(int storage) { return storage == kF32 ? 4 : 2; }

cudaError_t launch_step(int storage, bool moments, const StepArgs &a, int bx,
                        int by, cudaStream_t s);
// 16-bit storage, two x-adjacent nodes per thread (bxp pairs per block row,
// a multiple of 32).
// 16-bit storage, two x-adjacent nodes per thread without exchange between
// threads (bxp pairs per block row, `by` rows).
cudaError_t launch_step_x2(int storage, bool moments, const StepArgs &a, int bxp, int by,
                           cudaStream_t s);
cudaError_t launch_step_pair16(int storage, bool moments, const StepArgs &a, int bxp, int by,
                               cudaStream_t s);
// Four x-adjacent nodes per thread (bxq groups of four per block row, `by`
// rows); periodic axes and halfway walls.
cudaError_t launch_step_x4(int storage, bool moments, const StepArgs &a, int bxq, int by,
                           cudaStream_t s);
// Bulk-copy (TMA) staged step, persistent over tiles; variant 0: 2-row tiles,
// variant 1: 1-row tiles with a deeper pipeline. err receives kErrTimeout if
// a bounded mbarrier wait gave up.
cudaError_t launch_step_bulk(int storage, const StepArgs &a, int *err, int variant, int sms,
                             cudaStream_t s);
// Push iteration (Alg. 2) on post-streaming states, and streaming alone
// (form 0 gather, 1 scatter, 2 unshifted copy).
cudaError_t launch_step_push(int storage, const StepArgs &a, int bx, int by, cudaStream_t s);
cudaError_t launch_stream(int storage, const StepArgs &a, int form, int bx, int by,
                          cudaStream_t s);
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

cudaError_t launch_adjoint_step(const StepArgs &g, const float *lam_in,
                                float *lam_out, float *grad_force, int bx,
                                int by, cudaStream_t s);
// The reverse step from the moments rho^n, u^n of the forward collision
// (dense FP32 fields) instead of the state f^n.
cudaError_t launch_adjoint_step_mom(const StepArgs &g, const float *rho_n, const float *u_n,
                                    const float *lam_in, float *lam_out, float *grad_force,
                                    int bx, int by, cudaStream_t s);
cudaError_t launch_adjoint_seed(const StepArgs &g, const float *u_target,
                                float *lam_out, float *grad_force,
                                double *partials, cudaStream_t s);
cudaError_t launch_adjoint_u0(const StepArgs &g, const float *lam0,
                              const float *u0, float *grad, int bx, int by,
                              cudaStream_t s);

// ---- batched lattices -------------------------------------------------------

struct BatchDom {
  int nx, ny, nz, pitch;
  uint32_t plane, cells;
  uint64_t foff;       // first FP32 element of the domain's f region
  uint32_t coff;       // first dense node of the domain in field buffers
  uint32_t walls;      // LBM_WALL_* bits
  uint64_t m_nx, m_nxy;  // ceil(2^42 / nx), ceil(2^42 / (nx ny))
  float omega, kf;
  float lidc[19];
};

// Steps of one persistent batched launch (lbm_batch_run /
// lbm_batch_adjoint_run): per step its input and output f buffers and,
// optionally, the dense rho / u fields the step's collision writes.
constexpr int kMaxSeqSteps = 64;
struct BatchFwdSeq {
  int n;
  const float *fin[kMaxSeqSteps];
  float *fout[kMaxSeqSteps];
  float *rho[kMaxSeqSteps];
  float *u[kMaxSeqSteps];
};
// Reverse steps from stored moments: step s reads lam[s & 1] and writes
// lam[(s & 1) ^ 1], with the moments of the forward step it reverses.
struct BatchAdjSeq {
  int n;
  float *lam[2];
  float *gF;
  const float *rho[kMaxSeqSteps];
  const float *u[kMaxSeqSteps];
};

struct BatchArgs {
  float *f[2];
  const BatchDom *doms;
  const int2 *tiles;  // {domain, first dense node}
  int ntiles, nsteps, parity0, walls_any;
  int ndom;
  unsigned *bar_count, *bar_gen;
  int *err;
  unsigned expected;  // blocks that must reach each grid barrier
  unsigned long long timeout_ns;
#ifdef LBM_CHECK
  uint64_t f_elems;   // FP32 values per f (or lambda) buffer of the batch
  uint32_t cells;     // dense nodes of all domains (field buffers: 1 or 3 per node)
#endif
};

// Buffers of a batched launch for the LBM_CHECK tables: the domain and tile
// tables (read), the barrier words and the error word (read-write); the f
// buffers are listed by each launcher with the permission it needs.
#define LBM_BATCH_RANGES(a)                                                  \
  ::lbm::chk_r((a).doms, (size_t)(a).ndom * sizeof(::lbm::BatchDom)),        \
      ::lbm::chk_r((a).tiles, (size_t)(a).ntiles * sizeof(int2)),            \
      ::lbm::chk_rw((a).bar_count, sizeof(unsigned)),                        \
      ::lbm::chk_rw((a).bar_gen, sizeof(unsigned)), ::lbm::chk_rw((a).err, sizeof(int))
#define LBM_BATCH_F(a) ((size_t)(a).f_elems * sizeof(float))
#define LBM_BATCH_FIELD(a, comps) ((size_t)(a).cells * (comps) * sizeof(float))

// Relaxation rate omega passed to every kernel for a relaxation time tau:
// the FP32 value within 2^-22 (relative) of 1/tau for which omega * (1/12)
// is exactly omega/12 in FP32 and 12 times that is exactly omega (the
// momentum-exact coefficients of collide() in d3q19.cuh).
float relaxation_rate(float tau);

// Record a failure for lbm_last_error() (thread-local) and return code.
int set_error(int code, const char *what);
int set_cuda_error(cudaError_t e, const char *where);

const void *batch_persistent_kernel(bool walls);
// Dynamic shared memory of the persistent kernel (the domain table).
size_t batch_persistent_smem(int ndom);
constexpr int kMaxBatchDomains = 256;  // table must fit in 48 KB of smem
cudaError_t launch_batch_persistent(const BatchArgs &a, int grid, int threads,
                                    cudaStream_t s);
cudaError_t launch_batch_step(const BatchArgs &a, const float *fin, float *fout,
                              int threads, cudaStream_t s);
// Persistent cooperative launches of a step sequence (grid barrier between
// steps); the kernels behind them for the occupancy query.
const void *batch_fwd_seq_kernel(bool walls, bool moments);
const void *batch_adj_seq_kernel(bool gradf);
cudaError_t launch_batch_fwd_seq(const BatchArgs &a, const BatchFwdSeq &q, int grid, int threads,
                                 cudaStream_t s);
cudaError_t launch_batch_adj_seq(const BatchArgs &a, const BatchAdjSeq &q, int grid, int threads,
                                 cudaStream_t s);
cudaError_t launch_batch_step_mom(const BatchArgs &a, const float *fin, float *fout, float *rho,
                                  float *u, int threads, cudaStream_t s);
cudaError_t launch_batch_adjoint_step_mom(const BatchArgs &a, const float *rho, const float *u,
                                          const float *lam_in, float *lam_out, float *gF,
                                          int threads, cudaStream_t s);
cudaError_t launch_batch_rest(const BatchArgs &a, float *f, int threads, cudaStream_t s);
cudaError_t launch_batch_moments(const BatchArgs &a, const float *f, float *rho, float *u,
                                 int threads, cudaStream_t s);

cudaError_t launch_batch_init_eq(const BatchArgs &a, float *f, const float *u0, int threads,
                                 cudaStream_t s);
cudaError_t launch_batch_adjoint_step(const BatchArgs &a, const float *fn, const float *lam_in,
                                      float *lam_out, float *gF, int threads, cudaStream_t s);
cudaError_t launch_batch_adjoint_seed(const BatchArgs &a, const float *fT, const float *ut,
                                      float *lam, float *gF, double *partials, int threads,
                                      cudaStream_t s);
cudaError_t launch_batch_adjoint_u0(const BatchArgs &a, const float *lam0, const float *u0,
                                    float *grad, int threads, cudaStream_t s);

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
  int kernel;    // LBM_KERNEL_NODE, LBM_KERNEL_PAIR or LBM_KERNEL_BULK*
  int wall_mode; // LBM_WALLS_AUTO / BRANCH / SELECT
  int sms;       // SM count of the bound device
  int pbx, pby;  // block shape of the pair kernel (pairs along x, rows)
  int device;
  lbm::Scratch scr;
  // lbm_run_host pipeline (created on first use, released by lbm_destroy)
  static constexpr int kMaxSlabs = 16;
  cudaStream_t copy_in, copy_out;
  cudaEvent_t ev_start, ev_in[kMaxSlabs], ev_out[kMaxSlabs], ev_done;
  float *stage;  // 3 cells (u0) + 4 cells (rho, u) FP32
  bool pipe_ready;
  // multi-step calls replay CUDA graphs of graph_steps launches (one graph
  // per starting buffer); any change of the launch configuration bumps
  // config_version and the graphs are captured again on next use
  int graph_steps;  // 0: plain launches only
  unsigned config_version;
  cudaStream_t gcap;
  cudaGraphExec_t gexec[2];
  unsigned gexec_version[2];
};
