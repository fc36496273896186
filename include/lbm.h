/*
 * lbm.h - C ABI of liblbm.so, a GB300 (sm_103a) D3Q19 BGK lattice Boltzmann
 * library: the fused pull stream-and-collide step with halfway bounce-back
 * walls and a moving lid, moment extraction, 16-bit shifted storage, a
 * discrete adjoint, and a batched persistent path for many small domains.
 *
 * Method (Mawson & Revell, "Memory transfer optimization for a lattice
 * Boltzmann solver on Kepler architecture nVidia GPUs"):
 *   - D3Q19 velocity set e_i, i = 0..18, in the order of Eq. 4; weights
 *     1/3, 1/18 (i = 1..6), 1/36 (i = 7..18); c_s^2 = 1/3 (text after Eq. 5).
 *   - BGK update, Eq. 3: f_i(x + e_i, t + 1) = f_i + (f_i^eq - f_i)/tau, with
 *     f^eq from Eq. 5 and rho, u from Eqs. 6-7, executed in the pull order of
 *     Alg. 3 (gather f_i(x - e_i), boundary rule, moments, equilibrium,
 *     collide, store at x) into a second copy of f, the two copies swapping
 *     every step (Sec. 4.1 and its footnote).
 *   - Optional per-cell body force F with the Guo forcing term:
 *     f*_i = g_i - (g_i - f^eq_i)/tau + (1 - 1/(2 tau)) w_i [3(e_i - u)
 *     + 9 (e_i.u) e_i].F, with u = (sum e_i g_i + F/2)/rho.
 *   - Boundary rule: an axis with LBM_WALL_* has halfway bounce-back walls
 *     at -1/2 and n - 1/2; other axes are periodic. When x - e_i lies outside
 *     a walled axis, g_i(x) = f_ibar(x) + 6 w_i (e_i . u_w), u_w = the lid
 *     velocity if that source lies on the plane z = nz and LBM_LID is set,
 *     else 0 (wall density 1). The paper validated with the cavity of Sec. 5
 *     (top wall moving along x, no slip elsewhere).
 *
 * Conventions shared by every call
 *   - Every call returns an int status: LBM_OK (0) or a negative LBM_E*
 *     code; lbm_strerror() names it. No exception or abort crosses the ABI.
 *   - Handles are opaque. Device buffers are owned by the caller (for
 *     example torch tensors passed as raw pointers); the library never frees
 *     them. A handle allocates a small device scratch area (error word,
 *     reduction partials) on first bind, staging of 28 bytes per node on the
 *     first lbm_run_host, and a private stream with CUDA graphs on the first
 *     multi-step call; lbm_destroy releases all of them.
 *   - Work is enqueued on the bound CUDA stream and is asynchronous, except
 *     where a call returns a host value (documented per call), which
 *     synchronises that stream.
 *   - Distribution buffers ("f buffers") use the layout reported by
 *     lbm_get_layout: Structure of Arrays [19][nz][ny][pitch] (Sec. 4.1),
 *     x fastest, each x row padded to `pitch` elements (32-byte aligned
 *     rows), element type FP32, FP16 or BF16 per LBM_STORE_*, holding the
 *     SHIFTED value f_i - w_i. Padding elements never enter the result (the
 *     two-node 16-bit kernels load and store the padding element of an odd
 *     row together with the row's last node).
 *   - Field buffers (rho, velocity u, force F, targets, gradients) are dense
 *     FP32 planes without padding: scalars [nz][ny][nx], vectors
 *     [3][nz][ny][nx] (component-major).
 *   - Adjoint buffers (lambda) are FP32 with the FP32 f-buffer layout (same
 *     pitch), unshifted.
 *   - Device buffers must be aligned for the kernels' accesses: f buffers to
 *     256 bytes, field and lambda buffers to 4 bytes, a device FP64 result
 *     (loss) to 8 bytes. A call given a misaligned buffer returns LBM_EINVAL
 *     before it checks anything else about the handle and launches nothing.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define LBM_OK 0
#define LBM_EINVAL (-1)     /* bad argument (sizes, tau <= 1/2, flags, NULL) */
#define LBM_ENOMEM (-2)     /* device or host allocation failed */
#define LBM_ECUDA (-3)      /* a CUDA runtime call or kernel launch failed */
#define LBM_ETIMEOUT (-4)   /* a bounded device-side wait gave up */
#define LBM_ENONFINITE (-5) /* a non-finite density was detected */
#define LBM_EUNBOUND (-6)   /* no buffers bound to the handle yet */
#define LBM_ERANGE (-7)     /* size above a documented maximum */
#define LBM_ENOTSUP (-8)    /* not in this build (the LBM_CHECK calls) */

/* ---- lbm_create flags ---- */
#define LBM_WALL_X 0x01u     /* bounce-back walls on both x faces */
#define LBM_WALL_Y 0x02u     /* ... y faces */
#define LBM_WALL_Z 0x04u     /* ... z faces */
#define LBM_LID 0x08u        /* the z = nz face moves (needs LBM_WALL_Z) */
#define LBM_STORE_F32 0x00u  /* f_i - w_i stored as FP32 (152 B per update) */
#define LBM_STORE_F16 0x10u  /* ... as FP16, round to nearest even (76 B) */
#define LBM_STORE_BF16 0x20u /* ... as BF16, round to nearest even (76 B) */
#define LBM_FORCE 0x40u      /* read a per-cell body force F each step */
#define LBM_ADJOINT 0x80u    /* the handle will run the adjoint (FP32 storage only) */
/* LBM_WALLS_ONSITE: walled axes use the on-site velocity condition the paper
 * used for its cavity (Sec. 5: Hecht & Harting's D3Q19 on-site conditions)
 * instead of halfway bounce-back. The walls then lie ON the first and last
 * node planes of each walled axis (at least 3 nodes long, else LBM_EINVAL).
 * Those nodes stream and collide like any other; after the pull, the
 * populations they would take from outside the lattice are rebuilt so that
 * the node's velocity (sum e g + F/2)/rho is exactly the wall velocity:
 * non-equilibrium bounce-back along the normal plus a transverse momentum
 * correction, the density fixed by mass on a face. On edges and corners the
 * density is the inner diagonal neighbour's (stored state of the previous
 * step) and opposite populations that both point along the walls share the
 * remaining mass equally. With LBM_LID the interior of the top plane
 * z = nz - 1 moves with the lid velocity; its edges and every other wall
 * node are at rest. Runs on LBM_KERNEL_X2 and LBM_KERNEL_NODE; the adjoint,
 * lbm_step_push, lbm_stream and the batched path keep halfway walls only
 * (LBM_EINVAL with this flag). */
#define LBM_WALLS_ONSITE 0x100u
#define LBM_CAVITY (LBM_WALL_X | LBM_WALL_Y | LBM_WALL_Z | LBM_LID)

typedef struct lbm_lattice lbm_t;

typedef struct {
  int nx, ny, nz;
  int pitch;           /* elements per padded x row of an f buffer */
  int elem_bytes;      /* 4 (FP32) or 2 (FP16, BF16) */
  size_t plane;        /* elements per direction plane: nz * ny * pitch */
  size_t f_bytes;      /* bytes of one f buffer: 19 * plane * elem_bytes */
  size_t lambda_bytes; /* bytes of one adjoint buffer: 19 * plane * 4 */
  size_t cells;        /* nx * ny * nz: elements of one field plane */
} lbm_layout_t;

/* Name of a status code (static string, never NULL). */
const char *lbm_strerror(int code);

/* Text of the last failure seen by the calling thread (CUDA error string or
 * argument check), "" if none. Valid until the thread's next failing call. */
const char *lbm_last_error(void);

/* Create a lattice of nx * ny * nz nodes with relaxation time tau (Eq. 3)
 * and LBM_* flags. Host-only: no CUDA call is made. Requires every size >= 1,
 * tau > 1/2, at most one LBM_STORE_* value, LBM_LID only with LBM_WALL_Z,
 * LBM_ADJOINT only with FP32 storage, and nz * ny * pitch < 2^31. On
 * success *out owns the handle. The kernels relax with omega = 1/tau rounded
 * to the nearest FP32 value whose twelfth is exact (within 2^-22 of 1/tau for
 * tau <= 2, 2^-24 absolute above): the collision's momentum coefficients then
 * sum to exactly omega, so FP32 rounding does not bias the momentum step
 * after step. The same holds for lbm_set_tau and lbm_batch_create. */
int lbm_create(int nx, int ny, int nz, float tau, uint32_t flags,
               lbm_t **out);

/* Free the handle and its device scratch. NULL is accepted. */
int lbm_destroy(lbm_t *h);

/* Buffer layout of the handle (sizes the caller must allocate). */
int lbm_get_layout(const lbm_t *h, lbm_layout_t *out);

/* Bytes of one caller-owned buffer of the given kind: one f buffer, the
 * force field, rho, u, one adjoint (lambda) buffer, or the force gradient.
 * The same figures as lbm_get_layout, one at a time. LBM_EINVAL for a NULL
 * argument or an unknown kind. */
#define LBM_BUF_F 0
#define LBM_BUF_FORCE 1
#define LBM_BUF_RHO 2
#define LBM_BUF_U 3
#define LBM_BUF_LAMBDA 4
#define LBM_BUF_GRADF 5
int lbm_buffer_bytes(const lbm_t *h, int which, size_t *bytes);

/* Bind two caller-owned device f buffers of layout.f_bytes each (256-byte
 * aligned), an optional force field [3][nz][ny][nx] (required iff LBM_FORCE),
 * and a cudaStream_t (NULL = legacy default stream). f_a becomes the current
 * state. Re-binding is allowed at any time. Allocates the handle's device
 * scratch on first use. */
int lbm_bind(lbm_t *h, void *f_a, void *f_b, const float *force,
             void *stream);

/* Lid velocity u_w used by the boundary rule (needs LBM_LID). */
int lbm_set_lid(lbm_t *h, float ux, float uy, float uz);

/* Change tau (> 1/2). */
int lbm_set_tau(lbm_t *h, float tau);

/* Thread-block shape of the one-node kernels (LBM_KERNEL_NODE and BULK
 * steps, initialisation, the slab steps of lbm_run_host): bx threads along x
 * (a multiple of 32), by rows along y, bx * by <= 256 (x-dominant blocks,
 * Sec. 6). The default is bx = min(128, nx rounded up to 32), by = 256 / bx
 * capped at ny. The default two-node kernel takes lbm_set_pair_block. */
int lbm_set_block(lbm_t *h, int bx, int by);

/* Step kernel variant. LBM_KERNEL_NODE: one node per thread (every storage
 * type). LBM_KERNEL_PAIR: 16-bit storage only; two x-adjacent nodes per
 * thread with 32-bit packed loads and stores and warp shuffles for the
 * x-shifted pulls; bit-identical results (slower on GB300, like the shuffle
 * propagation the paper measured on Kepler, Sec. 4.3.2). Default:
 * LBM_KERNEL_X2 (below). */
#define LBM_KERNEL_NODE 0
#define LBM_KERNEL_PAIR 1
/* LBM_KERNEL_BULK / BULK1: the pulled rows are staged in shared memory by
 * bulk copies (TMA) in a persistent producer/consumer pipeline (2-row or
 * 1-row tiles); bit-identical results; lbm_step_moments still uses NODE. */
#define LBM_KERNEL_BULK 2
#define LBM_KERNEL_BULK1 3
/* LBM_KERNEL_X2 (default, every storage type): two x-adjacent nodes per
 * thread and no exchange between threads: one aligned two-value load per
 * pair for the 9 directions with e_x = 0, single-value loads for the others,
 * one two-value store per direction (16-bit: two-value conversions);
 * bit-identical results. Block shape: lbm_set_pair_block. */
#define LBM_KERNEL_X2 4
/* LBM_KERNEL_X4 (16-bit storage, periodic axes and halfway walls; a
 * measured alternative, slower than LBM_KERNEL_X2 on GB300): four
 * x-adjacent nodes per thread; per direction one aligned 4-value load, one
 * single-value load for the value beyond the group when e_x != 0, two
 * 2-value stores; walls on x need only that single load to point at the
 * bounced value, walls on y or z move the whole group load; bit-identical
 * results. Block shape: lbm_set_pair_block, read as groups of four along x.
 * With nx not a multiple of 4 the padding elements after a row's last node
 * up to the next multiple of 4 are loaded and stored (never used). */
#define LBM_KERNEL_X4 5
/* LBM_KERNEL_TMA (16-bit storage, periodic axes and halfway walls; a
 * measured alternative, slower than LBM_KERNEL_X2 on GB300): the pulled
 * values of a tile are staged in shared memory by tensor copies (TMA), one
 * copy per direction, in a persistent producer / consumer pipeline; each
 * thread then completes two x-adjacent nodes like LBM_KERNEL_X2 (the same
 * values). The tile is 64 x-consecutive nodes by 4 rows; the `by` of
 * lbm_set_pair_block selects others: 1 gives 128 nodes by 2 rows, 8 gives
 * 64 by 8.
 * A copy that never lands ends the step with LBM_ETIMEOUT at the next
 * lbm_sync (bounded waits, never a hang). A step fails with LBM_ECUDA if
 * the driver offers no tensor-map encoder. */
#define LBM_KERNEL_TMA 6
int lbm_set_kernel(lbm_t *h, int variant);

/* How the one-node kernel applies bounce-back: LBM_WALLS_SELECT picks each
 * direction's load address (pulled neighbour or opposite direction at the
 * node) for every node, with no divergence; LBM_WALLS_BRANCH gathers as if
 * periodic and re-reads the bounced directions only on wall nodes (fewer
 * instructions when wall nodes are rare in each warp). LBM_WALLS_AUTO
 * (default) selects for FP32 storage, for the LBM_KERNEL_X2 kernel (which
 * selects only in the warps that hold a wall node) and for rows shorter than
 * 256 nodes, else branches. The results are identical.
 * Returns LBM_EINVAL for any other mode. */
#define LBM_WALLS_AUTO 0
#define LBM_WALLS_BRANCH 1
#define LBM_WALLS_SELECT 2
int lbm_set_wall_mode(lbm_t *h, int mode);

/* Multi-step calls (lbm_step, lbm_step_moments, lbm_run_host with n > 1)
 * replay CUDA graphs of `steps` consecutive launches instead of launching
 * each step: one graph per starting buffer, captured on first use on a
 * private stream and again after any change of the launch configuration
 * (bind, tau, lid, block, kernel, wall mode). Removes the per-launch gap that
 * dominates small (L2-resident) lattices. `steps` even in [2, 1024], or 0 for
 * plain launches only (default 32). While the bound stream is itself being
 * captured, plain launches are used. Results are identical either way. */
int lbm_set_graph_steps(lbm_t *h, int steps);

/* Block shape of the pair kernel: bxp pairs along x (a multiple of 32) by
 * `by` rows, bxp * by <= 256, used by LBM_KERNEL_PAIR and LBM_KERNEL_X2
 * (the default kernel). Default: 64 x 2 (1 row when ny = 1). */
int lbm_set_pair_block(lbm_t *h, int bxp, int by);

/* Launch-shape autotuner (no counterpart in the paper, which fixed its block
 * shape by hand, Sec. 6). Times every x-dominant block shape (32..256 threads
 * along x, at most the rounded-up row; 1..8 rows; 64..256 threads) of the
 * current kernel variant (the pair block for LBM_KERNEL_PAIR) over `steps`
 * calls of lbm_step after the same number untimed, with CUDA events on the
 * bound stream, and applies the fastest. This ADVANCES THE STATE by all the
 * steps it runs: tune before initialising the state you want.
 * cache_path: NULL for no cache; else a text file of "key<TAB>a<TAB>b<TAB>ms"
 * lines, key = GPU name and SM count, lattice size, flags, kernel variant and
 * wall mode. A hit applies the cached shape without running anything; a miss
 * tunes and rewrites the file with the new line (temporary file + rename).
 * Outputs (may be NULL): the shape and its time per step in ms.
 * Errors: LBM_EINVAL (NULL handle, steps outside [1, 100000], cache not
 * writable), LBM_EUNBOUND, LBM_ECUDA from a step or the timing. */
int lbm_autotune(lbm_t *h, const char *cache_path, int steps, int *bx, int *by, float *ms);

/* Device pointers of the current state and of the other (scratch) buffer. */
int lbm_current(const lbm_t *h, void **f_cur, void **f_other);

/* Set the current state to f^eq(rho0, u0) (Eq. 5). rho: device [nz][ny][nx]
 * or NULL for rho0 = 1; u: device [3][nz][ny][nx] or NULL for u0 = 0. */
int lbm_init_equilibrium(lbm_t *h, const float *rho, const float *u);

/* Advance n >= 0 time steps: each one fused pull gather, boundary rule,
 * moments, equilibrium, BGK (+ force) collide and store (Alg. 3) from the
 * current buffer into the other one, then a swap. */
int lbm_step(lbm_t *h, int n);

/* As lbm_step, with the last of the n >= 1 steps also writing the density
 * rho [nz][ny][nx] and velocity u [3][nz][ny][nx] it used in its collision
 * (device FP32; the 168-byte-per-update variant of Sec. 4.1). */
int lbm_step_moments(lbm_t *h, int n, float *rho, float *u);

/* One step from an explicit device buffer f_in into f_out (same layout and
 * storage as the bound ones; they must not overlap). The bound pair and the
 * current-state pointer are not touched. */
int lbm_step_to(lbm_t *h, const void *f_in, void *f_out);

/* As lbm_step_to, also writing the density rho [nz][ny][nx] and velocity
 * u [3][nz][ny][nx] (device FP32) that the step's collision used: the inputs
 * of lbm_adjoint_step_moments for this step. */
int lbm_step_to_moments(lbm_t *h, const void *f_in, void *f_out, float *rho, float *u);

/* Push iteration (Alg. 2) for the streaming-order comparison of Sec. 4.2:
 * g_in and g_out hold POST-STREAMING distributions (layout and storage as
 * the f buffers); each node reads its own values (aligned), collides, and
 * writes f*_i to x + e_i (misaligned writes for e_x != 0), or back as the
 * opposite direction at x, plus the moving-wall term, when x + e_i lies
 * outside a walled axis. Starting from g^0 = P f^0 (P: lbm_stream, form
 * PULL) the push states are P applied to the pull states. */
int lbm_step_push(lbm_t *h, const void *g_in, void *g_out);

/* Streaming alone, f_out = P f_in (boundary rule included): form
 * LBM_STREAM_PULL gathers (misaligned reads, aligned writes),
 * LBM_STREAM_PUSH scatters (aligned reads, misaligned writes); both give the
 * same result. LBM_STREAM_COPY copies the 19 planes unshifted (the
 * bandwidth reference of the aligned/misaligned comparison, Sec. 4.3).
 * LBM_STREAM_PULL_L2 gathers like LBM_STREAM_PULL with loads that bypass
 * the L1 and read-only caches (ld.global.cg): the paper's misaligned reads
 * without the read-only data cache (Sec. 4.3). */
#define LBM_STREAM_PULL 0
#define LBM_STREAM_PUSH 1
#define LBM_STREAM_COPY 2
#define LBM_STREAM_PULL_L2 3
int lbm_stream(lbm_t *h, const void *f_in, void *f_out, int form);

/* Moments of the current (post-collision) state: rho = sum f_i (Eq. 6),
 * u = (sum e_i f_i - F/2)/rho (Eq. 7 with the half-force correction), into
 * device FP32 fields (either may be NULL). If mass != NULL the call also
 * reduces the total mass sum(rho) in FP64 into *mass (host), synchronises
 * the stream, and returns LBM_ENONFINITE if any density was not finite. */
int lbm_moments(lbm_t *h, float *rho, float *u, double *mass);

/* Allocation-free variant of lbm_moments (the paper has no counterpart).
 * For callers that cannot allocate device memory: code whose device memory
 * is owned in full by another allocator (a framework's caching pool, an
 * arena sized at start-up) and latency-critical loops in which cudaMalloc or
 * cudaFree may synchronise the device. Needs no handle: f is a device
 * distribution buffer in the library layout for (nx, ny, nz) and the storage
 * type in `flags` (other flag bits are ignored; LBM_FORCE makes it subtract
 * F/2 using `force`, [3][nz][ny][nx]). Writes rho [nz][ny][nx] and u
 * [3][nz][ny][nx] (device FP32, either may be NULL) and, if mass is non-NULL,
 * the FP64 total mass into the DEVICE double *mass; the work is enqueued on
 * `stream` (cudaStream_t) and the call does not wait for it. It calls no
 * cudaMalloc, cudaFree or allocating library routine: its reduction scratch is
 * a fixed 9.75 KiB static device array per GPU, created when the library's
 * device code is loaded on that GPU and kept until the process exits. The
 * first call in each CUDA context (per device, and again in a new context
 * after cudaDeviceReset) looks up that array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream capture.
 * All calls on a device share the array: calls that overlap on the GPU
 * (other streams or threads at the same time) race on it. Unlike
 * lbm_moments, this call does no non-finite check and never returns
 * LBM_ENONFINITE: a non-finite density shows only as a non-finite rho and
 * *mass. Limit: nz * ny * pitch < 2^31 nodes (as for lbm_create); larger
 * sizes return LBM_ERANGE without launching anything. */
int lbm_moments_noalloc(const void *f, int nx, int ny, int nz, uint32_t flags,
                        const float *force, float *rho, float *u, double *mass,
                        void *stream);

/* Synchronise the bound stream; LBM_ECUDA on a pending CUDA error,
 * LBM_ETIMEOUT if a bounded wait inside a step kernel gave up since the last
 * check. */
int lbm_sync(lbm_t *h);

/* Copy the current state to host as FP64 [19][nz][ny][nx], adding w_i back
 * (the plain f_i). Synchronous. */
int lbm_get_f(lbm_t *h, double *host_f);

/* As lbm_get_f for any device buffer `buf` in the handle's f layout. */
int lbm_get_buffer(lbm_t *h, const void *buf, double *host_f);

/* Set the current state from host FP64 [19][nz][ny][nx] (plain f_i; the
 * library subtracts w_i and rounds to the storage type). Synchronous. */
int lbm_set_f(lbm_t *h, const double *host_f);

/* End-to-end call on host buffers: copy u0 [3][nz][ny][nx] (host FP32,
 * pinned for asynchronous copies; NULL = rest) to the device, set the state
 * to f^eq(1, u0), advance n >= 1 steps, and copy rho [nz][ny][nx] and
 * u [3][nz][ny][nx] of the final state back to host. The transfers are
 * pipelined by z slabs on two copy streams: each slab is initialised as soon
 * as it has arrived, and each slab of the last step is copied out as soon as
 * its moments are done. On first use the handle allocates its device staging
 * (28 bytes per node), two streams and a few events, released by lbm_destroy.
 * Synchronous. */
int lbm_run_host(lbm_t *h, const float *u0_host, int n, float *rho_host,
                 float *u_host);

/* ---- discrete adjoint (FP32 storage only; not in the paper) --------------
 * Forward step f^{n+1} = C(P f^n; F): P the pull with bounce-back (affine,
 * the lid term a constant), C the per-node collision of Eq. 3 with the Guo
 * force term. Loss L = 1/2 sum_x |u(x, T) - u_target(x)|^2 with u from the
 * final stored state (Eq. 7 with the half-force correction).
 * lambda^n = dL/df^n = P^T J_C(P f^n)^T lambda^{n+1}. The lambda buffers are
 * FP32, lbm_layout_t.lambda_bytes each, same pitch as the FP32 f buffers;
 * they are not shifted. Each call only enqueues work on the bound stream. */

/* lambda_T = dL/df^T from the state f_T. If grad_force is non-NULL it is
 * OVERWRITTEN with the direct term dL/dF = -(u - u_target)/(2 rho); if loss is
 * non-NULL it must be a DEVICE pointer and receives the FP64 loss. */
int lbm_adjoint_seed(lbm_t *h, const void *f_T, const float *u_target,
                     float *lambda_T, float *grad_force, double *loss);

/* One reverse step: lambda_out = lambda^n from lambda_in = lambda^{n+1} and
 * the state f_n that entered the forward step (the step is recomputed from
 * it). If grad_force is non-NULL, (dC/dF)^T lambda^{n+1} is ADDED into it
 * (the gradient at the bound force, or at F = 0 without LBM_FORCE).
 * lambda_in and lambda_out must not overlap; every element of lambda_out is
 * written exactly once (the transposed pull is a permutation). Launch: 64 x 2
 * blocks (32 x 4 for rows of 32 nodes or fewer); walls by address selection when
 * the wall mode is LBM_WALLS_SELECT, or LBM_WALLS_AUTO with rows shorter than
 * 64 nodes, else only in the warps that hold a wall node (a warp vote). */
int lbm_adjoint_step(lbm_t *h, const void *f_n, const float *lambda_in,
                     float *lambda_out, float *grad_force);

/* The same reverse step from the moments instead of the state: rho_n
 * [nz][ny][nx] and u_n [3][nz][ny][nx] (device FP32) as lbm_step_moments or
 * lbm_step_to_moments wrote them for the forward step from f^n. The
 * collision Jacobian depends on the pulled state only through rho and u, so
 * the result is bit-identical to lbm_adjoint_step(f_n, ...) and the step
 * reads 16 bytes per node instead of gathering 76. Same launch and wall
 * rules and the same errors as lbm_adjoint_step. */
int lbm_adjoint_step_moments(lbm_t *h, const float *rho_n, const float *u_n,
                             const float *lambda_in, float *lambda_out, float *grad_force);

/* grad_u0 = sum_i lambda^0_i d f^eq_i(1, u0) / du0 (Eq. 5) for an initial
 * state f^0 = f^eq(1, u0); u0 may be NULL (zero velocity). Device buffers:
 * lambda0 FP32 lambda layout, u0 and grad_u0 [3][nz][ny][nx]. */
int lbm_adjoint_u0(lbm_t *h, const float *lambda0, const float *u0,
                   float *grad_u0);

/* ---- batched lattices (not in the paper) --------------------------------
 * Many independent lattices of uneven sizes, each with its own tau and lid
 * speed, advanced together with the same per-node update as lbm_step. FP32
 * storage only. The domains' f regions (SoA [19][nz][ny][nx], unpadded rows)
 * are concatenated in one pair of
 * caller-owned buffers, each region 256-byte aligned at the offsets given by
 * lbm_batch_layout. Field outputs are dense per-domain blocks: rho at
 * cell_offset[d] + node, u at 3 * cell_offset[d] + component * cells_d + node.
 * Limits: at most 256 domains, 2^22 nodes per domain and nx * ny < 2^20. */
typedef struct lbm_batch lbm_batch_t;

/* dims: [ndom][3] (nx, ny, nz); tau: [ndom] (> 1/2); lid_ux: [ndom] lid speed
 * along +x (NULL = 0; needs LBM_LID); flags: LBM_WALL_* and LBM_LID only.
 * Host-only. */
int lbm_batch_create(int ndom, const int *dims, const float *tau,
                     const float *lid_ux, uint32_t flags, lbm_batch_t **out);
int lbm_batch_destroy(lbm_batch_t *b);

/* Bytes of one f buffer, total nodes, and per-domain offsets (FP32 elements
 * of the f region; first node in the field buffers); any output may be NULL;
 * the offset arrays hold ndom entries. */
int lbm_batch_layout(const lbm_batch_t *b, size_t *f_bytes, size_t *cells,
                     size_t *f_offsets, size_t *cell_offsets);

/* Bind two device f buffers (256-byte aligned) and a cudaStream_t; f_a
 * becomes current. Uploads the domain and tile tables and allocates the
 * barrier words on first use. */
int lbm_batch_bind(lbm_batch_t *b, void *f_a, void *f_b, void *stream);

/* Tiling of the batched kernels: `threads` nodes per tile and block (32..256,
 * multiple of 32); blocks_per_sm caps the persistent grid (0 = occupancy
 * limit). Chosen by the autotuner. */
int lbm_batch_set_tiling(lbm_batch_t *b, int threads, int blocks_per_sm);

/* Tiling autotuner of the persistent batched step: times threads in
 * {64, 128, 256} x blocks_per_sm in {0, 2, 4, 6, 8}, each over one
 * lbm_batch_step of `steps` steps (rounded up to even) after one untimed call
 * that also captures its graph, and applies the fastest. Advances the state.
 * The cache works as for lbm_autotune, keyed by GPU, domain count, a hash of
 * the domain sizes and walls, and the flags. Outputs may be NULL. Errors:
 * LBM_EINVAL (bad steps, cache not writable), LBM_EUNBOUND, LBM_ECUDA,
 * LBM_ETIMEOUT from a step. */
int lbm_batch_autotune(lbm_batch_t *b, const char *cache_path, int steps, int *threads,
                       int *blocks_per_sm, float *ms);

/* Wall-clock limit of one grid-barrier wait, (0, 60] seconds (default 1). */
int lbm_batch_set_timeout(lbm_batch_t *b, double seconds);

/* Fault injection for tests: the grid barrier expects `extra` more blocks
 * than the launch has, so it can never complete; lbm_batch_step then returns
 * LBM_ETIMEOUT after the timeout instead of hanging. 0 restores normal use. */
int lbm_batch_inject_barrier_fault(lbm_batch_t *b, int extra);

/* Capture the persistent launch in a CUDA graph (default on) or launch it
 * directly (on = 0). */
int lbm_batch_use_graph(lbm_batch_t *b, int on);

/* Persistent grid size, tile size, tile count, and whether the last
 * lbm_batch_step ran from a captured CUDA graph. Outputs may be NULL. */
int lbm_batch_info(const lbm_batch_t *b, int *grid, int *threads, int *ntiles,
                   int *graph_used);

int lbm_batch_current(const lbm_batch_t *b, void **f_cur, void **f_other);

/* Every domain to rest: f = w_i (rho = 1, u = 0). */
int lbm_batch_init_rest(lbm_batch_t *b);

/* n time steps of every domain in ONE persistent cooperative launch (a grid
 * barrier between steps, bounded waits), replayed from a CUDA graph. Waits
 * for the launch to finish; LBM_ETIMEOUT if a barrier wait ran out (the state
 * is then partly advanced and must be re-initialised). */
int lbm_batch_step(lbm_batch_t *b, int n);

/* The same n steps as n ordinary launches over the tile table (no grid
 * barrier); asynchronous. */
int lbm_batch_step_launches(lbm_batch_t *b, int n);

/* Every domain to f^eq(1, u0) (Eq. 5); u0 in the dense per-domain field
 * layout (NULL = rest). */
int lbm_batch_init_equilibrium(lbm_batch_t *b, const float *u0);

/* One step of every domain from an explicit f buffer into another (batch
 * layout, no overlap); the bound pair is not touched. */
int lbm_batch_step_to(lbm_batch_t *b, const void *f_in, void *f_out);

/* As lbm_batch_step_to, also writing every node's collision rho and u into
 * dense per-domain fields (the layout of lbm_batch_moments): the inputs of
 * lbm_batch_adjoint_step_moments for this step. */
int lbm_batch_step_to_moments(lbm_batch_t *b, const void *f_in, void *f_out, float *rho,
                              float *u);

/* Discrete adjoint over all domains, as lbm_adjoint_seed / _step / _u0 for a
 * single lattice (force F = 0; the force gradient is taken at F = 0). The
 * loss is the sum over domains of 1/2 sum_x |u - u_target|^2 (FP64, device
 * pointer). lambda buffers have the batch f layout (FP32); u_target,
 * grad_force, u0 and grad_u0 the dense per-domain field layout. */
int lbm_batch_adjoint_seed(lbm_batch_t *b, const void *f_T, const float *u_target,
                           float *lambda_T, float *grad_force, double *loss);
int lbm_batch_adjoint_step(lbm_batch_t *b, const void *f_n, const float *lambda_in,
                           float *lambda_out, float *grad_force);
/* The reverse step from the moments lbm_batch_step_to_moments wrote for the
 * forward step from f^n (bit-identical to lbm_batch_adjoint_step). */
int lbm_batch_adjoint_step_moments(lbm_batch_t *b, const float *rho_n, const float *u_n,
                                   const float *lambda_in, float *lambda_out,
                                   float *grad_force);
int lbm_batch_adjoint_u0(lbm_batch_t *b, const float *lambda0, const float *u0,
                         float *grad_u0);

/* Step sequences in ONE persistent cooperative launch each (a grid barrier
 * with bounded waits between steps, replayed from a CUDA graph cached per
 * distinct step table; the handle keeps up to 512 such graphs and drops
 * them all when a new table would exceed that, or on rebind or retiling),
 * for the checkpointed adjoint's forward segments, segment recompute and
 * reverse sweeps. Both wait for the launch; LBM_ETIMEOUT as lbm_batch_step.
 * f and lambda buffers must be 256-byte aligned (LBM_EINVAL otherwise).
 *
 * lbm_batch_run: n in [1, 64] steps; step k reads f_in[k] and writes
 * f_out[k] (device buffers in the batch layout, f_in[k] != f_out[k]; step
 * k + 1 sees step k's output only if f_in[k + 1] = f_out[k]). rho and u:
 * both NULL, or arrays of n dense field buffers that step k's collision
 * writes (as lbm_batch_step_to_moments). The bound pair is not touched.
 *
 * lbm_batch_adjoint_run: n in [1, 64] reverse steps from stored moments
 * (as lbm_batch_adjoint_step_moments): step k reads lambda from lambda_a
 * (k even) or lambda_b (k odd) and writes the other, with rho[k], u[k] the
 * moments of the forward step it reverses (so the caller lists them from
 * the last forward step backwards). After n steps lambda^0 of the sequence
 * is in lambda_a if n is even, else in lambda_b. grad_force: NULL or the
 * dense field the force cotangent is ADDED into. */
int lbm_batch_run(lbm_batch_t *b, int n, const void *const *f_in, void *const *f_out,
                  float *const *rho, float *const *u);
int lbm_batch_adjoint_run(lbm_batch_t *b, int n, const float *const *rho, const float *const *u,
                          float *lambda_a, float *lambda_b, float *grad_force);

/* rho and u of every node of the current state into dense device fields
 * (layout above); either may be NULL. */
int lbm_batch_moments(lbm_batch_t *b, float *rho, float *u);

/* Host FP64 copy in / out of one domain's state, [19][nz][ny][nx], plain f_i
 * (w_i added back). Synchronous. */
int lbm_batch_get_f(lbm_batch_t *b, int dom, double *host_f);
int lbm_batch_set_f(lbm_batch_t *b, int dom, const double *host_f);

/* ---- the LBM_CHECK debug build (a stand-in for a device memory checker) ----
 * liblbm_check.so is built from the same sources with -DLBM_CHECK
 * (paper_1309_1983_gb300/build.py: build(check=True)). In it, every load,
 * store and atomic that a kernel makes on global memory is first tested
 * against the table of buffers its launch was given (each buffer a call
 * receives or owns, with the extent and the read / write use documented
 * above) and against the natural alignment of the access. An access that
 * fails is NOT performed (a load reads 0, a store is dropped); it is counted
 * and the first one is kept. Nothing traps and nothing hangs; a refused bulk
 * copy of the shared-memory kernel (LBM_KERNEL_BULK*) ends in LBM_ETIMEOUT
 * through its bounded wait. Tables belong to a translation unit, not to a
 * stream: in a check build, run the calls of one stream at a time. The
 * normal liblbm.so returns LBM_ENOTSUP from these three calls.
 *
 * lbm_check_status: waits for the device, then *refused = accesses refused
 * since the last reset and *first_addr, *first_bytes, *first_kind (1 read,
 * 2 write, 3 read-modify-write) the first of them (zeros if none). Any
 * pointer may be NULL.
 * lbm_check_reset: waits for the device and zeroes the record.
 * lbm_check_narrow: every table built from now on ends each range longer
 * than `bytes` that many bytes before the end of the buffer it describes (0:
 * exact extents again), so that the kernels' accesses to the last `bytes`
 * of every such buffer are refused (and not made): a way to see refusals
 * detected and reported while every access that is made stays inside its
 * buffer. Ranges of at most `bytes` (the error word, small tables) keep
 * their extent, so that a launch can still report what the refusals caused
 * (a bounded wait that gave up). Launches replayed from CUDA graphs
 * captured earlier keep the tables they were captured with. */
int lbm_check_status(unsigned long long *refused, unsigned long long *first_addr,
                     unsigned int *first_bytes, unsigned int *first_kind);
int lbm_check_reset(void);
int lbm_check_narrow(size_t bytes);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
