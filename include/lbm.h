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
 *     them. A handle allocates only a small device scratch area (error word,
 *     reduction partials) on first bind, released by lbm_destroy.
 *   - Work is enqueued on the bound CUDA stream and is asynchronous, except
 *     where a call returns a host value (documented per call), which
 *     synchronises that stream.
 *   - Distribution buffers ("f buffers") use the layout reported by
 *     lbm_get_layout: Structure of Arrays [19][nz][ny][pitch] (Sec. 4.1),
 *     x fastest, each x row padded to `pitch` elements (32-byte aligned
 *     rows), element type FP32, FP16 or BF16 per LBM_STORE_*, holding the
 *     SHIFTED value f_i - w_i. Padding elements are never read.
 *   - Field buffers (rho, velocity u, force F, targets, gradients) are dense
 *     FP32 planes without padding: scalars [nz][ny][nx], vectors
 *     [3][nz][ny][nx] (component-major).
 *   - Adjoint buffers (lambda) are FP32 with the FP32 f-buffer layout (same
 *     pitch), unshifted.
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

/* ---- lbm_create flags ---- */
#define LBM_WALL_X 0x01u     /* bounce-back walls on both x faces */
#define LBM_WALL_Y 0x02u     /* ... y faces */
#define LBM_WALL_Z 0x04u     /* ... z faces */
#define LBM_LID 0x08u        /* the z = nz face moves (needs LBM_WALL_Z) */
#define LBM_STORE_F32 0x00u  /* f_i - w_i stored as FP32 (152 B per update) */
#define LBM_STORE_F16 0x10u  /* ... as FP16, round to nearest even (76 B) */
#define LBM_STORE_BF16 0x20u /* ... as BF16, round to nearest even (76 B) */
#define LBM_FORCE 0x40u      /* read a per-cell body force F each step */
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
 * and nz * ny * pitch < 2^31. On success *out owns the handle. */
int lbm_create(int nx, int ny, int nz, float tau, uint32_t flags,
               lbm_t **out);

/* Free the handle and its device scratch. NULL is accepted. */
int lbm_destroy(lbm_t *h);

/* Buffer layout of the handle (sizes the caller must allocate). */
int lbm_get_layout(const lbm_t *h, lbm_layout_t *out);

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

/* Thread-block shape of the node kernels: bx threads along x (a multiple of
 * 32), by rows along y, bx * by <= 256 (x-dominant blocks, Sec. 6). The
 * default is bx = min(128, nx rounded up to 32), by = 256 / bx capped at ny. */
int lbm_set_block(lbm_t *h, int bx, int by);

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

/* Moments of the current (post-collision) state: rho = sum f_i (Eq. 6),
 * u = (sum e_i f_i - F/2)/rho (Eq. 7 with the half-force correction), into
 * device FP32 fields (either may be NULL). If mass != NULL the call also
 * reduces the total mass sum(rho) in FP64 into *mass (host), synchronises
 * the stream, and returns LBM_ENONFINITE if any density was not finite. */
int lbm_moments(lbm_t *h, float *rho, float *u, double *mass);

/* Synchronise the bound stream; LBM_ECUDA on a pending CUDA error. */
int lbm_sync(lbm_t *h);

/* Copy the current state to host as FP64 [19][nz][ny][nx], adding w_i back
 * (the plain f_i). Synchronous. */
int lbm_get_f(lbm_t *h, double *host_f);

/* Set the current state from host FP64 [19][nz][ny][nx] (plain f_i; the
 * library subtracts w_i and rounds to the storage type). Synchronous. */
int lbm_set_f(lbm_t *h, const double *host_f);

/* End-to-end call on host buffers: copy u0 [3][nz][ny][nx] (host FP32,
 * ideally pinned) to the device, set the state to f^eq(1, u0), advance n >= 1
 * steps, and copy rho [nz][ny][nx] and u [3][nz][ny][nx] of the final state
 * back to host. The non-current f buffer is used as staging for the copies
 * (it is scratch between steps by design). Synchronous. */
int lbm_run_host(lbm_t *h, const float *u0_host, int n, float *rho_host,
                 float *u_host);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
