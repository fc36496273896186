/*
 * FP64 CPU oracle for the D3Q19 BGK lattice Boltzmann step.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow reference that the
 * CUDA path is checked against. Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it. It shares no code, header, table
 * or constant with the CUDA library: the velocity set and the weights below
 * are written out here a second time from the paper.
 *
 * Layout: Array of Structures (the CPU-friendly arrangement of Sec. 4.1),
 * f[cell*19 + i] with cell = (z*ny + y)*nx + x, all values FP64 and unshifted
 * (the plain f_i, not f_i - w_i). Vector fields (velocity, body force) are
 * three planes [3][nz][ny][nx].
 *
 * One time step is computed as two separate passes over the lattice:
 *   1. stream: g_i(x) = f_i(x - e_i)  (pull, Alg. 3), boundary rule applied;
 *   2. collide: rho, u (Eqs. 6-7), f^eq (Eq. 5), BGK relaxation (Eq. 3)
 *      plus the Guo body-force term.
 * The stored state is the post-collision distribution (Sec. 4.1 footnote on
 * the redundant copy; pull order of Alg. 3).
 *
 * Boundary rule (halfway bounce-back). An axis flagged as walled has walls at
 * -1/2 and n-1/2; every other axis is periodic. When the source node x - e_i
 * lies outside a walled axis, g_i(x) = f_ibar(x) + 6 w_i rho_w (e_i . u_w),
 * where ibar is the opposite direction, rho_w = 1, and u_w is the lid
 * velocity when the source lies on the virtual plane z = nz (lid enabled),
 * else zero. (The paper itself used on-site velocity conditions for the
 * cavity, Sec. 5; the halfway rule is the one this library implements.)
 *
 * On-site velocity boundary (the scheme the paper used for its cavity,
 * Sec. 5, citing Hecht & Harting's D3Q19 on-site conditions), selected by
 * the lattice's `onsite` field: the walls of a walled axis then lie ON its
 * first and last node planes. Those nodes stream and collide like any other;
 * after streaming, the populations they would pull from outside the lattice
 * (unknown) are rebuilt so that the node has the prescribed velocity u_w
 * (lid velocity on the top plane z = nz-1, zero elsewhere). The rule is the
 * Zou-He non-equilibrium bounce-back with Hecht & Harting's transverse
 * momentum correction, stated as constraints and solved here directly:
 *   unknown i, opposite known:  g_i = g_ibar + 6 w_i (e_i . j) - e_i . N
 *   "buried" pairs (i and ibar both unknown): equal values b
 * with j = rho u_w - F/2 (so that (sum e g + F/2)/rho = u_w), N the vector
 * that makes sum e_i g_i = j exactly (a 3x3 linear system), and mass fixing
 * rho on a face (rho = sum g) or, where the node lies on two or three walled
 * faces (edges, corners), fixing b, rho being then taken from the stored
 * state of the node one step inward along the diagonal.
 *
 * The discrete adjoint (gradient of L = 1/2 sum |u(T) - u_target|^2 with
 * respect to the initial velocity and the per-cell force) is computed with
 * an explicit dense 19x19 collision Jacobian per cell and a scatter-form
 * transpose of the streaming pass, serially, for small lattices only.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19

/* Eq. 4: the D3Q19 velocity set, one row per direction i = 0..18, columns
 * (e_x, e_y, e_z) in the order the paper prints them. */
static const int E[Q][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {0, 1, 1}, {0, -1, -1},
    {0, 1, -1}, {0, -1, 1}, {1, 0, 1},  {-1, 0, -1}, {-1, 0, 1}, {1, 0, -1}};

/* Weights stated after Eq. 5: 1/3 for i = 0, 1/18 for i = 1..6, 1/36 for the
 * twelve diagonal directions. */
static double weight(int i) {
  if (i == 0) return 1.0 / 3.0;
  if (i <= 6) return 1.0 / 18.0;
  return 1.0 / 36.0;
}

/* Opposite direction found by search, so no index formula is assumed. */
static int opposite(int i) {
  for (int j = 0; j < Q; ++j)
    if (E[j][0] == -E[i][0] && E[j][1] == -E[i][1] && E[j][2] == -E[i][2])
      return j;
  return -1;
}

typedef struct {
  int nx, ny, nz;
  int wall_x, wall_y, wall_z; /* 1: halfway bounce-back on both faces */
  int lid;                    /* 1: the plane z = nz moves with lid_u */
  double tau;
  double lid_u[3];
  int onsite;                 /* 1: on-site velocity walls (see above) */
} oracle_lattice;

/* ---- introspection (used by the tests to pin the tables to the paper) ---- */

int oracle_velocity(int i, int *ex, int *ey, int *ez) {
  if (i < 0 || i >= Q) return -1;
  *ex = E[i][0];
  *ey = E[i][1];
  *ez = E[i][2];
  return 0;
}

double oracle_weight(int i) { return (i >= 0 && i < Q) ? weight(i) : 0.0; }

int oracle_opposite(int i) { return (i >= 0 && i < Q) ? opposite(i) : -1; }

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

static int check_lattice(const oracle_lattice *L) {
  if (!L || L->nx < 1 || L->ny < 1 || L->nz < 1) return -1;
  if (!(L->tau > 0.5)) return -1;
  if (L->lid && !L->wall_z) return -1;
  /* on-site walls need an inner node next to every boundary node */
  if (L->onsite && ((L->wall_x && L->nx < 3) || (L->wall_y && L->ny < 3) ||
                    (L->wall_z && L->nz < 3)))
    return -1;
  return 0;
}

/* ---- Eq. 5: equilibrium ---- */

static double feq(int i, double rho, const double u[3]) {
  const double eu = E[i][0] * u[0] + E[i][1] * u[1] + E[i][2] * u[2];
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  /* c_s^2 = 1/3: 1/c_s^2 = 3, 1/(2 c_s^4) = 4.5, 1/(2 c_s^2) = 1.5 */
  return rho * weight(i) * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
}

/* Guo forcing source S_i(u, F) = w_i [3 (e_i - u) + 9 (e_i . u) e_i] . F */
static double guo_source(int i, const double u[3], const double F[3]) {
  const double eu = E[i][0] * u[0] + E[i][1] * u[1] + E[i][2] * u[2];
  double s = 0.0;
  for (int a = 0; a < 3; ++a)
    s += (3.0 * (E[i][a] - u[a]) + 9.0 * eu * E[i][a]) * F[a];
  return weight(i) * s;
}

/* f = f^eq(rho0, u0) everywhere; rho NULL means rho0 = 1, u NULL means
 * u0 = 0. */
int oracle_init_equilibrium(const oracle_lattice *L, const double *rho,
                            const double *u, double *f) {
  if (check_lattice(L)) return -1;
  const long n = (long)L->nx * L->ny * L->nz;
  for (long c = 0; c < n; ++c) {
    double r = rho ? rho[c] : 1.0;
    double uc[3] = {0.0, 0.0, 0.0};
    if (u)
      for (int a = 0; a < 3; ++a) uc[a] = u[a * n + c];
    for (int i = 0; i < Q; ++i) f[c * Q + i] = feq(i, r, uc);
  }
  return 0;
}

/* Where the pull for direction i at node (x,y,z) comes from.
 * Returns 1 when the source lies outside a walled axis (bounce-back), with
 * *lidsrc set when that source is on the moving plane z = nz; otherwise
 * returns 0 and *src is the (periodically wrapped) source cell. */
static int pull_source(const oracle_lattice *L, int x, int y, int z, int i,
                       long *src, int *lidsrc) {
  int sx = x - E[i][0], sy = y - E[i][1], sz = z - E[i][2];
  int out = 0;
  if (L->wall_x && (sx < 0 || sx >= L->nx)) out = 1;
  if (L->wall_y && (sy < 0 || sy >= L->ny)) out = 1;
  if (L->wall_z && (sz < 0 || sz >= L->nz)) out = 1;
  *lidsrc = (out && L->lid && sz == L->nz);
  if (out) return 1;
  /* periodic wrap; |e_i| components are at most 1 */
  if (sx < 0) sx += L->nx;
  if (sx >= L->nx) sx -= L->nx;
  if (sy < 0) sy += L->ny;
  if (sy >= L->ny) sy -= L->ny;
  if (sz < 0) sz += L->nz;
  if (sz >= L->nz) sz -= L->nz;
  *src = ((long)sz * L->ny + sy) * L->nx + sx;
  return 0;
}

/* ---- on-site velocity boundary (Hecht & Harting), see the header ---- */

/* Solve the 3x3 system A v = r by Gaussian elimination with partial
 * pivoting. Returns -1 if A is singular. */
static int solve3(double A[3][3], double r[3], double v[3]) {
  for (int k = 0; k < 3; ++k) {
    int p = k;
    for (int m = k + 1; m < 3; ++m)
      if (fabs(A[m][k]) > fabs(A[p][k])) p = m;
    if (fabs(A[p][k]) < 1e-300) return -1;
    if (p != k) {
      for (int q = 0; q < 3; ++q) {
        const double t = A[k][q];
        A[k][q] = A[p][q];
        A[p][q] = t;
      }
      const double t = r[k];
      r[k] = r[p];
      r[p] = t;
    }
    for (int m = k + 1; m < 3; ++m) {
      const double l = A[m][k] / A[k][k];
      for (int q = k; q < 3; ++q) A[m][q] -= l * A[k][q];
      r[m] -= l * r[k];
    }
  }
  for (int k = 2; k >= 0; --k) {
    double s = r[k];
    for (int q = k + 1; q < 3; ++q) s -= A[k][q] * v[q];
    v[k] = s / A[k][k];
  }
  return 0;
}

/* Rebuild the unknown populations of gc (unknown[i] = 1) for density rho and
 * target momentum j (see the header); returns the node's total mass. */
static double onsite_fill(const int unknown[Q], double rho, const double j[3],
                          double *gc) {
  double M[3][3] = {{0}}, r[3], N[3] = {0, 0, 0};
  for (int a = 0; a < 3; ++a) r[a] = -j[a];
  int nburied = 0;
  for (int i = 0; i < Q; ++i) {
    const int ib = opposite(i);
    if (!unknown[i]) {
      for (int a = 0; a < 3; ++a) r[a] += E[i][a] * gc[i];
    } else if (unknown[ib]) {
      ++nburied; /* buried: its pair member contributes -e_i b, they cancel */
    } else {
      const double ej = E[i][0] * j[0] + E[i][1] * j[1] + E[i][2] * j[2];
      for (int a = 0; a < 3; ++a) {
        r[a] += E[i][a] * (gc[ib] + 6.0 * weight(i) * ej);
        for (int b = 0; b < 3; ++b) M[a][b] += E[i][a] * E[i][b];
      }
    }
  }
  /* momentum of the rebuilt node: r - M N = 0 */
  solve3(M, r, N);
  double mass = 0.0;
  for (int i = 0; i < Q; ++i) {
    const int ib = opposite(i);
    if (unknown[i] && !unknown[ib]) {
      const double ej = E[i][0] * j[0] + E[i][1] * j[1] + E[i][2] * j[2];
      const double eN = E[i][0] * N[0] + E[i][1] * N[1] + E[i][2] * N[2];
      gc[i] = gc[ib] + 6.0 * weight(i) * ej - eN;
    }
    if (!(unknown[i] && unknown[ib])) mass += gc[i];
  }
  if (nburied) {
    const double b = (rho - mass) / nburied;
    for (int i = 0; i < Q; ++i)
      if (unknown[i] && unknown[opposite(i)]) gc[i] = b;
    mass = rho;
  }
  return mass;
}

/* Inward normals of the walled faces node (x,y,z) lies on; returns their
 * count and sums them into s. */
static int onsite_faces(const oracle_lattice *L, int x, int y, int z, int s[3]) {
  const int p[3] = {x, y, z}, n[3] = {L->nx, L->ny, L->nz};
  const int walled[3] = {L->wall_x, L->wall_y, L->wall_z};
  int count = 0;
  for (int a = 0; a < 3; ++a) {
    s[a] = 0;
    if (!walled[a]) continue;
    if (p[a] == 0) s[a] = 1;
    if (p[a] == n[a] - 1) s[a] = -1;
    count += s[a] != 0;
  }
  return count;
}

/* On-site rule at boundary node (x,y,z): gc holds the pulled populations
 * (unknown ones are overwritten), f the state before streaming (AoS). */
static void onsite_node(const oracle_lattice *L, int x, int y, int z,
                        const int unknown[Q], const double *f,
                        const double *force, double *gc) {
  const long n = (long)L->nx * L->ny * L->nz;
  const long c = ((long)z * L->ny + y) * L->nx + x;
  int s[3];
  const int faces = onsite_faces(L, x, y, z, s);
  double uw[3] = {0.0, 0.0, 0.0}, F[3] = {0.0, 0.0, 0.0};
  if (L->lid && faces == 1 && z == L->nz - 1)
    for (int a = 0; a < 3; ++a) uw[a] = L->lid_u[a];
  if (force)
    for (int a = 0; a < 3; ++a) F[a] = force[a * n + c];
  double rho;
  if (faces == 1) {
    /* mass = sum g is affine in rho: solve it from two evaluations */
    double g0[Q], g1[Q], j[3];
    memcpy(g0, gc, sizeof(g0));
    memcpy(g1, gc, sizeof(g1));
    for (int a = 0; a < 3; ++a) j[a] = -0.5 * F[a];
    const double m0 = onsite_fill(unknown, 0.0, j, g0);
    for (int a = 0; a < 3; ++a) j[a] = uw[a] - 0.5 * F[a];
    const double m1 = onsite_fill(unknown, 1.0, j, g1);
    rho = m0 / (1.0 - (m1 - m0));
  } else {
    /* edge or corner: density of the inner diagonal neighbour, stored state */
    const long nb = ((long)(z + s[2]) * L->ny + (y + s[1])) * L->nx + (x + s[0]);
    rho = 0.0;
    for (int i = 0; i < Q; ++i) rho += f[nb * Q + i];
  }
  double j[3];
  for (int a = 0; a < 3; ++a) j[a] = rho * uw[a] - 0.5 * F[a];
  onsite_fill(unknown, rho, j, gc);
}

/* Pass 1 with on-site walls: plain pulls where the source is inside, then
 * the on-site rule on every boundary node. */
static int stream_onsite(const oracle_lattice *L, const double *f,
                         const double *force, double *g) {
  const int nx = L->nx, ny = L->ny, nz = L->nz;
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const long c = ((long)z * ny + y) * nx + x;
        int unknown[Q], any = 0;
        for (int i = 0; i < Q; ++i) {
          long src = 0;
          int lidsrc = 0;
          unknown[i] = pull_source(L, x, y, z, i, &src, &lidsrc);
          g[c * Q + i] = unknown[i] ? 0.0 : f[src * Q + i];
          any |= unknown[i];
        }
        if (any) onsite_node(L, x, y, z, unknown, f, force, g + c * Q);
      }
  return 0;
}

/* Pass 1: streaming with the boundary rule (Alg. 3, first loop, then the
 * boundary step). The on-site rule uses the body force (its target momentum
 * is rho u_w - F/2); the halfway rule ignores it. */
int oracle_stream_forced(const oracle_lattice *L, const double *f,
                         const double *force, double *g) {
  if (check_lattice(L)) return -1;
  if (L->onsite) return stream_onsite(L, f, force, g);
  const int nx = L->nx, ny = L->ny, nz = L->nz;
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const long c = ((long)z * ny + y) * nx + x;
        for (int i = 0; i < Q; ++i) {
          long src = 0;
          int lidsrc = 0;
          if (pull_source(L, x, y, z, i, &src, &lidsrc)) {
            double corr = 0.0;
            if (lidsrc)
              corr = 6.0 * weight(i) * 1.0 *
                     (E[i][0] * L->lid_u[0] + E[i][1] * L->lid_u[1] +
                      E[i][2] * L->lid_u[2]);
            g[c * Q + i] = f[c * Q + opposite(i)] + corr;
          } else {
            g[c * Q + i] = f[src * Q + i];
          }
        }
      }
  return 0;
}

int oracle_stream(const oracle_lattice *L, const double *f, double *g) {
  return oracle_stream_forced(L, f, NULL, g);
}

/* Pass 2: moments (Eqs. 6-7, with half the force added to the momentum),
 * equilibrium (Eq. 5) and the BGK relaxation of Eq. 3 with the Guo term:
 *   f*_i = g_i - (g_i - f_i^eq)/tau + (1 - 1/(2 tau)) S_i(u, F). */
int oracle_collide(const oracle_lattice *L, const double *g,
                   const double *force, double *fout) {
  if (check_lattice(L)) return -1;
  const long n = (long)L->nx * L->ny * L->nz;
  const double tau = L->tau;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < n; ++c) {
    const double *gc = g + c * Q;
    double F[3] = {0.0, 0.0, 0.0};
    if (force)
      for (int a = 0; a < 3; ++a) F[a] = force[a * n + c];
    double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
      rho += gc[i];
      for (int a = 0; a < 3; ++a) m[a] += E[i][a] * gc[i];
    }
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = (m[a] + 0.5 * F[a]) / rho;
    for (int i = 0; i < Q; ++i)
      fout[c * Q + i] = gc[i] - (gc[i] - feq(i, rho, u)) / tau +
                        (1.0 - 0.5 / tau) * guo_source(i, u, F);
  }
  return 0;
}

/* n full time steps; f_in and f_out may alias. */
int oracle_run(const oracle_lattice *L, const double *f_in, const double *force,
               int nsteps, double *f_out) {
  if (check_lattice(L) || nsteps < 0) return -1;
  const long len = (long)L->nx * L->ny * L->nz * Q;
  double *a = (double *)malloc(sizeof(double) * len);
  double *g = (double *)malloc(sizeof(double) * len);
  if (!a || !g) {
    free(a);
    free(g);
    return -2;
  }
  memcpy(a, f_in, sizeof(double) * len);
  for (int s = 0; s < nsteps; ++s) {
    oracle_stream_forced(L, a, force, g);
    oracle_collide(L, g, force, a);
  }
  memcpy(f_out, a, sizeof(double) * len);
  free(a);
  free(g);
  return 0;
}

/* Moments of a stored (post-collision) state: rho = sum f_i (Eq. 6) and
 * u = (sum e_i f_i - F/2)/rho (Eq. 7; the collision adds F to the momentum,
 * so the post-collision momentum exceeds rho u by F/2). */
int oracle_moments(const oracle_lattice *L, const double *f,
                   const double *force, double *rho, double *u) {
  if (check_lattice(L)) return -1;
  const long n = (long)L->nx * L->ny * L->nz;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < n; ++c) {
    double r = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
      r += f[c * Q + i];
      for (int a = 0; a < 3; ++a) m[a] += E[i][a] * f[c * Q + i];
    }
    rho[c] = r;
    for (int a = 0; a < 3; ++a) {
      const double F = force ? force[a * n + c] : 0.0;
      u[a * n + c] = (m[a] - 0.5 * F) / r;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------
 * Discrete adjoint (not in the paper: the exact transpose of the forward
 * step above). Forward step: f^{n+1} = C(P f^n; F) with P the pull with
 * bounce-back (affine; the lid term is a constant) and C the per-cell
 * collision. Backward: lambda^n = P^T J_C(P f^n)^T lambda^{n+1}, and the
 * force cotangent gains (dC/dF)^T lambda^{n+1} at every step.
 * ---------------------------------------------------------------------- */

/* Dense Jacobians of the collision at one cell:
 *   Jg[i][j] = d f*_i / d g_j  (19x19),  JF[i][a] = d f*_i / d F_a  (19x3).
 * Chain rule through rho = sum g, m = sum e g + F/2, u = m/rho. */
static void collision_jacobian(const double *gc, const double F[3], double tau,
                               double Jg[Q][Q], double JF[Q][3]) {
  const double om = 1.0 / tau, kf = 1.0 - 0.5 * om;
  double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < Q; ++i) {
    rho += gc[i];
    for (int a = 0; a < 3; ++a) m[a] += E[i][a] * gc[i];
  }
  double u[3];
  for (int a = 0; a < 3; ++a) u[a] = (m[a] + 0.5 * F[a]) / rho;
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < Q; ++i) {
    const double w = weight(i);
    const double eu = E[i][0] * u[0] + E[i][1] * u[1] + E[i][2] * u[2];
    const double eF = E[i][0] * F[0] + E[i][1] * F[1] + E[i][2] * F[2];
    /* partial derivatives of f^eq_i at fixed u, and with respect to u */
    const double dfeq_drho = w * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    double dfeq_du[3], dS_du[3], dS_dF[3];
    for (int a = 0; a < 3; ++a) {
      dfeq_du[a] = w * rho * (3.0 * E[i][a] + 9.0 * eu * E[i][a] - 3.0 * u[a]);
      dS_du[a] = w * (-3.0 * F[a] + 9.0 * eF * E[i][a]);
      dS_dF[a] = w * (3.0 * (E[i][a] - u[a]) + 9.0 * eu * E[i][a]);
    }
    for (int j = 0; j < Q; ++j) {
      /* du/dg_j = (e_j - u)/rho, drho/dg_j = 1 */
      double v = (i == j) ? (1.0 - om) : 0.0;
      v += om * dfeq_drho;
      for (int a = 0; a < 3; ++a)
        v += (om * dfeq_du[a] + kf * dS_du[a]) * (E[j][a] - u[a]) / rho;
      Jg[i][j] = v;
    }
    for (int a = 0; a < 3; ++a)
      /* du/dF_a = e_a / (2 rho) */
      JF[i][a] = kf * dS_dF[a] + (om * dfeq_du[a] + kf * dS_du[a]) * 0.5 / rho;
  }
}

/* One reverse step. lam_in = lambda^{n+1} (cotangent of the state after the
 * step), f_n = the state before it; writes lam_out = lambda^n and, when
 * grad_force is non-NULL, adds (dC/dF)^T lambda^{n+1} into it. Serial. */
int oracle_adjoint_step(const oracle_lattice *L, const double *f_n,
                        const double *force, const double *lam_in,
                        double *lam_out, double *grad_force) {
  if (check_lattice(L)) return -1;
  if (L->onsite) return -1; /* the transpose below is that of the halfway rule */
  const int nx = L->nx, ny = L->ny, nz = L->nz;
  const long n = (long)nx * ny * nz;
  double *g = (double *)malloc(sizeof(double) * n * Q);
  if (!g) return -2;
  oracle_stream(L, f_n, g);
  memset(lam_out, 0, sizeof(double) * n * Q);
  double Jg[Q][Q], JF[Q][3];
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const long c = ((long)z * ny + y) * nx + x;
        double F[3] = {0.0, 0.0, 0.0};
        if (force)
          for (int a = 0; a < 3; ++a) F[a] = force[a * n + c];
        collision_jacobian(g + c * Q, F, L->tau, Jg, JF);
        const double *lam = lam_in + c * Q;
        double mu[Q];
        for (int j = 0; j < Q; ++j) {
          double s = 0.0;
          for (int i = 0; i < Q; ++i) s += Jg[i][j] * lam[i];
          mu[j] = s;
        }
        if (grad_force)
          for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (int i = 0; i < Q; ++i) s += JF[i][a] * lam[i];
            grad_force[a * n + c] += s;
          }
        /* transpose of the pull: g_i(x) read f_i(src) or f_ibar(x) */
        for (int i = 0; i < Q; ++i) {
          long src = 0;
          int lidsrc = 0;
          if (pull_source(L, x, y, z, i, &src, &lidsrc))
            lam_out[c * Q + opposite(i)] += mu[i];
          else
            lam_out[src * Q + i] += mu[i];
        }
      }
  free(g);
  return 0;
}

/* Loss L = 1/2 sum_x |u(x) - u_target(x)|^2 on the final state, its
 * cotangent lambda^T = dL/df^T, and (when grad_force is non-NULL) the direct
 * force term dL/dF = -(u - u_target)/(2 rho) written into grad_force. */
int oracle_adjoint_seed(const oracle_lattice *L, const double *f_T,
                        const double *force, const double *u_target,
                        double *lam_T, double *grad_force, double *loss) {
  if (check_lattice(L)) return -1;
  const long n = (long)L->nx * L->ny * L->nz;
  double acc = 0.0;
  for (long c = 0; c < n; ++c) {
    double r = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
      r += f_T[c * Q + i];
      for (int a = 0; a < 3; ++a) m[a] += E[i][a] * f_T[c * Q + i];
    }
    double u[3], d[3];
    for (int a = 0; a < 3; ++a) {
      const double F = force ? force[a * n + c] : 0.0;
      u[a] = (m[a] - 0.5 * F) / r;
      d[a] = u[a] - u_target[a * n + c];
      acc += 0.5 * d[a] * d[a];
    }
    /* du_a/df_j = (e_ja - u_a)/rho */
    for (int j = 0; j < Q; ++j) {
      double s = 0.0;
      for (int a = 0; a < 3; ++a) s += d[a] * (E[j][a] - u[a]);
      lam_T[c * Q + j] = s / r;
    }
    if (grad_force)
      for (int a = 0; a < 3; ++a) grad_force[a * n + c] = -0.5 * d[a] / r;
  }
  *loss = acc;
  return 0;
}

/* Gradient with respect to the initial velocity when f^0 = f^eq(1, u0):
 * grad_u0(x) = sum_i lambda^0_i(x) d f^eq_i / du at rho = 1. */
int oracle_adjoint_u0(const oracle_lattice *L, const double *lam0,
                      const double *u0, double *grad_u0) {
  if (check_lattice(L)) return -1;
  const long n = (long)L->nx * L->ny * L->nz;
  for (long c = 0; c < n; ++c) {
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = u0 ? u0[a * n + c] : 0.0;
    double gacc[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
      const double eu = E[i][0] * u[0] + E[i][1] * u[1] + E[i][2] * u[2];
      for (int a = 0; a < 3; ++a)
        gacc[a] += lam0[c * Q + i] * weight(i) *
                   (3.0 * E[i][a] + 9.0 * eu * E[i][a] - 3.0 * u[a]);
    }
    for (int a = 0; a < 3; ++a) grad_u0[a * n + c] = gacc[a];
  }
  return 0;
}
