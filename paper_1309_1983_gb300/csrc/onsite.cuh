// onsite.cuh - on-site velocity walls: the boundary scheme the paper used for
// its lid-driven cavity (Sec. 5), the D3Q19 on-site velocity conditions of
// Hecht & Harting (J. Stat. Mech. 2010, P01018): Zou-He bounce-back of the
// non-equilibrium part along the wall normal plus a transverse momentum
// correction.
//
// Walls lie ON the first and last node planes of every walled axis. Those
// nodes stream and collide like interior nodes; after the pull, the
// populations they would take from outside the lattice ("unknown": e_i has a
// component equal to an inward normal) are rebuilt so that the node moves
// with the wall velocity u_w (the lid velocity on the interior of the top
// plane z = nz - 1, zero elsewhere). With j = rho u_w - F/2 (so that the
// Guo velocity (sum e g + F/2)/rho is exactly u_w):
//   face, inward normal n:
//     rho = (S_0 + 2 S_- - F.n/2) / (1 - u_w.n),  S_0 / S_-: sums over
//           e.n = 0 / e.n = -1 of the pulled values,
//     N_t = 1/2 sum_{e.n=0} e_t g - j_t / 3 for the two tangential axes t,
//     g_n       = g_-n + j.n / 3,
//     g_{n+t}   = g_{-n-t} + (j.n + j.t) / 6 - N_t, g_{n-t} likewise;
//   edge (inward normals n_a, n_b; tangent axis c) and corner: the known
//     values do not fix rho; it is taken from the stored state of the inner
//     diagonal neighbour x + n_a + n_b (+ n_c). Unknown i whose opposite is
//     known: g_i = g_ibar + 6 w_i (e_i.j) - e_i.N with the N that makes the
//     momentum exactly j:
//       edge:   N'_a = (j'_b - j'_a)/18, N'_b = -N'_a,
//               N_c  = (g_{+c} - g_{-c})/4 - j_c/12,
//       corner: N'_a = (j'_b + j'_c - 2 j'_a)/12 (and cyclically),
//     with primes the components along the inward normals (x'_a = s_a x_a).
//     "Buried" pairs (i and ibar both unknown, pointing along the walls)
//     share the remaining mass equally.
// All of this acts on the shifted values d_i = g_i - w_i: the shifts cancel
// in every difference g_i - g_ibar, and the weights of the sums S_0 + 2 S_-
// add up to 1.
#pragma once

#include "d3q19.cuh"
#include "internal.h"
#include "stream.cuh"

namespace lbm {

template <int i>
__device__ __forceinline__ int e_comp(int axis) {
  constexpr int ex = kEx[i], ey = kEy[i], ez = kEz[i];
  return axis == 0 ? ex : axis == 1 ? ey : ez;
}

// Whether e_i has a component equal to one of the nonzero inward normals
// (sx, sy, sz): direction i is then pulled from outside the lattice. With
// the signs flipped, whether its opposite is.
template <int i>
__device__ __forceinline__ bool from_outside(int sx, int sy, int sz) {
  constexpr int ex = kEx[i], ey = kEy[i], ez = kEz[i];
  return (sx != 0 && ex == sx) || (sy != 0 && ey == sy) || (sz != 0 && ez == sz);
}

// Face rule (one inward normal: axis AXIS, sign SGN) on shifted values. The
// rule and its callers are inlined: a call that takes d by reference would
// keep every thread's populations in local memory, wall node or not.
template <int AXIS, int SGN>
__device__ __forceinline__ void onsite_face(float (&d)[Q], float ux, float uy, float uz, float Fx,
                                            float Fy, float Fz) {
  constexpr int axis = AXIS, sgn = SGN;
  float s0 = 0.0f, sm = 0.0f, tx = 0.0f, ty = 0.0f, tz = 0.0f;
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int ex = kEx[i], ey = kEy[i], ez = kEz[i];
    const int en = sgn * e_comp<i>(axis);
    if (en == 0) {
      s0 += d[i];
      if constexpr (ex != 0) tx += ex * d[i];
      if constexpr (ey != 0) ty += ey * d[i];
      if constexpr (ez != 0) tz += ez * d[i];
    } else if (en < 0) {
      sm += d[i];
    }
  });
  const float un = sgn * (axis == 0 ? ux : axis == 1 ? uy : uz);
  const float Fn = sgn * (axis == 0 ? Fx : axis == 1 ? Fy : Fz);
  // rho - 1 = (S_0 + 2 S_- - F.n/2 - (1 - u.n)) / (1 - u.n) in shifted sums
  const float dr = (s0 + 2.0f * sm - 0.5f * Fn + un) / (1.0f - un);
  const float rho = 1.0f + dr;
  const float jx = fmaf(rho, ux, -0.5f * Fx), jy = fmaf(rho, uy, -0.5f * Fy),
              jz = fmaf(rho, uz, -0.5f * Fz);
  const float Nx = axis == 0 ? 0.0f : fmaf(0.5f, tx, -jx * (1.0f / 3.0f));
  const float Ny = axis == 1 ? 0.0f : fmaf(0.5f, ty, -jy * (1.0f / 3.0f));
  const float Nz = axis == 2 ? 0.0f : fmaf(0.5f, tz, -jz * (1.0f / 3.0f));
  static_for<1, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if (sgn * e_comp<i>(axis) == 1) {
      constexpr float cx = (float)kEx[i], cy = (float)kEy[i], cz = (float)kEz[i];
      constexpr float k = 6.0f * weight(i);  // 1/3 (normal) or 1/6 (diagonal)
      const float ej = cx * jx + cy * jy + cz * jz;
      const float eN = cx * Nx + cy * Ny + cz * Nz;
      d[i] = d[kOpp_v<i>] + fmaf(k, ej, -eN);
    }
  });
}

// Edge and corner rule (two or three inward normals s, u_w = 0) on shifted
// values; dr = rho - 1 of the inner diagonal neighbour.
__device__ __forceinline__ void onsite_edge_corner(float (&d)[Q], int sx, int sy, int sz, float dr,
                                                   float Fx, float Fy, float Fz) {
  const float jx = -0.5f * Fx, jy = -0.5f * Fy, jz = -0.5f * Fz;
  // components along the inward normals (zero on the unwalled axis)
  const float px = sx * jx, py = sy * jy, pz = sz * jz;
  float Nx, Ny, Nz;
  if (sx != 0 && sy != 0 && sz != 0) {
    Nx = sx * (py + pz - 2.0f * px) * (1.0f / 12.0f);
    Ny = sy * (px + pz - 2.0f * py) * (1.0f / 12.0f);
    Nz = sz * (px + py - 2.0f * pz) * (1.0f / 12.0f);
  } else if (sx == 0) {  // edge along x: normals y, z
    Ny = sy * (pz - py) * (1.0f / 18.0f);
    Nz = -sz * (pz - py) * (1.0f / 18.0f);
    Nx = fmaf(0.25f, d[1] - d[2], -jx * (1.0f / 12.0f));
  } else if (sy == 0) {  // edge along y: normals x, z
    Nx = sx * (pz - px) * (1.0f / 18.0f);
    Nz = -sz * (pz - px) * (1.0f / 18.0f);
    Ny = fmaf(0.25f, d[3] - d[4], -jy * (1.0f / 12.0f));
  } else {  // edge along z: normals x, y
    Nx = sx * (py - px) * (1.0f / 18.0f);
    Ny = -sy * (py - px) * (1.0f / 18.0f);
    Nz = fmaf(0.25f, d[5] - d[6], -jz * (1.0f / 12.0f));
  }
  float rest = 0.0f;  // mass of every population except the buried ones
  int nburied = 0;
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const bool unk = from_outside<i>(sx, sy, sz);
    const bool opp_unk = from_outside<i>(-sx, -sy, -sz);
    if (unk && opp_unk) {
      ++nburied;
    } else {
      if (unk) {
        constexpr float cx = (float)kEx[i], cy = (float)kEy[i], cz = (float)kEz[i];
        constexpr float k = 6.0f * weight(i);
        const float ej = cx * jx + cy * jy + cz * jz;
        const float eN = cx * Nx + cy * Ny + cz * Nz;
        d[i] = d[kOpp_v<i>] + fmaf(k, ej, -eN);
      }
      rest += d[i];
    }
  });
  // every buried direction has weight 1/36: equal g means equal shifted d
  const float b = (dr - rest) / (float)nburied;
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const bool unk = from_outside<i>(sx, sy, sz);
    const bool opp_unk = from_outside<i>(-sx, -sy, -sz);
    if (unk && opp_unk) d[i] = b;
  });
}

// Apply the on-site rule at node n after a plain (periodically wrapped)
// pull into d: nothing happens off the walls. fin is the state the pull
// read (the stored state of the previous step).
template <int S>
__device__ __forceinline__ void onsite_apply(const typename Store<S>::T *__restrict__ fin,
                                             const StepArgs &a, const NodeIdx &n, float Fx,
                                             float Fy, float Fz, float (&d)[Q]) {
  const int sx = n.x0 ? 1 : (n.x1 ? -1 : 0);
  const int sy = n.y0 ? 1 : (n.y1 ? -1 : 0);
  const int sz = n.z0 ? 1 : (n.z1 ? -1 : 0);
  const int faces = (sx != 0) + (sy != 0) + (sz != 0);
  if (faces == 0) return;
  if (faces == 1) {
    // one instance per face: the wall velocity is zero except on the lid
    // (selected before the branches: 6% faster for 16-bit storage than
    // selecting it inside the lid's branch)
    const bool lid = a.onsite_lid && sz == -1;
    const float ux = lid ? a.lid[0] : 0.0f, uy = lid ? a.lid[1] : 0.0f, uz = lid ? a.lid[2] : 0.0f;
    if (sx == 1) onsite_face<0, 1>(d, 0.0f, 0.0f, 0.0f, Fx, Fy, Fz);
    else if (sx == -1) onsite_face<0, -1>(d, 0.0f, 0.0f, 0.0f, Fx, Fy, Fz);
    else if (sy == 1) onsite_face<1, 1>(d, 0.0f, 0.0f, 0.0f, Fx, Fy, Fz);
    else if (sy == -1) onsite_face<1, -1>(d, 0.0f, 0.0f, 0.0f, Fx, Fy, Fz);
    else if (sz == 1) onsite_face<2, 1>(d, 0.0f, 0.0f, 0.0f, Fx, Fy, Fz);
    else onsite_face<2, -1>(d, ux, uy, uz, Fx, Fy, Fz);
  } else {
    const long long cn = (long long)n.c + (long long)sz * a.ny * a.pitch +
                         (long long)sy * a.pitch + sx;
    float dr = 0.0f;
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      dr += Store<S>::ld(fin + (size_t)i * a.plane + (size_t)cn);
    });
    onsite_edge_corner(d, sx, sy, sz, dr, Fx, Fy, Fz);
  }
}

}  // namespace lbm
