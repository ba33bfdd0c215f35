// Colour-gradient repulsion force (Sec. 2.3, Eqs. repForce, potential, normal1, normal2).
//
//   F_rep(x) = Pi psi_rep(rho^N(x)) sum_{i>=1} H(-(n.c_i)(n'_i.c_i)) [(n.c_i) n + (n'_i.c_i) n'_i] / |c_i|
//
// with n the unit colour gradient at x and n'_i the one at x + c_i.  The force needs the
// colour gradient one node away, i.e. rho^N two nodes away, so it is computed from two
// pre-pass fields written before each step that has it enabled:
//   colour_kernel : rho^N(x) from the stored populations (the same density bookkeeping as
//                   the step kernel);
//   normals_kernel: n(x) = grad rho^N / |grad rho^N| (zero vector where |grad rho^N| <= eps,
//                   which then contributes nothing), gradient by the isotropic stencil.
// Readings: psi_rep = (1 - |rho^N|)^chi (or the printed (1 + |rho^N|)^chi), H(0) = 0,
// direction 0 skipped, a wall neighbour contributes nothing.
#pragma once

#include <cstdint>

#include "lbm_lattice.cuh"

namespace lbm {

template <class T>
__device__ __forceinline__ T fpow(T b, T e);
template <>
__device__ __forceinline__ float fpow<float>(float b, float e) { return e == 2.0f ? b * b : powf(b, e); }
template <>
__device__ __forceinline__ double fpow<double>(double b, double e) { return e == 2.0 ? b * b : pow(b, e); }

struct RepParams {
  int nx, ny, nz;
  long long n;
  int color_norm, psi_kind;
  double inv_rho_r0, inv_rho_b0, grad_eps, pi, chi;
};

__device__ __forceinline__ long long wrap_index(int x, int y, int z, int nx, int ny, int nz) {
  x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
  y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
  z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
  return x + (long long)nx * (y + (long long)ny * z);
}
// The same in index type I (int when every node index of the lattice fits 32 bits).
template <class I>
__device__ __forceinline__ I wrap_index_t(int x, int y, int z, int nx, int ny, int nz) {
  x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
  y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
  z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
  return x + I(nx) * (y + I(ny) * z);
}

// normals[3][N] (zero where undefined)
template <class L, class T, class I = long long>
__global__ void normals_kernel(const T* __restrict__ colour, const uint8_t* __restrict__ solid,
                               T* __restrict__ normals, RepParams a) {
  const I N = I(a.n);
  for (I m = blockIdx.x * I(blockDim.x) + threadIdx.x; m < N; m += I(gridDim.x) * blockDim.x) {
    int x, y, z;
    node_coords(m, a.nx, a.ny, a.n, x, y, z);
    T g[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int q = 0; q < L::NP; q++) {
      const I mp = wrap_index_t<I>(x + L::pcx(q), y + L::pcy(q), z + L::pcz(q), a.nx, a.ny, a.nz);
      const I mm = wrap_index_t<I>(x - L::pcx(q), y - L::pcy(q), z - L::pcz(q), a.nx, a.ny, a.nz);
      const T vp = (solid && solid[mp]) ? colour[m] : colour[mp];
      const T vm = (solid && solid[mm]) ? colour[m] : colour[mm];
      const T d = T(3.0 * L::w(L::pgrp(q))) * (vp - vm);
      if (L::pcx(q)) g[0] += L::pcx(q) * d;
      if (L::pcy(q)) g[1] += L::pcy(q) * d;
      if (L::pcz(q)) g[2] += L::pcz(q) * d;
    }
    const T gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    const bool ok = gn > T(a.grad_eps) && !(solid && solid[m]);
    for (int d = 0; d < 3; d++) normals[I(d) * N + m] = ok ? g[d] / gn : T(0);
  }
}

// F_rep at node (x, y, z) from the normal and colour fields (Eq. repForce); I: the
// caller's index type.
template <class L, class T, class I = long long>
__device__ __forceinline__ void rep_force(const T* __restrict__ normals, const T* __restrict__ colour,
                                          const uint8_t* __restrict__ solid, int x, int y, int z, const RepParams& a,
                                          T (&F)[3]) {
  F[0] = F[1] = F[2] = T(0);
  const I N = I(a.n);
  const I m = x + I(a.nx) * (y + I(a.ny) * z);
  const T n0 = normals[m], n1 = normals[N + m], n2 = normals[2 * N + m];
  if (n0 == T(0) && n1 == T(0) && n2 == T(0)) return;  // no normal at x
  T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int i = 1; i < L::Q; i++) {
    const I mm = wrap_index_t<I>(x + cx<L>(i), y + cy<L>(i), z + cz<L>(i), a.nx, a.ny, a.nz);
    if (solid && solid[mm]) continue;
    const T p0 = normals[mm], p1 = normals[N + mm], p2 = normals[2 * N + mm];
    const T nc = cx<L>(i) * n0 + cy<L>(i) * n1 + cz<L>(i) * n2;
    const T pc = cx<L>(i) * p0 + cy<L>(i) * p1 + cz<L>(i) * p2;
    if (-(nc * pc) > T(0)) {  // H(0) = 0; an undefined neighbour normal gives pc = 0
      const T il = grp<L>(i) == 1 ? T(1) : T(0.70710678118654752440);
      acc[0] += (nc * n0 + pc * p0) * il;
      acc[1] += (nc * n1 + pc * p1) * il;
      acc[2] += (nc * n2 + pc * p2) * il;
    }
  }
  const T c = colour[m];
  const T base = a.psi_kind ? T(1) + fabs(c) : T(1) - fabs(c);
  // outward (repulsive, Sec. 2.3): the printed sum points toward the rho^N extremum
  const T s = -T(a.pi) * fpow<T>(base, T(a.chi));
  for (int d = 0; d < 3; d++) F[d] = s * acc[d];
}

}  // namespace lbm
