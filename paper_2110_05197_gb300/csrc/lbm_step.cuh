// Fused per-timestep kernels of the two-component lattice Boltzmann step.
//
// One launch performs one full step for every node: moments, the non-local stencil
// (colour / density gradients for CG, pseudopotential or cross force for SC), collision and
// streaming.  Populations are structure-of-arrays [k][i][node] holding the post-streaming
// state; the kernel reads time t from `fin` (own node, coalesced) and pushes post-collision
// values to the neighbours' slots in `fout` (two-lattice A/B scheme).
//
// Storage as deviations.  A stored population is g^k_i(x) = f^k_i(x) - phi^k_i q_k(x), where
// q_k is the density of component k at x one step earlier, kept in a reference field
// (double-buffered like the populations; phi^k_i = the rest-state equilibrium weight, Eq. phi
// for CG, w_i for SC).  The writer knows q at the destination from its staged stencil and
// the reader reads its own q, both the same stored value, so the shift is exactly
// reversible; stored values are the small non-equilibrium and velocity parts instead of
// O(0.1) populations, which keeps FP32 (and 16-bit) storage accurate.  The density update
// rho = q + sum_i g_i is done with an exact rounding-error term (TwoSum).
//
// The stencils need scalar fields (densities, colour, psi) of the time-t state at the 18
// neighbours.  A block owns a TX x TY column of nodes and marches through a chunk of z
// planes.  For every plane it stages those fields on the (TX+2) x (TY+2) extended plane in
// shared memory, recomputing the ring nodes' densities from their populations (the
// neighbouring blocks' own reads, served by L2), so no gradient or force field is stored:
// a step moves 2*K*Q populations plus 2*K reference densities per node.  Interior
// populations read during staging stay in shared memory for that plane's collision; three
// field planes rotate (z-1, z, z+1).
//
// Model passages: CG Sec. 2.2 (Eqs. equiliCG, phi, tensorG, interpVisc, effRelax,
// perturbationOp, recoloringOpR/B, cosphi, streaming) with forces by Guo (Eqs. guoforce,
// source); SC Sec. 2.1 (Eqs. interactionforceMP, pseudopotential, guoforce2, source,
// collisSC, equiliSC; two-component cross force Eq. doublebeltrepulsionforce2).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "lbm_lattice.cuh"
#include "lbm_rep.cuh"

namespace lbm {

enum Model : int { kCG = 0, kSCMP = 1, kSC2C = 2, kSCMR = 3 };

// Step parameters, converted to the compute type on the host.
template <class T>
struct StepParams {
  int nx, ny, nz;
  int ncx, ncol;          // block columns along x, and in total (ncx * columns along y)
  int nchunks;            // z-chunks per column
  int nblk;               // blocks in the grid (WorkRange)
  long long n;            // nodes
  T phi[2][3];            // rest-state weights per component and group (CG: Eq. phi; SC: w)
  // CG
  T inv_nu_r, inv_nu_b;   // 1/nu_k, nu_k = (tau_k - 1/2)/3
  T A, beta, grad_eps;
  T inv_rho_r0, inv_rho_b0;
  int enhanced, color_norm;
  // SC
  T G, rho0, inv_rho0;    // multiphase: G, rho_0; two-component: G_eff = G/rho0^2 in G
  T Ga[2], Gr[2];         // multirange: attractive / repulsive self-couplings per species
  T omega_r, omega_b;     // 1/tau_k (SC)
  // forces
  T body[3];
  int has_body;
};

template <int MODEL>
struct ModelTraits;
template <>
struct ModelTraits<kCG> {
  static constexpr int K = 2;   // population sets
  static constexpr int NF = 2;  // staged fields: rho (total), rho^N
};
template <>
struct ModelTraits<kSCMP> {
  static constexpr int K = 1;
  static constexpr int NF = 1;  // psi
};
template <>
struct ModelTraits<kSC2C> {
  static constexpr int K = 2;
  static constexpr int NF = 2;  // rho_1, rho_2
};
template <>
struct ModelTraits<kSCMR> {
  static constexpr int K = 2;
  static constexpr int NF = 4;  // rho_1, rho_2, Psi_1, Psi_2
};

// ---- storage conversions ----
template <class S, class T>
__device__ __forceinline__ T ld_s(S v) { return T(v); }
template <>
__device__ __forceinline__ float ld_s<__half, float>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float ld_s<__nv_bfloat16, float>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <class S, class T>
__device__ __forceinline__ S st_s(T v) { return S(v); }
template <>
__device__ __forceinline__ __half st_s<__half, float>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 st_s<__nv_bfloat16, float>(float v) { return __float2bfloat16_rn(v); }

__device__ __forceinline__ float fexp(float x) { return expf(x); }
__device__ __forceinline__ double fexp(double x) { return exp(x); }
__device__ __forceinline__ float fsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double fsqrt(double x) { return sqrt(x); }
// correctly rounded reciprocal (cheaper than a full division in FP32)
__device__ __forceinline__ float frcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double frcp(double x) { return 1.0 / x; }

__host__ __device__ __forceinline__ int wrap(int v, int n) {
  int r = v % n;
  return r < 0 ? r + n : r;
}

// s = fl(a + b) and the exact rounding error e = (a + b) - s (Knuth's TwoSum).
template <class T>
__device__ __forceinline__ T two_sum(T a, T b, T& e) {
  const T s = a + b;
  const T bb = s - a;
  e = (a - (s - bb)) + (b - bb);
  return s;
}

// Work partition.  The lattice is cut into ncol block columns (tiles of TX x TY nodes,
// all of z) and every column's nz planes into nchunks z-chunks of near-equal length; a
// work unit is one (chunk, column) pair, numbered u = chunk * ncol + col.  Block b takes the
// units b, b + nblk, b + 2 nblk, ...: with nblk = ncol * nchunks (one unit per block) the
// hardware runs them in waves, with nblk = the resident block count (a persistent grid)
// every block loops.  Either way the blocks running at one time hold consecutive units,
// i.e. neighbouring columns at the same z, so the halo rows one block reads were just
// read (and are still in L2) for its neighbour.  A unit is marched with its own halo planes.
struct Segment {
  int col, z0, z1;  // column and z range [z0, z1)
};
struct WorkRange {
  int next, end, stride, ncol, nz, nchunks;
  __device__ WorkRange(int b, int nblk, int ncol_, int nz_, int nchunks_)
      : next(b), end(ncol_ * nchunks_), stride(nblk), ncol(ncol_), nz(nz_), nchunks(nchunks_) {}
  __device__ bool pop(Segment& s) {
    if (next >= end) return false;
    const int chunk = next / ncol;
    s.col = next - chunk * ncol;
    s.z0 = (int)(((long long)chunk * nz) / nchunks);
    s.z1 = (int)(((long long)(chunk + 1) * nz) / nchunks);
    next += stride;
    return true;
  }
};

// Scalar fields staged for the stencils from the component densities of one node.
template <int MODEL, class T>
__device__ __forceinline__ void node_fields(const StepParams<T>& p, T s0, T s1, T* out) {
  if constexpr (MODEL == kCG) {
    // colour field rho^N (text after Eq. perturbationOp); color_norm scales by rho_k0
    T rho = s0 + s1;
    out[0] = rho;
    if (p.color_norm) {
      T a = s0 * p.inv_rho_r0, b = s1 * p.inv_rho_b0;
      out[1] = (a - b) * frcp(a + b);
    } else {
      out[1] = (s0 - s1) * frcp(rho);
    }
  } else if constexpr (MODEL == kSCMP) {
    out[0] = p.rho0 * (T(1) - fexp(-s0 * p.inv_rho0));  // Eq. pseudopotential
  } else if constexpr (MODEL == kSCMR) {
    out[0] = s0;
    out[1] = s1;
    out[2] = p.rho0 * (T(1) - fexp(-s0 * p.inv_rho0));  // Psi_s, Eq. pseudopotential per species
    out[3] = p.rho0 * (T(1) - fexp(-s1 * p.inv_rho0));
  } else {
    out[0] = s0;
    out[1] = s1;
  }
}

// Deviation sum over the Q directions as a fixed balanced tree (short dependency chain),
// used for every node so that a node's density is bitwise the same whichever kernel or
// block computes it.
template <int N, class T>
__device__ __forceinline__ T tree_sum(const T* v) {
  if constexpr (N == 1) {
    return v[0];
  } else {
    return tree_sum<N / 2, T>(v) + tree_sum<N - N / 2, T>(v + N / 2);
  }
}
template <class L, class T>
__device__ __forceinline__ T sum_q(const T* v) {
  return tree_sum<L::Q, T>(v);
}

// Per-node density bookkeeping of one component: the stored deviations g (relative to
// phi * r_old) become deviations G relative to phi * q with q = RT(rho), rho = r_old + sum g.
template <class T>
struct CompState {
  T rho;   // density, rounded to the compute precision
  T q;     // new reference density (the value written to the reference field)
  T dq;    // exact density minus q: (r_old + delta) - q, from the TwoSum error
  T d;     // change of reference: G_i = g_i + phi_i d with d = r_old - q = dq - delta
};

template <class L, class T, class RT>
__device__ __forceinline__ CompState<T> comp_state(const T* g, T r_old) {
  CompState<T> c;
  const T delta = sum_q<L, T>(g);
  T e1;
  const T rho = two_sum(r_old, delta, e1);  // rho + e1 == r_old + delta exactly
  c.rho = rho;
  c.q = T(RT(rho));
  c.dq = (rho - c.q) + e1;
  c.d = c.dq - delta;
  return c;
}

// ---------------------------------------------------------------------------------------
// CG collision (Eqs. BGK, perturbation, recoloring) for one node, on deviations.
//   g[K][Q]  : stored deviations at x, relative to phi^k r_old_k; overwritten with the
//              post-collision deviations relative to phi^k q_k(x)
//   nbr(f,i) : staged field f at neighbour i (walls already substituted)
// Both colours relax with the same omega_eff, so BGK acts on the total population with
// the summed equilibrium sum_k f^{k,eq}, whose enhanced part involves grad(rho_R + rho_B).
template <class L, class T, class NB>
__device__ __forceinline__ void cg_collide(const StepParams<T>& p, T (&g)[2][L::Q], const CompState<T>& cr,
                                           const CompState<T>& cb, const NB& nbr, const T (&Fx)[3]) {
  constexpr int Q = L::Q;
  // gradients of the total density and of rho^N: grad phi = 3 sum_i w_i phi(x+c_i) c_i,
  // summed as opposite-pair differences
  T gr[3] = {T(0), T(0), T(0)}, gn[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int q = 0; q < L::NP; q++) {
    const int i = 2 * q + 1, j = 2 * q + 2;
    const T wq = T(3.0 * L::w(L::pgrp(q)));
    const T dr = wq * (nbr(0, i) - nbr(0, j));
    const T dn = wq * (nbr(1, i) - nbr(1, j));
    if (L::pcx(q)) { gr[0] += L::pcx(q) * dr; gn[0] += L::pcx(q) * dn; }
    if (L::pcy(q)) { gr[1] += L::pcy(q) * dr; gn[1] += L::pcy(q) * dn; }
    if (L::pcz(q)) { gr[2] += L::pcz(q) * dr; gn[2] += L::pcz(q) * dn; }
  }
  const T rr = cr.rho, rb = cb.rho;
  const T rho = rr + rb;
  const T inv = frcp(rho);
  // total deviation relative to s_i = phi^R_i q_R + phi^B_i q_B
  T G[Q];
#pragma unroll
  for (int i = 0; i < Q; i++) {
    const int gi = grp<L>(i);
    G[i] = (g[0][i] + g[1][i]) + (p.phi[0][gi] * cr.d + p.phi[1][gi] * cb.d);
  }
  // momentum (Eq. totalMomentum2; the symmetric shift carries none) and the Guo-shifted
  // velocity (Eq. guoforce)
  T jm[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int q = 0; q < L::NP; q++) {
    const T dd = (g[0][2 * q + 1] + g[1][2 * q + 1]) - (g[0][2 * q + 2] + g[1][2 * q + 2]);
    if (L::pcx(q)) jm[0] += L::pcx(q) * dd;
    if (L::pcy(q)) jm[1] += L::pcy(q) * dd;
    if (L::pcz(q)) jm[2] += L::pcz(q) * dd;
  }
  // body force plus the extra (repulsion) force
  T F[3] = {Fx[0], Fx[1], Fx[2]};
  if (p.has_body) { F[0] += p.body[0]; F[1] += p.body[1]; F[2] += p.body[2]; }
  const bool forced = F[0] != T(0) || F[1] != T(0) || F[2] != T(0);
  T u[3];
#pragma unroll
  for (int a = 0; a < 3; a++) u[a] = (jm[a] + T(0.5) * F[a]) * inv;
  // Eq. interpVisc and Eq. effRelax: 1/nubar = (rho_R/nu_R + rho_B/nu_B)/rho
  const T nubar = rho * frcp(rr * p.inv_nu_r + rb * p.inv_nu_b);
  const T omega = T(2) * frcp(T(6) * nubar + T(1));
  const T en = p.enhanced ? nubar : T(0);
  const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const T ugr = u[0] * gr[0] + u[1] * gr[1] + u[2] * gr[2];
  const T uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
  const T kg = T(1) - T(0.5) * omega;
  const T gg = gn[0] * gn[0] + gn[1] * gn[1] + gn[2] * gn[2];
  const T gabs = fsqrt(gg);
  const bool hasg = gabs > p.grad_eps;
  const T Ag = hasg ? p.A * gabs : T(0);
  const T inv_g = hasg ? frcp(gabs) : T(0);
  const T inv_gg = inv_g * inv_g;
  const T cR = rr * inv;
  const T rec = p.beta * rr * rb * inv * inv;
  // Equilibrium relative to s: f^eq_i - s_i = sum_k phi^k_i (rho_k - q_k) + velocity and
  // enhanced parts, with rho_k - q_k = dq_k exact (a few ulps of the density)
  const T dR = cr.dq, dB = cb.dq;
  // per-group constants (group 1: axis, 2: diagonal)
  T c_rest[3], c_u2[3], c_uu[3], c_od[3], c_fe[3], c_rc[3], c_base[3], c_sev[3], c_sod[3];  // [0] unused
#pragma unroll
  for (int gi = 1; gi <= 2; gi++) {
    const T w = T(L::w(gi));
    const T phR = p.phi[0][gi], phB = p.phi[1][gi];
    c_rest[gi] = en * T(L::psi(gi)) * ugr + phR * dR + phB * dB - rho * w * T(1.5) * uu;  // even, u-independent of c
    c_u2[gi] = rho * w * T(4.5);
    c_uu[gi] = en * T(2.0 * L::xi(gi));
    c_od[gi] = rho * w * T(3);
    c_fe[gi] = rr * phR + rb * phB;                                        // f^eq|_{u=0}
    c_rc[gi] = rec * c_fe[gi] * inv_g * ((gi == 1) ? T(1) : T(0.70710678118654752440));
    c_base[gi] = (rr * phB * cb.q - rb * phR * cr.q) * inv;
    c_sev[gi] = w * kg;
    c_sod[gi] = w * kg * T(3);
  }
  // rest direction (cos phi_0 = 0, c_0 = 0)
  {
    const T eq = en * T(L::psi(0)) * ugr + rho * T(L::w(0)) * (T(-1.5) * uu) + p.phi[0][0] * dR + p.phi[1][0] * dB;
    T Gs = G[0] + omega * (eq - G[0]);
    if (forced) Gs += T(L::w(0)) * kg * (T(-3) * uF);
    Gs -= Ag * T(L::B(0));
    const T base = (rr * p.phi[1][0] * cb.q - rb * p.phi[0][0] * cr.q) * inv;
    const T gR = cR * Gs + base;
    g[0][0] = gR;
    g[1][0] = Gs - gR;
  }
  auto pairs = [&](auto with_force) {
    constexpr bool FORCE = decltype(with_force)::value;
#pragma unroll
    for (int q = 0; q < L::NP; q++) {
      const int i = 2 * q + 1, j = 2 * q + 2;
      const int gi = L::pgrp(q);
      const T cu = T(L::pcx(q)) * u[0] + T(L::pcy(q)) * u[1] + T(L::pcz(q)) * u[2];
      const T cg = T(L::pcx(q)) * gr[0] + T(L::pcy(q)) * gr[1] + T(L::pcz(q)) * gr[2];
      const T cn = T(L::pcx(q)) * gn[0] + T(L::pcy(q)) * gn[1] + T(L::pcz(q)) * gn[2];
      // Eq. equiliCG summed over colours, minus phi^k q_k: even and odd parts in c_i
      const T ev = c_rest[gi] + cu * (c_u2[gi] * cu + c_uu[gi] * cg);
      const T od = c_od[gi] * cu;
      // Eq. perturbationOp (A|grad rho^N| on the total), even in c_i
      const T pert = Ag * (T(L::w(gi)) * cn * cn * inv_gg - T(L::B(gi)));
      T Gsi = G[i] + omega * (ev + od - G[i]) + pert;
      T Gsj = G[j] + omega * (ev - od - G[j]) + pert;
      if constexpr (FORCE) {
        // Eq. source (Guo) with tau = 1/omega_eff: even and odd parts
        const T cF = T(L::pcx(q)) * F[0] + T(L::pcy(q)) * F[1] + T(L::pcz(q)) * F[2];
        const T sev = c_sev[gi] * (T(9) * cu * cF - T(3) * uF);
        const T sod = c_sod[gi] * cF;
        Gsi += sev + sod;
        Gsj += sev - sod;
      }
      // Eqs. recoloringOpR/B with cos(phi_i) = c_i.grad rho^N / (|c_i| |grad rho^N|) and
      // f^eq|_{u=0} = sum_k rho_k phi^k_i; red part relative to phi^R q_R
      const T rc = c_rc[gi] * cn;
      const T gRi = cR * Gsi + c_base[gi] + rc;
      const T gRj = cR * Gsj + c_base[gi] - rc;
      g[0][i] = gRi;
      g[1][i] = Gsi - gRi;
      g[0][j] = gRj;
      g[1][j] = Gsj - gRj;
    }
  };
  if (forced)
    pairs(std::true_type{});
  else
    pairs(std::false_type{});
}

// ---------------------------------------------------------------------------------------
// SC collisions (Eqs. collisSC, equiliSC, source) on deviations relative to w_i q.
template <class L, class T>
__device__ __forceinline__ void bgk_guo(const StepParams<T>& p, T (&g)[L::Q], const CompState<T>& c,
                                        const T (&u)[3], const T (&F)[3], T omega) {
  const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const T uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
  const T kg = T(1) - T(0.5) * omega;
  const T rho = c.rho;
  const T dq = c.dq;
  {
    const T w0 = T(L::w(0));
    const T G = g[0] + w0 * c.d;
    const T eq = w0 * dq + rho * w0 * (T(-1.5) * uu);
    g[0] = G + omega * (eq - G) + w0 * kg * (T(-3) * uF);
  }
#pragma unroll
  for (int q = 0; q < L::NP; q++) {
    const int i = 2 * q + 1, j = 2 * q + 2;
    const T w = T(L::w(L::pgrp(q)));
    const T cu = T(L::pcx(q)) * u[0] + T(L::pcy(q)) * u[1] + T(L::pcz(q)) * u[2];
    const T cF = T(L::pcx(q)) * F[0] + T(L::pcy(q)) * F[1] + T(L::pcz(q)) * F[2];
    const T ev = w * dq + rho * w * (T(4.5) * cu * cu - T(1.5) * uu);
    const T od = rho * w * T(3) * cu;
    const T sev = w * kg * (T(9) * cu * cF - T(3) * uF);
    const T sod = w * kg * T(3) * cF;
    const T Gi = g[i] + w * c.d, Gj = g[j] + w * c.d;
    g[i] = Gi + omega * (ev + od - Gi) + sev + sod;
    g[j] = Gj + omega * (ev - od - Gj) + sev - sod;
  }
}

template <class L, class T>
__device__ __forceinline__ void momentum(const T (&g)[L::Q], T (&jm)[3]) {
  jm[0] = jm[1] = jm[2] = T(0);
#pragma unroll
  for (int q = 0; q < L::NP; q++) {
    const T d = g[2 * q + 1] - g[2 * q + 2];
    if (L::pcx(q)) jm[0] += L::pcx(q) * d;
    if (L::pcy(q)) jm[1] += L::pcy(q) * d;
    if (L::pcz(q)) jm[2] += L::pcz(q) * d;
  }
}

// sum_i w_i phi(x + c_i) c_i over the staged field `fi` (pair differences)
template <class L, class T, class NB>
__device__ __forceinline__ void weighted_sum(const NB& nbr, int fi, T (&acc)[3]) {
  acc[0] = acc[1] = acc[2] = T(0);
#pragma unroll
  for (int q = 0; q < L::NP; q++) {
    const T d = T(L::w(L::pgrp(q))) * (nbr(fi, 2 * q + 1) - nbr(fi, 2 * q + 2));
    if (L::pcx(q)) acc[0] += L::pcx(q) * d;
    if (L::pcy(q)) acc[1] += L::pcy(q) * d;
    if (L::pcz(q)) acc[2] += L::pcz(q) * d;
  }
}

template <class L, class T, class NB>
__device__ __forceinline__ void scmp_collide(const StepParams<T>& p, T (&g)[1][L::Q], const CompState<T>& c,
                                             const NB& nbr) {
  T acc[3];
  weighted_sum<L, T>(nbr, 0, acc);
  const T psic = nbr(0, 0);
  T F[3];
#pragma unroll
  for (int a = 0; a < 3; a++) F[a] = -p.G * psic * acc[a] + (p.has_body ? p.body[a] : T(0));
  T jm[3];
  momentum<L, T>(g[0], jm);
  const T inv = frcp(c.rho);
  T u[3];
#pragma unroll
  for (int a = 0; a < 3; a++) u[a] = (jm[a] + T(0.5) * F[a]) * inv;
  bgk_guo<L, T>(p, g[0], c, u, F, p.omega_r);
}

template <class L, class T, class NB>
__device__ __forceinline__ void sc2c_collide(const StepParams<T>& p, T (&g)[2][L::Q], const CompState<T>& c1,
                                             const CompState<T>& c2, const NB& nbr) {
  const T r1 = c1.rho, r2 = c2.rho;
  const T rho = r1 + r2;
  const T inv = frcp(rho);
  T a1[3], a2[3];
  weighted_sum<L, T>(nbr, 1, a1);  // sum w_i rho_2(x+c_i) c_i
  weighted_sum<L, T>(nbr, 0, a2);  // sum w_i rho_1(x+c_i) c_i
  T F1[3], F2[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const T b = p.has_body ? p.body[a] : T(0);
    F1[a] = -p.G * r1 * a1[a] + b * r1 * inv;
    F2[a] = -p.G * r2 * a2[a] + b * r2 * inv;
  }
  T j1[3], j2[3];
  momentum<L, T>(g[0], j1);
  momentum<L, T>(g[1], j2);
  T u[3];
#pragma unroll
  for (int a = 0; a < 3; a++) u[a] = (j1[a] + j2[a] + T(0.5) * (F1[a] + F2[a])) * inv;
  bgk_guo<L, T>(p, g[0], c1, u, F1, p.omega_r);
  bgk_guo<L, T>(p, g[1], c2, u, F2, p.omega_b);
}

// Forcing weight p of a belt vector with |c|^2 = r2 (Eq. pweights).
__host__ __device__ constexpr double mr_weight(int r2) {
  return r2 == 1 ? 4.0 / 135.0
       : r2 == 2 ? 1.0 / 63.0
       : r2 == 3 ? 2.0 / 315.0
       : r2 == 4 ? 5.0 / 1512.0
       : r2 == 5 ? 1.0 / 945.0
       : r2 == 6 ? 1.0 / 1890.0
       : r2 == 8 ? 1.0 / 15120.0
                 : 0.0;
}

// sum_j p_j phi(x + e_j) e_j over belts 1 and 2 (the 92 non-zero integer vectors with
// |e|^2 <= 8), as 46 opposite-pair differences; far(fi, dx, dy, dz) reads the field fi.
template <class T, class FAR>
__device__ __forceinline__ void belt_sum(const FAR& far, int fi, T (&acc)[3]) {
  acc[0] = acc[1] = acc[2] = T(0);
#pragma unroll
  for (int dz = 0; dz <= 2; dz++)
#pragma unroll
    for (int dy = -2; dy <= 2; dy++)
#pragma unroll
      for (int dx = -2; dx <= 2; dx++) {
        const int r2 = dx * dx + dy * dy + dz * dz;
        const bool positive = dz > 0 || (dy > 0 || (dy == 0 && dx > 0));  // one of each pair
        if (r2 == 0 || r2 > 8 || mr_weight(r2) == 0.0 || !positive) continue;
        const T d = T(mr_weight(r2)) * (far(fi, dx, dy, dz) - far(fi, -dx, -dy, -dz));
        if (dx) acc[0] += T(dx) * d;
        if (dy) acc[1] += T(dy) * d;
        if (dz) acc[2] += T(dz) * d;
      }
}

// Multicomponent SC with multirange potentials (Eq. benziforces): per species s the
// attractive belt-1 force -G^a_s Psi_s sum_i w_i Psi_s(x+c_i) c_i (Eq.
// doublebeltattractiveforce), the repulsive belts-1+2 force -G^r_s Psi_s sum_j p_j
// Psi_s(x+e_j) e_j (Eq. doublebeltrepulsionforce) and the cross force of Eq.
// doublebeltrepulsionforce2; then BGK + Guo with the common velocity as sc2c_collide.
// Fields: 0 rho_1, 1 rho_2, 2 Psi_1, 3 Psi_2; nbr(fi, i) at the lattice neighbours,
// far(fi, dx, dy, dz) at any offset up to 2.
template <class L, class T, class NB, class FAR>
__device__ __forceinline__ void scmr_collide(const StepParams<T>& p, T (&g)[2][L::Q], const CompState<T>& c1,
                                             const CompState<T>& c2, const NB& nbr, const FAR& far) {
  const T r1 = c1.rho, r2 = c2.rho;
  const T rho = r1 + r2;
  const T inv = frcp(rho);
  T F[2][3];
#pragma unroll
  for (int s = 0; s < 2; s++) {
    T att[3], rep[3], crs[3];
    weighted_sum<L, T>(nbr, 2 + s, att);  // belt 1, w: Psi_s
    belt_sum<T>(far, 2 + s, rep);         // belts 1 + 2, p: Psi_s
    weighted_sum<L, T>(nbr, 1 - s, crs);  // belt 1, w: rho of the other species
    const T psic = nbr(2 + s, 0);
    const T rs = s == 0 ? r1 : r2;
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const T b = p.has_body ? p.body[a] : T(0);
      F[s][a] = -p.Ga[s] * psic * att[a] - p.Gr[s] * psic * rep[a] - p.G * rs * crs[a] + b * rs * inv;
    }
  }
  T j1[3], j2[3];
  momentum<L, T>(g[0], j1);
  momentum<L, T>(g[1], j2);
  T u[3];
#pragma unroll
  for (int a = 0; a < 3; a++) u[a] = (j1[a] + j2[a] + T(0.5) * (F[0][a] + F[1][a])) * inv;
  bgk_guo<L, T>(p, g[0], c1, u, F[0], p.omega_r);
  bgk_guo<L, T>(p, g[1], c2, u, F[1], p.omega_b);
}

// ---------------------------------------------------------------------------------------
// The fused step kernel.  blockDim = (TX, TY); a 1-D grid of p.nblk blocks, each marching
// the segments of its work range (WorkRange).  Dynamic shared memory: step_smem_bytes().
template <class L>
__host__ __device__ constexpr int planes_of() { return L::D == 3 ? 3 : 1; }

template <class L, class T, int MODEL, bool WALLS>
__host__ size_t step_smem_bytes(int tx, int ty) {
  constexpr int K = ModelTraits<MODEL>::K, NF = ModelTraits<MODEL>::NF;
  constexpr int NPL = planes_of<L>();
  const size_t ne = size_t(tx + 2) * (ty + 2), ni = size_t(tx) * ty;
  size_t b = NPL * (NF + K) * ne * sizeof(T) + 2 * K * (L::Q + 1) * ni * sizeof(T);
  if (WALLS) b += NPL * ne;
  return (b + 15) & ~size_t(15);
}

template <class T>
__host__ __device__ constexpr int min_blocks() { return sizeof(T) == 8 ? 1 : 2; }

// Population and reference arrays of one step: the state at t (in) and at t+1 (out).
template <class S, class RT>
struct StepArrays {
  const S* __restrict__ fin;
  S* __restrict__ fout;
  const RT* __restrict__ rin;
  RT* __restrict__ rout;
  const uint8_t* __restrict__ solid;
};

// March one work unit (column sg.col, planes [sg.z0, sg.z1)) of a lattice through a full
// step with the block's TX x TY threads; smem_raw holds step_smem_bytes() bytes.  Ends with
// a block barrier, so the caller may reuse shared memory right away.
// REP (CG only): add the repulsion force of Eq. repForce from the pre-pass fields
// colour / normals (lbm_rep.cuh).  I: the integer type of node and array indices, int
// when K * Q * N < 2^31 (the launcher's choice), else long long.
template <class L, class T, class S, class RT, int MODEL, bool WALLS, bool REP, class I = long long>
__device__ __forceinline__ void march_segment(const StepArrays<S, RT>& a, const StepParams<T>& p,
                                              const T* __restrict__ colour, const T* __restrict__ normals,
                                              const RepParams& rp, const Segment& sg,
                                              unsigned char* __restrict__ smem_raw) {
  constexpr int Q = L::Q;
  constexpr int K = ModelTraits<MODEL>::K, NF = ModelTraits<MODEL>::NF;
  constexpr int NPL = planes_of<L>();
  constexpr int NV = NF + K;  // staged values per ext node: fields, then reference q_k
  const S* __restrict__ fin = a.fin;
  S* __restrict__ fout = a.fout;
  const RT* __restrict__ rin = a.rin;
  RT* __restrict__ rout = a.rout;
  const uint8_t* __restrict__ solid = a.solid;

  const int TX = blockDim.x, TY = blockDim.y;
  const int EX = TX + 2;
  const int NE = EX * (TY + 2), NI = TX * TY;
  const int tid = threadIdx.y * TX + threadIdx.x;
  const I N = I(p.n);
  const int x0 = (sg.col % p.ncx) * TX, y0 = (sg.col / p.ncx) * TY;

  T* fld = reinterpret_cast<T*>(smem_raw);           // [NPL][NV][NE]
  T* pops = fld + NPL * NV * NE;                     // [2][K*Q][NI] deviations
  T* rold = pops + 2 * K * Q * NI;                   // [2][K][NI] old reference densities
  uint8_t* msk = reinterpret_cast<uint8_t*>(rold + 2 * K * NI);  // [NPL][NE]

  // Stage plane z (periodic) into slot `sl`; keep interior deviations in buffer `pb` when
  // pb >= 0.
  auto stage = [&](int z, int sl, int pb) {
    const int gz = wrap(z, p.nz);
    for (int e = tid; e < NE; e += NI) {
      const int ey = e / EX, ex = e - ey * EX;
      const int gx = wrap(x0 - 1 + ex, p.nx), gy = wrap(y0 - 1 + ey, p.ny);
      const I n = gx + I(p.nx) * (gy + I(p.ny) * gz);
      const bool inner = pb >= 0 && ex >= 1 && ex <= TX && ey >= 1 && ey <= TY;
      const int ii = (ey - 1) * TX + (ex - 1);
      T rho[2] = {T(0), T(0)};
#pragma unroll
      for (int k = 0; k < K; k++) {
        T v[Q];
#pragma unroll
        for (int i = 0; i < Q; i++) v[i] = ld_s<S, T>(fin[I(k * Q + i) * N + n]);
        const T r_old = T(rin[I(k) * N + n]);
        const CompState<T> c = comp_state<L, T, RT>(v, r_old);
        rho[k] = c.rho;
        fld[(sl * NV + NF + k) * NE + e] = c.q;
        if (inner) {
#pragma unroll
          for (int i = 0; i < Q; i++) pops[(pb * K * Q + k * Q + i) * NI + ii] = v[i];
          rold[(pb * K + k) * NI + ii] = r_old;
        }
      }
      T out[2];
      node_fields<MODEL, T>(p, rho[0], rho[1], out);
#pragma unroll
      for (int f = 0; f < NF; f++) fld[(sl * NV + f) * NE + e] = out[f];
      if (WALLS) msk[sl * NE + e] = solid[n];
    }
  };

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int e0 = (ty + 1) * EX + (tx + 1);
  const int gx = x0 + tx, gy = y0 + ty;
  const bool valid = gx < p.nx && gy < p.ny;
  const int xm = gx == 0 ? p.nx - 1 : gx - 1, xp = gx + 1 >= p.nx ? 0 : gx + 1;
  const int ym = gy == 0 ? p.ny - 1 : gy - 1, yp = gy + 1 >= p.ny ? 0 : gy + 1;

  auto collide = [&](int z, int slm, int sl0, int slp, int pb) {
    if (!valid) return;
    if (WALLS && msk[sl0 * NE + e0]) return;
    T g[K][Q];
    CompState<T> cs[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
#pragma unroll
      for (int i = 0; i < Q; i++) g[k][i] = pops[(pb * K * Q + k * Q + i) * NI + tid];
      cs[k] = comp_state<L, T, RT>(g[k], rold[(pb * K + k) * NI + tid]);
    }
    auto slot_of = [&](int czv) { return czv == 0 ? sl0 : (czv > 0 ? slp : slm); };
    auto nbr = [&](int fi, int i) -> T {
      const int sl = slot_of(cz<L>(i));
      const int e = e0 + cy<L>(i) * EX + cx<L>(i);
      if (WALLS && msk[sl * NE + e]) return fld[(sl0 * NV + fi) * NE + e0];
      return fld[(sl * NV + fi) * NE + e];
    };
    if constexpr (MODEL == kCG) {
      T Fx[3] = {T(0), T(0), T(0)};
      if constexpr (REP) rep_force<L, T, I>(normals, colour, WALLS ? solid : nullptr, gx, gy, z, rp, Fx);
      cg_collide<L, T>(p, g, cs[0], cs[1], nbr, Fx);
    } else if constexpr (MODEL == kSCMP) {
      scmp_collide<L, T>(p, g, cs[0], nbr);
    } else {
      sc2c_collide<L, T>(p, g, cs[0], cs[1], nbr);
    }
    // new reference densities of this node
    const int zz = z, zm = zz == 0 ? p.nz - 1 : zz - 1, zpp = zz + 1 >= p.nz ? 0 : zz + 1;
    const I n0 = gx + I(p.nx) * (gy + I(p.ny) * zz);
#pragma unroll
    for (int k = 0; k < K; k++) rout[I(k) * N + n0] = RT(cs[k].q);
    // push to y = x + c_i (periodic), re-referenced to phi_i q(y); halfway bounce-back to
    // x, direction opp(i), at walls
#pragma unroll
    for (int i = 0; i < Q; i++) {
      const int dxv = cx<L>(i), dyv = cy<L>(i), dzv = cz<L>(i);
      const int X = dxv == 0 ? gx : (dxv > 0 ? xp : xm);
      const int Y = dyv == 0 ? gy : (dyv > 0 ? yp : ym);
      const int Z = dzv == 0 ? zz : (dzv > 0 ? zpp : zm);
      I nd = X + I(p.nx) * (Y + I(p.ny) * Z);
      int id = i;
      const int sl = slot_of(dzv);
      const int ed = e0 + dyv * EX + dxv;
      bool bounce = false;
      if (WALLS && i != 0) {
        if (msk[sl * NE + ed]) {
          nd = n0;
          id = opp<L>(i);
          bounce = true;
        }
      }
#pragma unroll
      for (int k = 0; k < K; k++) {
        T v = g[k][i];
        if (i != 0 && !bounce) v += p.phi[k][grp<L>(i)] * (cs[k].q - fld[(sl * NV + NF + k) * NE + ed]);
        fout[I(k * Q + id) * N + nd] = st_s<S, T>(v);
      }
    }
  };

  const int z0 = sg.z0, z1 = sg.z1;
  if constexpr (NPL == 3) {
    stage(z0 - 1, 0, -1);
    stage(z0, 1, 0);
    for (int z = z0; z < z1; z++) {
      const int r = z - z0;
      const int slm = r % 3, sl0 = (r + 1) % 3, slp = (r + 2) % 3;
      stage(z + 1, slp, (z + 1 < z1) ? ((r + 1) & 1) : -1);
      __syncthreads();
      collide(z, slm, sl0, slp, r & 1);
      __syncthreads();
    }
  } else {
    for (int z = z0; z < z1; z++) {
      stage(z, 0, 0);
      __syncthreads();
      collide(z, 0, 0, 0, 0);
      __syncthreads();
    }
  }
}

template <class L, class T, class S, class RT, int MODEL, bool WALLS, bool REP, class I = long long>
__global__ void __launch_bounds__(256, min_blocks<T>()) step_kernel(
    const S* __restrict__ fin, S* __restrict__ fout, const RT* __restrict__ rin, RT* __restrict__ rout,
    const uint8_t* __restrict__ solid, const int* __restrict__ status, const __grid_constant__ StepParams<T> p,
    const T* __restrict__ colour, const T* __restrict__ normals, const __grid_constant__ RepParams rp) {
  if (status != nullptr && *status != 0) return;  // blown-up state: stop stepping
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const StepArrays<S, RT> a{fin, fout, rin, rout, solid};
  WorkRange work(blockIdx.x, p.nblk, p.ncol, p.nz, p.nchunks);
  Segment sg;
  while (work.pop(sg)) march_segment<L, T, S, RT, MODEL, WALLS, REP, I>(a, p, colour, normals, rp, sg, smem_raw);
}

}  // namespace lbm
