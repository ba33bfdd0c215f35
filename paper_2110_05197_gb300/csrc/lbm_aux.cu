// Auxiliary kernels: equilibrium initialisation, checkpoint import/export of populations,
// and the FP64 moment / diagnostics reductions (mass, momentum, E_kin, max|u|, blow-up).
//
// Populations are stored as deviations g^k_i = f^k_i - phi^k_i r_k from the rest-state
// equilibrium of a per-node reference density r_k (see lbm_step.cuh); every kernel here
// reconstructs f in FP64 as g + phi r.
#include <cmath>
#include <type_traits>

#include "lbm_launch.cuh"

namespace lbm {

namespace {

__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return (double)v; }
__device__ __forceinline__ double to_d(__half v) { return (double)__half2float(v); }
__device__ __forceinline__ double to_d(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
template <class S>
__device__ __forceinline__ S from_d(double v);
template <>
__device__ __forceinline__ double from_d<double>(double v) { return v; }
template <>
__device__ __forceinline__ float from_d<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ __half from_d<__half>(double v) { return __float2half_rn((float)v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double v) { return __float2bfloat16_rn((float)v); }

// Index of the periodic neighbour (x + dx, y + dy, z + dz) in index type I.
template <class I>
__device__ __forceinline__ I nb_index_t(int x, int y, int z, int dx, int dy, int dz, int nx, int ny, int nz) {
  x += dx;
  y += dy;
  z += dz;
  x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
  y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
  z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
  return x + I(nx) * (y + I(ny) * z);
}

struct AuxParams {
  int nx, ny, nz;
  long long n;
  int model, enhanced, K;
  double phi[2][3];      // rest-state weights per component and group
  double nu_r, nu_b;
  double G, rho0;        // SC two-component: G = G_eff
  double body[3];
  double umax, neg_tol;
  double Ga[2], Gr[2];   // multirange SC self-couplings
  int aa;                // in-place streaming: the state's layout parity is its buffer index
};

AuxParams aux_params(const lbm_ctx* c) {
  const lbm_params& q = c->p;
  AuxParams a{};
  a.nx = q.nx;
  a.ny = q.ny;
  a.nz = q.nz;
  a.n = c->N;
  a.aa = c->aa;
  a.model = q.model;
  a.enhanced = q.enhanced_eq;
  a.K = c->K;
  rest_weights(q, a.phi);
  a.nu_r = (q.tau_r - 0.5) / 3.0;
  a.nu_b = (q.tau_b - 0.5) / 3.0;
  a.G = (q.model == LBM_MODEL_SC_2C || q.model == LBM_MODEL_SC_MR) ? q.G / (q.rho0_psi * q.rho0_psi) : q.G;
  for (int k = 0; k < 2; k++) {
    a.Ga[k] = q.Ga[k];
    a.Gr[k] = q.Gr[k];
  }
  a.rho0 = q.rho0_psi;
  for (int d = 0; d < 3; d++) a.body[d] = q.body_force[d];
  a.umax = q.umax_unstable > 0 ? q.umax_unstable : 0.5;
  double scale = 1.0;
  if (q.model == LBM_MODEL_CG) scale = fmax(scale, fmax(q.rho_r0, q.rho_b0));
  a.neg_tol = kNegDensityTol * scale;
  return a;
}

// The buffer pair holding the current state: the host's index, or the pair frozen by a
// tripped blow-up check (the host cannot know when that happened).
__device__ __forceinline__ int state_index(const lbm_diag* d, int cur) { return d->status ? d->trip_buf : cur; }

// Compute type of the step for a storage type: per-node arithmetic of the auxiliary
// kernels runs in it (FP64 only for FP64 storage); sums over the lattice stay FP64.
template <class S>
using step_t = typename std::conditional<std::is_same<S, double>::value, double, float>::type;

// Sum of values of the compute type C whose FP64 result is as accurate as FP64 summation.
// For C = float the sum is carried as an unevaluated pair s + c and the rounding error of
// every addition is kept exactly (TwoSum), at FP32 cost: GB300's FP64 rate is a small
// fraction of its FP32 rate, and the reductions here would otherwise be FP64 bound.
template <class C>
struct ExactSum;
template <>
struct ExactSum<double> {
  double s = 0.0;
  __device__ explicit ExactSum(double v = 0.0) : s(v) {}
  __device__ void add(double v) { s += v; }
  __device__ double value() const { return s; }
};
template <>
struct ExactSum<float> {
  float s = 0.f, c = 0.f;
  __device__ explicit ExactSum(float v = 0.f) : s(v) {}
  __device__ void add(float v) {
    float e;
    s = two_sum(s, v, e);
    c += e;
  }
  __device__ double value() const { return double(s) + double(c); }
};

// x, y, z of node n
__device__ __forceinline__ void node_xyz(long long n, const AuxParams& a, int& x, int& y, int& z) {
  node_coords(n, a.nx, a.ny, a.n, x, y, z);
}

// 3 sum_i w_i phi(x + c_i) c_i with a wall neighbour replaced by the centre value.
template <class L, class C, class E, class I>
__device__ void grad_c(const E* phi, const uint8_t* solid, I n, int x, int y, int z, const AuxParams& a, C g[3]) {
  g[0] = g[1] = g[2] = C(0);
#pragma unroll
  for (int q = 0; q < L::NP; q++) {
    const int i = 2 * q + 1;
    const I mp = nb_index_t<I>(x, y, z, cx<L>(i), cy<L>(i), cz<L>(i), a.nx, a.ny, a.nz);
    const I mm = nb_index_t<I>(x, y, z, -cx<L>(i), -cy<L>(i), -cz<L>(i), a.nx, a.ny, a.nz);
    const C vp = C((solid && solid[mp]) ? phi[n] : phi[mp]);
    const C vm = C((solid && solid[mm]) ? phi[n] : phi[mm]);
    const C d = C(3.0 * L::w(L::pgrp(q))) * (vp - vm);
    g[0] += C(L::pcx(q)) * d;
    g[1] += C(L::pcy(q)) * d;
    g[2] += C(L::pcz(q)) * d;
  }
}

// Eq. equiliCG for one colour (phi from Eq. phi, enhanced part optional) or Eq. equiliSC
// (phi = w, no enhanced part), minus phi_i * rref, into out[Q]; drho = rho_k - rref (exact
// in FP64, then rounded), so every term is a small deviation.
template <class L, class C>
__device__ void feq_dev(C rho_k, const double* phi, C nubar_en, const C u[3], const C g[3], C drho, C* out) {
  const C uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const C ug = u[0] * g[0] + u[1] * g[1] + u[2] * g[2];
  for (int i = 0; i < L::Q; i++) {
    const int gr = grp<L>(i);
    const C cu = C(cx<L>(i)) * u[0] + C(cy<L>(i)) * u[1] + C(cz<L>(i)) * u[2];
    const C cgr = C(cx<L>(i)) * g[0] + C(cy<L>(i)) * g[1] + C(cz<L>(i)) * g[2];
    const C w = C(L::w(gr));
    const C enh = nubar_en * (C(L::psi(gr)) * ug + C(2.0 * L::xi(gr)) * cu * cgr);
    out[i] = enh + C(phi[gr]) * drho + rho_k * w * (C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu);
  }
}

// Both component densities rounded to the compute type: out[k][n] = C(rho_k[n]).
template <class C>
__global__ void to_compute_kernel(const double* __restrict__ rr, const double* __restrict__ rb, C* __restrict__ out,
                                  long long n) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < n; m += (long long)gridDim.x * blockDim.x) {
    out[m] = C(rr[m]);
    out[n + m] = C(rb[m]);
  }
}

template <class L, class S, class RT, class I>
__global__ void init_eq_kernel(S* __restrict__ fa, S* __restrict__ fb, RT* __restrict__ ra, RT* __restrict__ rb_,
                               const double* __restrict__ rr, const double* __restrict__ rb,
                               const double* __restrict__ U, const uint8_t* __restrict__ solid,
                               const step_t<S>* __restrict__ fc, AuxParams a) {
  using C = step_t<S>;
  const I N = I(a.n);
  for (I n = blockIdx.x * I(blockDim.x) + threadIdx.x; n < N; n += I(gridDim.x) * blockDim.x) {
    C out[L::Q];
    if (solid && solid[n]) {
      for (int k = 0; k < a.K; k++) {
        ra[I(k) * N + n] = RT(0);
        if (rb_) rb_[I(k) * N + n] = RT(0);
        for (int i = 0; i < L::Q; i++) {
          fa[I(k * L::Q + i) * N + n] = from_d<S>(0.0);
          if (fb) fb[I(k * L::Q + i) * N + n] = from_d<S>(0.0);
        }
      }
      continue;
    }
    int x, y, z;
    node_xyz(n, a, x, y, z);
    C u[3] = {C(0), C(0), C(0)};
    if (U) {
      u[0] = C(U[n]);
      u[1] = C(U[N + n]);
      u[2] = C(U[2 * N + n]);
    }
    C en = C(0);
    if (a.model == LBM_MODEL_CG && a.enhanced) {
      const C r = fc ? fc[n] : C(rr[n]), b = fc ? fc[N + n] : C(rb[n]), rho = r + b;
      en = C(1) / ((r / rho) / C(a.nu_r) + (b / rho) / C(a.nu_b));  // Eq. interpVisc
    }
    // Only pair 0 is written for fluid nodes: the first step writes every population and
    // reference density of every fluid node of pair 1.
    for (int k = 0; k < a.K; k++) {
      const double* phi = k == 0 ? rr : rb;
      const RT rref = RT(phi[n]);  // reference density: the initial density, rounded
      C g[3] = {C(0), C(0), C(0)};
      if (a.model == LBM_MODEL_CG) {
        if (fc)
          grad_c<L, C>(fc + I(k) * N, solid, n, x, y, z, a, g);
        else
          grad_c<L, C>(phi, solid, n, x, y, z, a, g);
      }
      feq_dev<L, C>(C(phi[n]), a.phi[k], en, u, g, C(phi[n] - (double)rref), out);
      ra[I(k) * N + n] = rref;
      for (int i = 0; i < L::Q; i++) {
        fa[I(k * L::Q + i) * N + n] = st_s<S, C>(out[i]);
      }
    }
  }
}

__global__ void restore_acc_kernel(const double* __restrict__ plane, double* __restrict__ acc, long long n, bool first) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < n; m += (long long)gridDim.x * blockDim.x)
    acc[m] = first ? plane[m] : acc[m] + plane[m];
}

template <class S, class RT>
__global__ void restore_plane_kernel(S* __restrict__ fa, S* __restrict__ fb, RT* __restrict__ ra,
                                     RT* __restrict__ rb_, const double* __restrict__ plane,
                                     const double* __restrict__ acc, const uint8_t* __restrict__ solid, long long n,
                                     long long off, long long roff, double phi, bool write_ref) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < n; m += (long long)gridDim.x * blockDim.x) {
    const bool wall = solid && solid[m];
    const RT r = wall ? RT(0) : RT(acc[m]);
    const S v = wall ? from_d<S>(0.0) : from_d<S>(plane[m] - phi * (double)r);
    fa[off + m] = v;
    if (fb) fb[off + m] = v;
    if (write_ref) {
      ra[roff + m] = r;
      if (rb_) rb_[roff + m] = r;
    }
  }
}

// canonical populations f = g + phi r, FP64; `out` holds planes [first_plane, first_plane+np);
// 0 on wall nodes (whose slots the in-place scheme uses for bounced populations)
template <class L, class S, class RT>
__global__ void export_kernel(const S* __restrict__ f0, const S* __restrict__ f1, const RT* __restrict__ r0,
                              const RT* __restrict__ r1, const lbm_diag* __restrict__ d, int cur, int first_plane,
                              int np, double* __restrict__ out, const uint8_t* __restrict__ solid, AuxParams a) {
  const int b = state_index(d, cur);
  const S* f = b ? f1 : f0;
  const RT* r = b ? r1 : r0;
  const bool odd = a.aa && (b & 1);
  const long long total = (long long)np * a.n;
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < total; m += (long long)gridDim.x * blockDim.x) {
    const int plane = first_plane + (int)(m / a.n);
    const long long node = m - (long long)(plane - first_plane) * a.n;
    const int k = plane / L::Q, i = plane - k * L::Q;
    out[m] = (solid && solid[node]) ? 0.0
                                    : to_d(f[aa_index_n<L>(k, i, node, a.nx, a.ny, a.nz, a.n, odd)]) +
                                          a.phi[k][grp<L>(i)] * to_d(r[(long long)k * a.n + node]);
  }
}

// stored plane (k, i) of the even layout from the odd in-place layout (0 on wall nodes)
template <class L, class S>
__global__ void aa_gather_kernel(const S* __restrict__ f, S* __restrict__ out, const uint8_t* __restrict__ solid,
                                 int k, int i, AuxParams a) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < a.n; m += (long long)gridDim.x * blockDim.x) {
    out[m] = (solid && solid[m]) ? from_d<S>(0.0) : f[aa_index_n<L>(k, i, m, a.nx, a.ny, a.nz, a.n, true)];
  }
}


// One pass over the populations: the component densities rr, rb (FP64, as exact as FP64
// summation), psi of Eq. pseudopotential (SC multiphase, FP64), the momentum
// j = sum_k sum_i c_i f^k_i into jm [3][N] (FP64), and for the multirange model the
// pseudopotentials Psi_s of both species in the step's compute type into mrpsi [2][N]
// (read 92 times per node by the diagnostics' belt sums).
template <class L, class S, class RT, class I>
__global__ void densities_kernel(const S* __restrict__ f0, const S* __restrict__ f1, const RT* __restrict__ r0,
                                 const RT* __restrict__ r1, const lbm_diag* __restrict__ d, int cur,
                                 double* __restrict__ rr, double* __restrict__ rb, double* __restrict__ psi,
                                 double* __restrict__ jm, step_t<S>* __restrict__ mrpsi, AuxParams a) {
  using C = step_t<S>;
  const int b = state_index(d, cur);
  const S* f = b ? f1 : f0;
  const RT* r = b ? r1 : r0;
  const bool odd = a.aa && (b & 1);
  const I N = I(a.n);
  for (I m = blockIdx.x * I(blockDim.x) + threadIdx.x; m < N; m += I(gridDim.x) * blockDim.x) {
    // momentum summed exactly (ExactSum): the colours' momenta nearly cancel at
    // interfaces, so rounding in the sum would show up in the reported u; the shift
    // phi_i r is symmetric in c_i and carries no momentum: opposite pairs of the stored
    // deviations
    ExactSum<C> jx, jy, jz;
    for (int k = 0; k < 2; k++) {
      double s = 0.0;
      if (k < a.K) {
        ExactSum<C> acc{static_cast<C>(r[I(k) * N + m])};  // sum_i phi_i = 1
#pragma unroll
        for (int i = 0; i < L::Q; i++)
          acc.add(ld_s<S, C>(f[aa_index_nt<L, I>(k, i, m, a.nx, a.ny, a.nz, N, odd)]));
        s = acc.value();
#pragma unroll
        for (int q = 0; q < L::NP; q++) {
          const C vp = ld_s<S, C>(f[aa_index_nt<L, I>(k, 2 * q + 1, m, a.nx, a.ny, a.nz, N, odd)]);
          const C vm = ld_s<S, C>(f[aa_index_nt<L, I>(k, 2 * q + 2, m, a.nx, a.ny, a.nz, N, odd)]);
          if (L::pcx(q)) { jx.add(L::pcx(q) > 0 ? vp : -vp); jx.add(L::pcx(q) > 0 ? -vm : vm); }
          if (L::pcy(q)) { jy.add(L::pcy(q) > 0 ? vp : -vp); jy.add(L::pcy(q) > 0 ? -vm : vm); }
          if (L::pcz(q)) { jz.add(L::pcz(q) > 0 ? vp : -vp); jz.add(L::pcz(q) > 0 ? -vm : vm); }
        }
      }
      (k == 0 ? rr : rb)[m] = s;
      // Eq. pseudopotential, once per node (the force stencil reads it 18 times)
      if (k == 0 && a.model == LBM_MODEL_SC_MP) psi[m] = a.rho0 * (1.0 - exp(-s / a.rho0));
      if (mrpsi) {  // Psi_s = rho_0 (1 - exp(-rho_s / rho_0)) in the compute type
        const C c0 = C(a.rho0), ic0 = C(1.0 / a.rho0);
        mrpsi[I(k) * N + m] = c0 * (C(1) - exp(-C(s) * ic0));
      }
    }
    jm[m] = jx.value();
    jm[N + m] = jy.value();
    jm[2 * N + m] = jz.value();
  }
}

// x is finite: its exponent field is not all ones (integer test of the high word; GB300
// runs FP64 compares at its low FP64 rate).
__device__ __forceinline__ bool finite_bits(double x) { return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000; }

// ---- fixed-order block reductions ----
struct Acc {
  double v[LBM_NTOTALS];
};
// slots: 0 mass_r 1 mass_b 2-4 mom 5 ekin 6 max|u| 7 nonfinite 8 min rr 9 min rb
__device__ __forceinline__ void acc_init(Acc& a) {
  for (int s = 0; s < LBM_NTOTALS; s++) a.v[s] = 0.0;
  a.v[8] = INFINITY;
  a.v[9] = INFINITY;
}
__device__ __forceinline__ void acc_merge(Acc& a, const Acc& b) {
  for (int s = 0; s < 6; s++) a.v[s] += b.v[s];
  a.v[6] = fmax(a.v[6], b.v[6]);
  a.v[7] += b.v[7];
  a.v[8] = fmin(a.v[8], b.v[8]);
  a.v[9] = fmin(a.v[9], b.v[9]);
}
__device__ void block_reduce(Acc& a) {
  __shared__ double sh[kDiagThreads / 32][LBM_NTOTALS];
  for (int off = 16; off > 0; off >>= 1) {
    Acc o;
    for (int s = 0; s < LBM_NTOTALS; s++) o.v[s] = __shfl_xor_sync(0xffffffffu, a.v[s], off);
    acc_merge(a, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    for (int s = 0; s < LBM_NTOTALS; s++) sh[warp][s] = a.v[s];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
      Acc o;
      for (int s = 0; s < LBM_NTOTALS; s++) o.v[s] = sh[w][s];
      acc_merge(a, o);
    }
  }
}

// Fixed-order reduction of the nblk block partials into the totals and the blow-up status
// (all threads of one block take part).
__device__ void reduce_partials(const double* partials, int nblk, lbm_diag* d, int cur, const AuxParams& a) {
  Acc acc;
  acc_init(acc);
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    Acc o;
    for (int s = 0; s < LBM_NTOTALS; s++) o.v[s] = __ldcg(&partials[b * LBM_NTOTALS + s]);
    acc_merge(acc, o);
  }
  block_reduce(acc);
  if (threadIdx.x == 0) {
    acc.v[6] = sqrt(acc.v[6]);  // max |u| from max |u|^2 (sqrt is monotonic and correctly rounded)
    int st = 0;
    if (acc.v[7] > 0 || !isfinite(acc.v[0]) || !isfinite(acc.v[1])) st |= 1;
    if (acc.v[8] < -a.neg_tol || acc.v[9] < -a.neg_tol) st |= 2;
    if (!(acc.v[6] <= a.umax)) st |= 4;
    for (int s = 0; s < LBM_NTOTALS; s++) d->totals[s] = acc.v[s];
    if (d->status == 0 && st != 0) d->trip_buf = cur;
    d->status |= st;
  }
}

// Per-node velocity and the block partials of the totals, from the staged densities and
// momentum (densities_kernel): no population is read again.  u (force-shifted, Eq.
// guoforce) may be written over jm (uo == jm): each node reads its own momentum first.
// Slot 6 of the partials holds max |u|^2 (its square root is taken in the final pass).
template <class L, class S, class RT>
__global__ void __launch_bounds__(kDiagThreads) diag_kernel(const double* __restrict__ rr,
                                                            const double* __restrict__ rb,
                                                            const double* __restrict__ psi,
                                                            const double* jm,
                                                            const step_t<S>* __restrict__ mrpsi,
                                                            const uint8_t* __restrict__ solid, double* uo,
                                                            double* __restrict__ partials, AuxParams a,
                                                            const step_t<S>* __restrict__ colour,
                                                            const step_t<S>* __restrict__ normals, RepParams rp,
                                                            lbm_diag* __restrict__ d, int cur) {
  using C = step_t<S>;  // per-node arithmetic of the multirange belts; the sums below are FP64
  Acc acc;
  acc_init(acc);
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < a.n; n += (long long)gridDim.x * blockDim.x) {
    const bool wall = solid && solid[n];
    const double j[3] = {jm[n], jm[a.n + n], jm[2 * a.n + n]};
    const double r = rr[n], b = rb[n], rho = r + b;
    const int bad = !(finite_bits(r) && finite_bits(b) && finite_bits(j[0]) && finite_bits(j[1]) && finite_bits(j[2]));
    double F[3] = {a.body[0], a.body[1], a.body[2]};
    if (!wall && a.model == LBM_MODEL_CG && normals) {
      int x, y, z;
      node_xyz(n, a, x, y, z);
      C Fr[3];
      rep_force<L, C>(normals, colour, solid, x, y, z, rp, Fr);  // the step's own precision
      for (int dd = 0; dd < 3; dd++) F[dd] += double(Fr[dd]);
    }
    if (!wall && a.model != LBM_MODEL_CG) {
      int x, y, z;
      node_xyz(n, a, x, y, z);
      // sum_i w_i phi(x + c_i) c_i as opposite-pair differences in FP64 (the force is a
      // small difference of O(1) values); neighbour indices in 32-bit arithmetic when the
      // node count allows it
      double s1[3] = {0.0, 0.0, 0.0}, s2[3] = {0.0, 0.0, 0.0};
      const double psic = a.model == LBM_MODEL_SC_MP ? psi[n] : 0.0;
      const bool small = a.n < (1LL << 31);
      const int xm = x == 0 ? a.nx - 1 : x - 1, xp = x + 1 == a.nx ? 0 : x + 1;
      const int ym = y == 0 ? a.ny - 1 : y - 1, yp = y + 1 == a.ny ? 0 : y + 1;
      const int zm = z == 0 ? a.nz - 1 : z - 1, zp = z + 1 == a.nz ? 0 : z + 1;
      auto nbi = [&](int dx, int dy, int dz) -> long long {
        const int X = dx == 0 ? x : (dx > 0 ? xp : xm);
        const int Y = dy == 0 ? y : (dy > 0 ? yp : ym);
        const int Z = dz == 0 ? z : (dz > 0 ? zp : zm);
        return small ? (long long)(unsigned)(X + a.nx * (Y + a.ny * Z))
                     : X + (long long)a.nx * (Y + (long long)a.ny * Z);
      };
#pragma unroll
      for (int q = 0; q < L::NP; q++) {
        const int i = 2 * q + 1;
        const long long mp = nbi(cx<L>(i), cy<L>(i), cz<L>(i));
        const long long mm = nbi(-cx<L>(i), -cy<L>(i), -cz<L>(i));
        const bool swp = solid && solid[mp], swm = solid && solid[mm];
        const double w = L::w(L::pgrp(q));
        double d1, d2 = 0.0;
        if (a.model == LBM_MODEL_SC_MP) {
          d1 = w * ((swp ? psic : psi[mp]) - (swm ? psic : psi[mm]));
        } else {
          d1 = w * ((swp ? b : rb[mp]) - (swm ? b : rb[mm]));
          d2 = w * ((swp ? r : rr[mp]) - (swm ? r : rr[mm]));
        }
        if (L::pcx(q)) { s1[0] += L::pcx(q) * d1; s2[0] += L::pcx(q) * d2; }
        if (L::pcy(q)) { s1[1] += L::pcy(q) * d1; s2[1] += L::pcy(q) * d2; }
        if (L::pcz(q)) { s1[2] += L::pcz(q) * d1; s2[2] += L::pcz(q) * d2; }
      }
      for (int dd = 0; dd < 3; dd++) {
        if (a.model == LBM_MODEL_SC_MP)
          F[dd] = -a.G * psic * s1[dd] + a.body[dd];
        else
          F[dd] = -a.G * r * s1[dd] - a.G * b * s2[dd] + a.body[dd];
      }
      if (a.model == LBM_MODEL_SC_MR) {
        // self forces of Eqs. doublebeltattractiveforce / doublebeltrepulsionforce with
        // the staged Psi_s, summed in the step's compute type C as the step kernel sums
        // them (FP64 only for FP64 storage); a wall neighbour takes the centre value
        const bool small = a.n < (1LL << 31);
        for (int sp = 0; sp < 2; sp++) {
          const C* ps = mrpsi + (long long)sp * a.n;
          const C pc = ps[n];
          auto psi_at = [&](int dx, int dy, int dz) -> C {
            int X = x + dx, Y = y + dy, Z = z + dz;
            X = X < 0 ? X + a.nx : (X >= a.nx ? X - a.nx : X);
            Y = Y < 0 ? Y + a.ny : (Y >= a.ny ? Y - a.ny : Y);
            Z = Z < 0 ? Z + a.nz : (Z >= a.nz ? Z - a.nz : Z);
            const long long m = small ? (long long)(unsigned)(X + a.nx * (Y + a.ny * Z))
                                      : X + (long long)a.nx * (Y + (long long)a.ny * Z);
            return (solid && solid[m]) ? pc : ps[m];
          };
          C att[3] = {C(0), C(0), C(0)}, rep[3] = {C(0), C(0), C(0)};
#pragma unroll
          for (int q = 0; q < L::NP; q++) {
            const C d = C(L::w(L::pgrp(q))) * (psi_at(L::pcx(q), L::pcy(q), L::pcz(q)) -
                                               psi_at(-L::pcx(q), -L::pcy(q), -L::pcz(q)));
            if (L::pcx(q)) att[0] += L::pcx(q) * d;
            if (L::pcy(q)) att[1] += L::pcy(q) * d;
            if (L::pcz(q)) att[2] += L::pcz(q) * d;
          }
#pragma unroll
          for (int dz = 0; dz <= 2; dz++)
#pragma unroll
            for (int dy = -2; dy <= 2; dy++)
#pragma unroll
              for (int dx = -2; dx <= 2; dx++) {
                const int r2 = dx * dx + dy * dy + dz * dz;
                if (r2 == 0 || r2 > 8 || mr_weight(r2) == 0.0 || !(dz > 0 || dy > 0 || (dy == 0 && dx > 0))) continue;
                const C d = C(mr_weight(r2)) * (psi_at(dx, dy, dz) - psi_at(-dx, -dy, -dz));
                if (dx) rep[0] += C(dx) * d;
                if (dy) rep[1] += C(dy) * d;
                if (dz) rep[2] += C(dz) * d;
              }
          for (int dd = 0; dd < 3; dd++)
            F[dd] += -a.Ga[sp] * double(pc) * double(att[dd]) - a.Gr[sp] * double(pc) * double(rep[dd]);
        }
      }
    }
    double u[3] = {0.0, 0.0, 0.0};
    if (!wall) {
      const double inv = 1.0 / rho;
      for (int dd = 0; dd < 3; dd++) u[dd] = (j[dd] + 0.5 * F[dd]) * inv;
    }
    if (uo) {
      uo[n] = u[0];
      uo[a.n + n] = u[1];
      uo[2 * a.n + n] = u[2];
    }
    if (wall) continue;
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    acc.v[0] += r;
    acc.v[1] += b;
    acc.v[2] += j[0];
    acc.v[3] += j[1];
    acc.v[4] += j[2];
    acc.v[5] += 0.5 * rho * uu;
    acc.v[6] = fmax(acc.v[6], uu);
    acc.v[7] += bad;
    acc.v[8] = fmin(acc.v[8], r);
    acc.v[9] = fmin(acc.v[9], b);
  }
  block_reduce(acc);
  // The block that finishes last reduces every block's partial (in block order, whatever
  // the finishing order): partial written, fence, count; the counter goes back to 0.
  __shared__ bool last;
  if (threadIdx.x == 0) {
    for (int s = 0; s < LBM_NTOTALS; s++) partials[blockIdx.x * LBM_NTOTALS + s] = acc.v[s];
    __threadfence();
    last = atomicAdd(&d->done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    reduce_partials(partials, gridDim.x, d, cur, a);
    if (threadIdx.x == 0) d->done = 0;
  }
}


int grid_for(long long n, int threads, int cap) {
  long long b = (n + threads - 1) / threads;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

template <class L, class S, class RT>
cudaError_t init_t(lbm_ctx* c, const double* rr, const double* rb, const double* u) {
  using C = step_t<S>;
  const AuxParams a = aux_params(c);
  // CG in a compute type narrower than FP64: the gradient stencil reads each density 19
  // times, so the fields are rounded to the compute type once, into the free tail of the
  // staging buffer ([5N, 6N) doubles hold 2N values of at most 4 bytes); the stencil gives
  // the same values as rounding at every read
  C* fc = nullptr;
  if (sizeof(C) < sizeof(double) && c->p.model == LBM_MODEL_CG) {
    fc = reinterpret_cast<C*>(c->stage + 5 * c->N);
    to_compute_kernel<C><<<grid_for(c->N, 256, 8192), 256, 0, c->stream>>>(rr, rb, fc, c->N);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    c->launches += 1;
  }
  // in-place streaming: one buffer pair (the second pointers alias the first)
  // 32-bit indices where every index (populations K Q N, velocity 3 N) fits
  auto kern = (long long)c->K * c->Q * c->N < (1LL << 31) ? init_eq_kernel<L, S, RT, int>
                                                          : init_eq_kernel<L, S, RT, long long>;
  kern<<<grid_for(c->N, 256, 8192), 256, 0, c->stream>>>(
      static_cast<S*>(c->f[0]), c->aa ? nullptr : static_cast<S*>(c->f[1]), static_cast<RT*>(c->r[0]),
      c->aa ? nullptr : static_cast<RT*>(c->r[1]), rr, rb, u, c->has_walls ? c->solid : nullptr, fc, a);
  return cudaGetLastError();
}

template <class L, class S, class RT>
cudaError_t restore_t(lbm_ctx* c, const double* plane, int k, int i, const double* acc) {
  double phi[2][3];
  rest_weights(c->p, phi);
  restore_plane_kernel<S, RT><<<grid_for(c->N, 256, 8192), 256, 0, c->stream>>>(
      static_cast<S*>(c->f[0]), c->aa ? nullptr : static_cast<S*>(c->f[1]), static_cast<RT*>(c->r[0]),
      c->aa ? nullptr : static_cast<RT*>(c->r[1]),
      plane, acc + (long long)k * c->N, c->has_walls ? c->solid : nullptr, c->N, (long long)(k * c->Q + i) * c->N,
      (long long)k * c->N, phi[k][grp<L>(i)], i == 0);
  return cudaGetLastError();
}

template <class L, class S, class RT>
cudaError_t export_t(lbm_ctx* c, double* out, int first_plane, int np) {
  const AuxParams a = aux_params(c);
  export_kernel<L, S, RT><<<grid_for((long long)np * c->N, 256, 16384), 256, 0, c->stream>>>(
      static_cast<const S*>(c->f[0]), static_cast<const S*>(c->f[1]), static_cast<const RT*>(c->r[0]),
      static_cast<const RT*>(c->r[1]), c->diag, c->cur, first_plane, np, out, c->has_walls ? c->solid : nullptr, a);
  return cudaGetLastError();
}

template <class L, class S, class RT>
cudaError_t gather_t(lbm_ctx* c, void* out, int k, int i) {
  const AuxParams a = aux_params(c);
  aa_gather_kernel<L, S><<<grid_for(c->N, 256, 8192), 256, 0, c->stream>>>(
      static_cast<const S*>(c->f[0]), static_cast<S*>(out), c->has_walls ? c->solid : nullptr, k, i, a);
  return cudaGetLastError();
}

template <class L, class S, class RT>
cudaError_t diag_t(lbm_ctx* c, double* uo) {
  const AuxParams a = aux_params(c);
  const S* f0 = static_cast<const S*>(c->f[0]);
  const S* f1 = static_cast<const S*>(c->f[1]);
  const RT* r0 = static_cast<const RT*>(c->r[0]);
  const RT* r1 = static_cast<const RT*>(c->r[1]);
  double* rr = c->stage;
  double* rb = c->stage + c->N;
  double* jm = c->stage + 2 * c->N;   // momentum, then (if requested here) the velocity
  double* psi = c->stage + 5 * c->N;  // SC multiphase psi (FP64), or the multirange Psi_s
  step_t<S>* mrpsi = c->p.model == LBM_MODEL_SC_MR ? reinterpret_cast<step_t<S>*>(psi) : nullptr;
  auto dens = (long long)c->K * c->Q * c->N < (1LL << 31) ? densities_kernel<L, S, RT, int>
                                                          : densities_kernel<L, S, RT, long long>;
  dens<<<grid_for(c->N, 256, 8192), 256, 0, c->stream>>>(f0, f1, r0, r1, c->diag, c->cur, rr, rb, psi, jm, mrpsi, a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (c->rep) {
    e = launch_rep_prepass_t<L, step_t<S>, S, RT>(c, c->cur);
    if (e != cudaSuccess) return e;
  }
  diag_kernel<L, S, RT><<<c->nblk_diag, kDiagThreads, 0, c->stream>>>(
      rr, rb, psi, jm, mrpsi, c->has_walls ? c->solid : nullptr, uo, c->partials, a,
      static_cast<const step_t<S>*>(c->colour), static_cast<const step_t<S>*>(c->normals), rep_params(c), c->diag,
      c->cur);
  c->launches += 2;
  return cudaGetLastError();
}

// Dispatch on (lattice, storage precision) to an operation templated on <L, S, RT>.
template <template <class, class, class> class F, class... Args>
cudaError_t by_lattice_precision(lbm_ctx* c, Args... args) {
  const bool d3 = c->p.lattice == LBM_D3Q19;
  switch (c->p.precision) {
    case LBM_FP64:
      return d3 ? F<D3Q19, double, double>::run(c, args...) : F<D2Q9, double, double>::run(c, args...);
    case LBM_FP32:
      return d3 ? F<D3Q19, float, float>::run(c, args...) : F<D2Q9, float, float>::run(c, args...);
    case LBM_FP16:
      return d3 ? F<D3Q19, __half, float>::run(c, args...) : F<D2Q9, __half, float>::run(c, args...);
    default:
      return d3 ? F<D3Q19, __nv_bfloat16, float>::run(c, args...) : F<D2Q9, __nv_bfloat16, float>::run(c, args...);
  }
}

template <class L, class S, class RT>
struct InitOp {
  static cudaError_t run(lbm_ctx* c, const double* rr, const double* rb, const double* u) {
    return init_t<L, S, RT>(c, rr, rb, u);
  }
};
template <class L, class S, class RT>
struct RestoreOp {
  static cudaError_t run(lbm_ctx* c, const double* plane, int k, int i, const double* acc) {
    return restore_t<L, S, RT>(c, plane, k, i, acc);
  }
};
template <class L, class S, class RT>
struct ExportOp {
  static cudaError_t run(lbm_ctx* c, double* out, int first, int np) { return export_t<L, S, RT>(c, out, first, np); }
};
template <class L, class S, class RT>
struct GatherOp {
  static cudaError_t run(lbm_ctx* c, void* out, int k, int i) { return gather_t<L, S, RT>(c, out, k, i); }
};
template <class L, class S, class RT>
struct DiagOp {
  static cudaError_t run(lbm_ctx* c, double* uo) { return diag_t<L, S, RT>(c, uo); }
};

}  // namespace

cudaError_t launch_init_eq(lbm_ctx* c, const double* rr, const double* rb, const double* u) {
  c->launches += 1;
  return by_lattice_precision<InitOp>(c, rr, rb, u);
}

cudaError_t launch_restore_accumulate(lbm_ctx* c, const double* plane, int k, double* acc, bool first) {
  c->launches += 1;
  restore_acc_kernel<<<grid_for(c->N, 256, 8192), 256, 0, c->stream>>>(plane, acc + (long long)k * c->N, c->N, first);
  return cudaGetLastError();
}

cudaError_t launch_restore_plane(lbm_ctx* c, const double* plane, int k, int i, const double* acc) {
  c->launches += 1;
  return by_lattice_precision<RestoreOp>(c, plane, k, i, acc);
}

cudaError_t launch_export_plane(lbm_ctx* c, double* plane, int k, int i) {
  c->launches += 1;
  return by_lattice_precision<ExportOp>(c, plane, k * c->Q + i, 1);
}

cudaError_t launch_export_all(lbm_ctx* c, double* pops) {
  c->launches += 1;
  return by_lattice_precision<ExportOp>(c, pops, 0, c->K * c->Q);
}

cudaError_t launch_aa_gather_plane(lbm_ctx* c, void* out, int k, int i) {
  c->launches += 1;
  return by_lattice_precision<GatherOp>(c, out, k, i);
}

cudaError_t launch_diagnostics(lbm_ctx* c, double* u_out, bool want_u) {
  double* uo = u_out ? u_out : (want_u ? c->stage + 2 * c->N : nullptr);
  return by_lattice_precision<DiagOp>(c, uo);
}

}  // namespace lbm
