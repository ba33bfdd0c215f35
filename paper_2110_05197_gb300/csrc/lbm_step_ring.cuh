// D3Q19 step kernel with a two-plane TMA ring and the next plane's node state carried in
// registers (16-bit and FP32 storage; colour-gradient and Shan-Chen multiphase models).
//
// Same step and per-node arithmetic as the other step kernels (lbm_step.cuh): the same
// density sums (comp_state), stencil fields (node_fields), pair-difference gradients,
// collision and re-referenced push.  What differs is the work split.  Every thread owns one
// (x, y) column of a TX x TY tile (512 threads: 16 warps per SM, one block per SM) and
// marches z; there are no producer, staging or collision roles.  Per plane J of the
// block's sequence, each thread
//   1. reads its own node of plane J from the raw plane buffer (a TMA copy of the tile's
//      TX x (TY + 2) rows: interior rows plus one halo row above and below), forms the
//      component densities (comp_state) and keeps in registers what the collision of that
//      node needs one plane later: the density bookkeeping (rho, dq, d per colour) and the
//      colour sums t_i = g^R_i + g^B_i of the stored deviations (the CG collision acts on
//      the total population and never reads a single colour's input; SC: the deviations);
//      for CG the sums are read after step 4 instead (ring_late_hold);
//   2. writes the node's stencil fields into field slot J; threads of the first two tile
//      rows also reduce one node of the top or bottom halo row;
//   3. passes a block barrier; then the threads of the tile's first and last column send
//      their fields to the x-neighbours' halo columns in distributed shared memory (a
//      cluster of nx / TX blocks spans a full x-row of tiles, so the periodic wrap in x
//      stays inside the cluster) as asynchronous remote stores (st.async) that complete on
//      the receiver's mbarrier of slot J, and every thread waits on its own block's
//      mbarrier of slot J for the neighbours' columns;
//   4. collides plane J-1 from the registers of step 1 and the field slots J-2, J-1, J,
//      and pushes the post-collision deviations to their destinations in global memory.
// No thread ever releases at cluster scope: a cluster barrier (or any release at cluster
// scope) would make every thread wait, once per plane, until its 38 global stores of the
// previous collision had reached L2 -- measured at a third of the step's time.  The remote
// columns are ordered by the mbarrier's transaction count instead.
// A raw plane buffer is only read in iteration J of its own plane, so with R buffers the
// copy of plane J+R-1 is issued at the start of iteration J (after step 3 when the sums
// are read late), once a block barrier has retired every read of the buffer it
// overwrites (plane J-1's), and has about R-1 planes of work to land; R is 2 to 4, as
// shared memory allows.  Field slot J (last read by the collision of plane J-3, in iteration
// J-2) is written locally after the block barrier of iteration J-1, and remotely by a
// neighbour only after that neighbour has received this block's columns of plane J-1,
// which are sent after this block's barrier of iteration J-1: four field slots.  Without
// a population ring for the collision, shared memory holds 16 warps' nodes instead of 8,
// which is what the step needs to hide its latencies.
//
// CG fields per extended node: q_R, q_B (the new reference densities, equal to the
// component densities in FP32; rho = q_R + q_B is formed where it is read, bitwise equal to
// the staged total of the other kernels) and rho^N.  SC multiphase: psi and q.
#pragma once

#include "lbm_step_tmac.cuh"

namespace lbm {

template <int MODEL>
struct RingTraits;
template <>
struct RingTraits<kCG> {
  static constexpr int NV = 3;  // q_R, q_B, rho^N
  static constexpr int NH = 19; // colour sums carried per node
};
template <>
struct RingTraits<kSCMP> {
  static constexpr int NV = 2;  // psi, q
  static constexpr int NH = 19; // the deviations themselves
};

constexpr int kRingFields = 4;    // field slots
// Whether the sums a thread carries to the next plane are read from the raw plane buffer
// after the collision rather than while staging: then only one plane's sums are live
// across the collision (fewer registers), but the plane's copy can only be issued after
// the block barrier that retires those late reads, half a plane later.  Measured at
// 128^3: CG in 16-bit storage 166 -> 160 us (64 x 4 tiles), 189 -> 176 us (32 x 16), FP32
// CG unchanged; SC multiphase, whose planes are quicker, 83 -> 95 us.  So CG only.
template <int MODEL>
__host__ __device__ constexpr bool ring_late_hold() { return MODEL == kCG; }
constexpr int kRingHeader = 128;  // mbarriers, then 128-byte aligned plane buffers

// Blocks per SM: 16 warps per SM either as one 512-thread block or as two 256-thread
// blocks (whose per-plane barriers then fall at different times).
template <int TX, int TY>
__host__ __device__ constexpr int ring_blocks() { return 512 / (TX * TY); }

template <class L, class S, class RT, int MODEL, int TX, int TY>
__host__ __device__ constexpr size_t ring_bytes_for(int raw) {
  using Lay = TmaLayout<L, S, RT, MODEL, TX, TY>;
  return kRingHeader + size_t(raw) * Lay::BUF_MAIN + size_t(kRingFields) * RingTraits<MODEL>::NV * Lay::NE * 4;
}
// Raw plane buffers: as many (2 to 4) as the block's share of shared memory holds (227 KB
// for one block per SM, 113 KB each for two); 0 when two do not fit.  A third buffer gives
// each copy two planes of work to land instead of one.
template <class L, class S, class RT, int MODEL, int TX, int TY>
__host__ __device__ constexpr int ring_raw() {
  constexpr size_t budget = ring_blocks<TX, TY>() == 1 ? 232448 : 115712;
  return ring_bytes_for<L, S, RT, MODEL, TX, TY>(4) <= budget   ? 4
         : ring_bytes_for<L, S, RT, MODEL, TX, TY>(3) <= budget ? 3
         : ring_bytes_for<L, S, RT, MODEL, TX, TY>(2) <= budget ? 2
                                                                : 0;
}

// Asynchronous 32-bit store into another block's shared memory (addresses from mapa);
// completion is counted, in bytes, on that block's mbarrier `bar`.
__device__ __forceinline__ void st_async_f32(uint32_t cluster_addr, float v, uint32_t cluster_bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(cluster_addr),
               "r"(__float_as_uint(v)), "r"(cluster_bar)
               : "memory");
}

template <class L, class S, class RT, int MODEL, int TX, int TY>
__host__ __device__ constexpr size_t ring_smem_bytes() {
  return ring_bytes_for<L, S, RT, MODEL, TX, TY>(ring_raw<L, S, RT, MODEL, TX, TY>());
}

// Tensor maps of the ring kernel's tiles: TY interior rows, and single halo rows.
template <int TX, int TY>
__device__ __forceinline__ const CUtensorMap* ring_pop_map(const TmaMaps& m, bool mid) {
  if constexpr (TX == 64) return mid ? (TY == 8 ? &m.pop_w_mid8 : &m.pop_w_mid4) : &m.pop_w_row;
  return mid ? (TY == 16 ? &m.pop_main_mid16 : &m.pop_main_mid) : &m.pop_main_row;
}
template <int TX, int TY>
__device__ __forceinline__ const CUtensorMap* ring_ref_map(const TmaMaps& m, bool mid) {
  if constexpr (TX == 64) return mid ? (TY == 8 ? &m.ref_w_mid8 : &m.ref_w_mid4) : &m.ref_w_row;
  return mid ? (TY == 16 ? &m.ref_main_mid16 : &m.ref_main_mid) : &m.ref_main_row;
}

// The sequence of planes a cluster stages: for each of its work units (tile row, z range
// [z0, z1)) the planes z0-1 .. z1; the first and last are halo planes (staged, not
// collided).
struct PlaneSeq {
  WorkRange work;
  Segment sg;
  int z;
  bool valid;
  __device__ PlaneSeq(int b, int nblk, int ncol, int nz, int nchunks) : work(b, nblk, ncol, nz, nchunks) {
    valid = work.pop(sg);
    z = sg.z0 - 1;
  }
  __device__ void next() {
    if (++z > sg.z1) {
      valid = work.pop(sg);
      z = sg.z0 - 1;
    }
  }
};

// CG collision (Eqs. BGK, equiliCG, guoforce/source with the body force, perturbationOp,
// recoloringOpR/B, cosphi) from the colour sums t_i = g^R_i + g^B_i of the stored
// deviations: the arithmetic of cg_collide (lbm_step.cuh) term for term, with the outputs
// handed to emit(i, g^R_i, g^B_i) as they are formed instead of written back.
template <class L, class T, class NB, class EMIT>
__device__ __forceinline__ void cg_collide_sums(const StepParams<T>& p, const T (&t)[L::Q], const CompState<T>& cr,
                                                const CompState<T>& cb, const NB& nbr, const EMIT& emit) {
  constexpr int Q = L::Q;
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
  T G[Q];
#pragma unroll
  for (int i = 0; i < Q; i++) {
    const int gi = grp<L>(i);
    G[i] = t[i] + (p.phi[0][gi] * cr.d + p.phi[1][gi] * cb.d);
  }
  T jm[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int q = 0; q < L::NP; q++) {
    const T dd = t[2 * q + 1] - t[2 * q + 2];
    if (L::pcx(q)) jm[0] += L::pcx(q) * dd;
    if (L::pcy(q)) jm[1] += L::pcy(q) * dd;
    if (L::pcz(q)) jm[2] += L::pcz(q) * dd;
  }
  T F[3] = {T(0), T(0), T(0)};
  if (p.has_body) { F[0] += p.body[0]; F[1] += p.body[1]; F[2] += p.body[2]; }
  const bool forced = F[0] != T(0) || F[1] != T(0) || F[2] != T(0);
  T u[3];
#pragma unroll
  for (int a = 0; a < 3; a++) u[a] = (jm[a] + T(0.5) * F[a]) * inv;
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
  const T dR = cr.dq, dB = cb.dq;
  T c_rest[3], c_u2[3], c_uu[3], c_od[3], c_fe[3], c_rc[3], c_base[3], c_sev[3], c_sod[3];  // [0] unused
#pragma unroll
  for (int gi = 1; gi <= 2; gi++) {
    const T w = T(L::w(gi));
    const T phR = p.phi[0][gi], phB = p.phi[1][gi];
    c_rest[gi] = en * T(L::psi(gi)) * ugr + phR * dR + phB * dB - rho * w * T(1.5) * uu;
    c_u2[gi] = rho * w * T(4.5);
    c_uu[gi] = en * T(2.0 * L::xi(gi));
    c_od[gi] = rho * w * T(3);
    c_fe[gi] = rr * phR + rb * phB;
    c_rc[gi] = rec * c_fe[gi] * inv_g * ((gi == 1) ? T(1) : T(0.70710678118654752440));
    c_base[gi] = (rr * phB * cb.q - rb * phR * cr.q) * inv;
    c_sev[gi] = w * kg;
    c_sod[gi] = w * kg * T(3);
  }
  {
    const T eq = en * T(L::psi(0)) * ugr + rho * T(L::w(0)) * (T(-1.5) * uu) + p.phi[0][0] * dR + p.phi[1][0] * dB;
    T Gs = G[0] + omega * (eq - G[0]);
    if (forced) Gs += T(L::w(0)) * kg * (T(-3) * uF);
    Gs -= Ag * T(L::B(0));
    const T base = (rr * p.phi[1][0] * cb.q - rb * p.phi[0][0] * cr.q) * inv;
    const T gR = cR * Gs + base;
    emit(0, gR, Gs - gR);
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
      const T ev = c_rest[gi] + cu * (c_u2[gi] * cu + c_uu[gi] * cg);
      const T od = c_od[gi] * cu;
      const T pert = Ag * (T(L::w(gi)) * cn * cn * inv_gg - T(L::B(gi)));
      T Gsi = G[i] + omega * (ev + od - G[i]) + pert;
      T Gsj = G[j] + omega * (ev - od - G[j]) + pert;
      if constexpr (FORCE) {
        const T cF = T(L::pcx(q)) * F[0] + T(L::pcy(q)) * F[1] + T(L::pcz(q)) * F[2];
        const T sev = c_sev[gi] * (T(9) * cu * cF - T(3) * uF);
        const T sod = c_sod[gi] * cF;
        Gsi += sev + sod;
        Gsj += sev - sod;
      }
      const T rc = c_rc[gi] * cn;
      const T gRi = cR * Gsi + c_base[gi] + rc;
      const T gRj = cR * Gsj + c_base[gi] - rc;
      emit(i, gRi, Gsi - gRi);
      emit(j, gRj, Gsj - gRj);
    }
  };
  if (forced)
    pairs(std::true_type{});
  else
    pairs(std::false_type{});
}

// Launch: cluster dims (C, 1, 1) with C = p.ncx = nx / TX; grid = p.nblk clusters * C
// blocks of TX * TY threads; p.ncol = ny / TY tile rows.  The launcher guarantees
// nx % TX == 0, ny % TY == 0, C <= kMaxCluster and K * Q * N < 2^31.
template <class L, class T, class S, class RT, int MODEL, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, ring_blocks<TX, TY>())
    step_kernel_ring(const __grid_constant__ TmaMaps maps, S* __restrict__ fout, RT* __restrict__ rout,
                     int* __restrict__ status, const __grid_constant__ StepParams<T> p) {
  static_assert(sizeof(T) == 4 && sizeof(RT) == 4, "fields are exchanged as 32-bit words");
  static_assert((TX * TY == 512 || TX * TY == 256) && TY >= 2, "16 warps per SM; two halo rows");
  constexpr int kRingRaw = ring_raw<L, S, RT, MODEL, TX, TY>();
  static_assert(kRingRaw >= 2, "two raw plane buffers fit");
  static_assert(MODEL == kCG || MODEL == kSCMP, "models with per-colour collisions keep the other kernels");
  using Lay = TmaLayout<L, S, RT, MODEL, TX, TY>;
  constexpr int Q = L::Q, K = Lay::K;
  constexpr int NV = RingTraits<MODEL>::NV;
  constexpr int EX = Lay::EX, NE = Lay::NE;
  constexpr int FS = kRingFields;
  constexpr bool kRingLateHold = ring_late_hold<MODEL>();
  // bytes of the two halo columns (all TY + 2 rows, NV fields) the x-neighbours send
  constexpr uint32_t kEdgeBytes = 2u * (TY + 2) * NV * 4u;
  // A blown-up (or timed-out) state stops stepping.  Every block still runs the same
  // number of cluster barriers as its neighbours (they take the same planes).
  const bool skip = *status != 0;

  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* raw_full = reinterpret_cast<uint64_t*>(smem);  // [kRingRaw]
  uint64_t* fld_full = raw_full + kRingRaw;                 // [FS]: the neighbours' columns
  unsigned char* bufs = smem + kRingHeader;                 // [kRingRaw][BUF_MAIN]
  T* fld = reinterpret_cast<T*>(bufs + kRingRaw * Lay::BUF_MAIN);  // [FS][NV][NE]

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int C = p.ncx;
  const uint32_t rank = cluster_ctarank();
  const uint32_t left = (rank + C - 1) % C, right = (rank + 1) % C;
  const int x0 = (int)rank * TX;
  const int cid = blockIdx.x / C;
  const int N32 = (int)p.n;
  const int plane_n = p.nx * p.ny;

  if (tid == 0) {
    for (int s = 0; s < kRingRaw; s++) mbar_init(&raw_full[s], 1);
    for (int s = 0; s < FS; s++) mbar_init(&fld_full[s], 1);  // the expect-tx arrival
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // barriers of every block initialised before any remote store
  cluster_sync_all();
  // copy destinations must be 128-byte aligned; a misaligned base stops the work (every
  // block of the cluster sees the same offset) but not the barriers
  const bool layout_ok = (smem_addr(bufs) & 127u) == 0;
  if (!layout_ok && tid == 0) atomicOr(status, kStatusLayout);
  bool alive = !skip && layout_ok;

  // TMA copy of one plane (raw buffer s): top halo row, TY interior rows, bottom halo row,
  // populations and reference densities
  auto issue = [&](const PlaneSeq& ps, int s) {
    const int y0 = ps.sg.col * TY;
    const int yt = y0 == 0 ? p.ny - 1 : y0 - 1, yb = y0 + TY == p.ny ? 0 : y0 + TY;
    const int gz = wrap(ps.z, p.nz);
    unsigned char* b = bufs + s * Lay::BUF_MAIN;
    uint64_t* bar = &raw_full[s];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(bar, Lay::TX_BYTES);
#pragma unroll
    for (int g = 0; g < 3; g++) {
      const bool mid = g == 1;
      const int y = g == 0 ? yt : (g == 1 ? y0 : yb);
      tma_load_4d(b + Lay::PM::group(g), ring_pop_map<TX, TY>(maps, mid), x0, 0, y, gz, bar);
      tma_load_4d(b + Lay::OFF_RM + Lay::RMR::group(g), ring_ref_map<TX, TY>(maps, mid), x0, 0, y, gz, bar);
    }
  };

  PlaneSeq ahead(cid, p.nblk, p.ncol, p.nz, p.nchunks);  // the next plane to copy
  PlaneSeq cur(cid, p.nblk, p.ncol, p.nz, p.nchunks);    // the plane being staged
  int issued = 0;                                         // planes whose copy was issued
  for (int j = 0; j < kRingRaw - 1; j++) {                // planes 0 .. RAW-2 ahead of the loop
    if (tid == 0 && alive && ahead.valid) {
      issue(ahead, j);
      issued = j + 1;
    }
    ahead.next();
  }

  // register-carried state of the node staged last (collided one plane later)
  T hold[RingTraits<MODEL>::NH];
  CompState<T> hcs[K];
  // previous plane's position in its unit (interior planes are collided)
  int prev_z = 0, prev_y0 = 0;
  bool prev_interior = false;

  for (int J = 0; cur.valid; J++) {
    // copy of plane J+RAW-1 into the buffer plane J-1 used (its reads retired at the last
    // block barrier)
    if constexpr (!kRingLateHold) {
      if (tid == 0 && alive && ahead.valid) {
        issue(ahead, (J + kRingRaw - 1) % kRingRaw);
        issued = J + kRingRaw;
      }
      ahead.next();
    }
    const int y0 = cur.sg.col * TY;
    const int z = cur.z;
    const bool interior_next = z >= cur.sg.z0 && z < cur.sg.z1;  // plane J is collided in iteration J+1
    // ---- stage plane J ----
    if (alive) {
      const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&raw_full[J % kRingRaw], (J / kRingRaw) & 1));
      if (!ok) {
        if ((tid & 31) == 0) atomicOr(status, kStatusTimeout);
        alive = false;
      }
    }
    const int fs = J % FS;
    T new_hold[RingTraits<MODEL>::NH];
    CompState<T> new_cs[K];
    if (alive && tid == 0) mbar_arrive_expect_tx(&fld_full[fs], kEdgeBytes);
    if (alive) {
      const unsigned char* b = bufs + (J % kRingRaw) * Lay::BUF_MAIN;
      // one extended node (ex, ey): densities, fields into slot fs (and into an
      // x-neighbour's halo column for the tile's edge columns); the register state too
      // when `own`
      auto stage_node = [&](int ex, int ey, bool own) {
        const S* pop = reinterpret_cast<const S*>(b + Lay::PM::row(ey)) + (ex - 1);
        const RT* ref = reinterpret_cast<const RT*>(b + Lay::OFF_RM + Lay::RMR::row(ey)) + (ex - 1);
        T val[NV];
        if constexpr (MODEL == kCG) {
          T g0[Q], g1[Q];
#pragma unroll
          for (int i = 0; i < Q; i++) g0[i] = ld_s<S, T>(pop[i * TX]);
#pragma unroll
          for (int i = 0; i < Q; i++) g1[i] = ld_s<S, T>(pop[(Q + i) * TX]);
          const CompState<T> c0 = comp_state<L, T, RT>(g0, T(ref[0]));
          const CompState<T> c1 = comp_state<L, T, RT>(g1, T(ref[TX]));
          T out[2];
          node_fields<MODEL, T>(p, c0.rho, c1.rho, out);
          val[0] = c0.q;
          val[1] = c1.q;
          val[2] = out[1];
          if (own) {
            if constexpr (!kRingLateHold) {
#pragma unroll
              for (int i = 0; i < Q; i++) new_hold[i] = g0[i] + g1[i];
            }
            new_cs[0] = c0;
            new_cs[1] = c1;
          }
        } else {
          T g0[Q];
#pragma unroll
          for (int i = 0; i < Q; i++) g0[i] = ld_s<S, T>(pop[i * TX]);
          const CompState<T> c0 = comp_state<L, T, RT>(g0, T(ref[0]));
          T out[2];
          node_fields<MODEL, T>(p, c0.rho, T(0), out);
          val[0] = out[0];
          val[1] = c0.q;
          if (own) {
            if constexpr (!kRingLateHold) {
#pragma unroll
              for (int i = 0; i < Q; i++) new_hold[i] = g0[i];
            }
            new_cs[0] = c0;
          }
        }
        const int e = ey * EX + ex;
#pragma unroll
        for (int f = 0; f < NV; f++) fld[(fs * NV + f) * NE + e] = val[f];
      };
      stage_node(tx + 1, ty + 1, true);
      if (ty < 2) stage_node(tx + 1, ty == 0 ? 0 : TY + 1, false);
    }
    __syncthreads();  // local fields of plane J complete; iteration J-1's collision retired
    if constexpr (kRingLateHold) {
      // the buffer of plane J-1: its last reads (the late sums) retired at this barrier
      if (tid == 0 && alive && ahead.valid) {
        issue(ahead, (J + kRingRaw - 1) % kRingRaw);
        issued = J + kRingRaw;
      }
      ahead.next();
    }
    if (alive) {
      if (tx == 0 || tx == TX - 1) {
        // the tile's first column is the left neighbour's right halo column, its last
        // column the right neighbour's left one
        const uint32_t peer = tx == 0 ? left : right;
        const int exd = tx == 0 ? TX + 1 : 0;
        const uint32_t bar = mapa_shared(smem_addr(&fld_full[fs]), peer);
        auto send = [&](int ey) {  // the fields this thread staged at (tx + 1, ey)
#pragma unroll
          for (int f = 0; f < NV; f++) {
            const T* src = &fld[(fs * NV + f) * NE + ey * EX];
            st_async_f32(mapa_shared(smem_addr(src + exd), peer), src[tx + 1], bar);
          }
        };
        send(ty + 1);
        if (ty < 2) send(ty == 0 ? 0 : TY + 1);
      }
      const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&fld_full[fs], (J / FS) & 1));
      if (!ok) {
        if ((tid & 31) == 0) atomicOr(status, kStatusTimeout);
        alive = false;
      }
    }
    // ---- collide plane J-1 ----
    if (alive && prev_interior) {
      const int slm = (J + FS - 2) % FS, sl0 = (J + FS - 1) % FS, slp = fs;
      const int e0 = (ty + 1) * EX + (tx + 1);
      const T* f_m = fld + slm * NV * NE + e0;
      const T* f_0 = fld + sl0 * NV * NE + e0;
      const T* f_p = fld + slp * NV * NE + e0;
      auto at = [&](int i) -> const T* {
        const T* base = cz<L>(i) == 0 ? f_0 : (cz<L>(i) > 0 ? f_p : f_m);
        return base + cy<L>(i) * EX + cx<L>(i);
      };
      const int gx = x0 + tx, gy = prev_y0 + ty;
      const int xm = gx == 0 ? p.nx - 1 : gx - 1, xp = gx + 1 >= p.nx ? 0 : gx + 1;
      const int ym = gy == 0 ? p.ny - 1 : gy - 1, yp = gy + 1 >= p.ny ? 0 : gy + 1;
      const int zz = prev_z, zm = zz == 0 ? p.nz - 1 : zz - 1, zpp = zz + 1 >= p.nz ? 0 : zz + 1;
      const int rowm = ym * p.nx, row0 = gy * p.nx, rowp = yp * p.nx;
      const int pm = zm * plane_n, p0 = zz * plane_n, pp = zpp * plane_n;
      const int n0 = gx + row0 + p0;
      auto dest = [&](int i) -> int {
        const int X = cx<L>(i) == 0 ? gx : (cx<L>(i) > 0 ? xp : xm);
        const int Y = cy<L>(i) == 0 ? row0 : (cy<L>(i) > 0 ? rowp : rowm);
        const int Z = cz<L>(i) == 0 ? p0 : (cz<L>(i) > 0 ? pp : pm);
        return X + Y + Z;
      };
#pragma unroll
      for (int k = 0; k < K; k++) rout[k * N32 + n0] = RT(hcs[k].q);
      if constexpr (MODEL == kCG) {
        auto nbr = [&](int fi, int i) -> T {
          const T* a = at(i);
          return fi == 0 ? a[0] + a[NE] : a[2 * NE];  // rho = q_R + q_B, rho^N
        };
        const T qR = hcs[0].q, qB = hcs[1].q;
        auto emit = [&](int i, T vR, T vB) {
          const int nd = dest(i);
          if (i != 0) {
            const T* a = at(i);
            const int gi = grp<L>(i);
            vR += p.phi[0][gi] * (qR - a[0]);
            vB += p.phi[1][gi] * (qB - a[NE]);
          }
          fout[i * N32 + nd] = st_s<S, T>(vR);
          fout[(Q + i) * N32 + nd] = st_s<S, T>(vB);
        };
        cg_collide_sums<L, T>(p, hold, hcs[0], hcs[1], nbr, emit);
      } else {
        T g[1][Q];
#pragma unroll
        for (int i = 0; i < Q; i++) g[0][i] = hold[i];
        auto nbr = [&](int fi, int i) -> T { return at(i)[fi * NE]; };
        scmp_collide<L, T>(p, g, hcs[0], nbr);
        const T q0 = hcs[0].q;
#pragma unroll
        for (int i = 0; i < Q; i++) {
          T v = g[0][i];
          if (i != 0) v += p.phi[0][grp<L>(i)] * (q0 - at(i)[NE]);
          fout[i * N32 + dest(i)] = st_s<S, T>(v);
        }
      }
    }
    if constexpr (kRingLateHold) {
      // the colour sums of this thread's node of plane J, from its raw buffer (intact until
      // the copy issued after the next block barrier)
      if (alive) {
        const S* pop = reinterpret_cast<const S*>(bufs + (J % kRingRaw) * Lay::BUF_MAIN + Lay::PM::row(ty + 1)) + tx;
#pragma unroll
        for (int i = 0; i < Q; i++) {
          if constexpr (MODEL == kCG)
            new_hold[i] = ld_s<S, T>(pop[i * TX]) + ld_s<S, T>(pop[(Q + i) * TX]);
          else
            new_hold[i] = ld_s<S, T>(pop[i * TX]);
        }
      }
    }
    // the node staged in this iteration is collided in the next one
#pragma unroll
    for (int i = 0; i < RingTraits<MODEL>::NH; i++) hold[i] = new_hold[i];
#pragma unroll
    for (int k = 0; k < K; k++) hcs[k] = new_cs[k];
    prev_interior = interior_next;
    prev_z = z;
    prev_y0 = y0;
    cur.next();
  }
  // the copies this block issued have landed before its shared memory is released
  if (tid == 0)
    for (int j = issued - kRingRaw; j < issued; j++)
      if (j >= 0) mbar_wait_bounded(&raw_full[j % kRingRaw], (j / kRingRaw) & 1);
  __syncwarp();
  cluster_sync_all();  // no block leaves while a neighbour may still write to it
}

}  // namespace lbm
