// Launch helper for the fused step kernel (one instantiation per lattice, storage
// precision, model and wall variant).
#pragma once

#include <algorithm>

#include "lbm_internal.cuh"
#include "lbm_step_aa.cuh"
#include "lbm_step_ring.cuh"
#include "lbm_step_tmac.cuh"

namespace lbm {

// rho^N for the repulsion pre-pass, with the step's density bookkeeping; odd: the state
// is in the odd in-place layout
template <class L, class T, class S, class RT>
__global__ void colour_kernel(const S* __restrict__ f, const RT* __restrict__ r, T* __restrict__ colour,
                              RepParams a, int odd) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < a.n; m += (long long)gridDim.x * blockDim.x) {
    T rho[2];
    for (int k = 0; k < 2; k++) {
      T g[L::Q];
#pragma unroll
      for (int i = 0; i < L::Q; i++) g[i] = ld_s<S, T>(f[aa_index_n<L>(k, i, m, a.nx, a.ny, a.nz, a.n, odd)]);
      rho[k] = comp_state<L, T, RT>(g, T(r[(long long)k * a.n + m])).rho;
    }
    T s0 = rho[0], s1 = rho[1];
    if (a.color_norm) {
      s0 = s0 * T(a.inv_rho_r0);
      s1 = s1 * T(a.inv_rho_b0);
    }
    colour[m] = (s0 - s1) / (s0 + s1);
  }
}


inline RepParams rep_params(const lbm_ctx* c) {
  RepParams a{};
  a.nx = c->p.nx;
  a.ny = c->p.ny;
  a.nz = c->p.nz;
  a.n = c->N;
  a.color_norm = c->p.color_norm;
  a.psi_kind = c->p.rep_psi_kind;
  a.inv_rho_r0 = 1.0 / c->p.rho_r0;
  a.inv_rho_b0 = 1.0 / c->p.rho_b0;
  a.grad_eps = c->p.grad_eps;
  a.pi = c->p.rep_pi;
  a.chi = c->p.rep_chi;
  return a;
}

// Colour and normal fields of the current state (repulsion pre-pass).
template <class L, class T, class S, class RT>
cudaError_t launch_rep_prepass_t(lbm_ctx* c, int buf) {
  const RepParams a = rep_params(c);
  const int grid = (int)std::min<long long>((c->N + 255) / 256, 8192);
  colour_kernel<L, T, S, RT><<<grid, 256, 0, c->stream>>>(static_cast<const S*>(c->f[buf]),
                                                           static_cast<const RT*>(c->r[buf]),
                                                           static_cast<T*>(c->colour), a, c->aa ? (buf & 1) : 0);
  if (3 * c->N < (1LL << 31))  // 32-bit indices: the normals array holds 3 N values
    normals_kernel<L, T, int><<<grid, 256, 0, c->stream>>>(
        static_cast<const T*>(c->colour), c->has_walls ? c->solid : nullptr, static_cast<T*>(c->normals), a);
  else
    normals_kernel<L, T, long long><<<grid, 256, 0, c->stream>>>(
        static_cast<const T*>(c->colour), c->has_walls ? c->solid : nullptr, static_cast<T*>(c->normals), a);
  c->launches += 2;
  return cudaGetLastError();
}

// Persistent grid: `resident` blocks (or clusters) loop over the units.  The z-chunk count
// trades the halo planes every unit re-reads (2 per unit) against the idle share of the
// last round of units; chunks stay at least 8 planes long.
template <class T>
void persistent_plan(StepParams<T>& sp, int resident) {
  resident = std::max(resident, 1);
  const int max_chunks = std::max(1, sp.nz / 8);
  double best = -1.0;
  int best_n = 1;
  for (int n = 1; n <= max_chunks; n++) {
    const long long units = (long long)sp.ncol * n;
    const long long rounds = (units + resident - 1) / resident;
    const double busy = double(units) / double(rounds * resident);  // share of block-rounds with a unit
    const double planes = double(sp.nz) / n;
    const double score = busy / (1.0 + 1.0 / planes);  // halo planes cost about half a plane each
    if (score > best + 1e-9) {
      best = score;
      best_n = n;
    }
  }
  sp.nchunks = best_n;
  sp.nblk = (int)std::min<long long>((long long)sp.ncol * best_n, resident);
}

template <class L, class T, class S, class RT, int MODEL, bool WALLS>
cudaError_t launch_tma_t(lbm_ctx* c) {
  constexpr int TX = kTmaTX, TY = kTmaTY;
  constexpr size_t smem = tma_smem_bytes<L, T, S, RT, MODEL, WALLS, TX, TY>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(step_kernel_tma<L, T, S, RT, MODEL, WALLS, TX, TY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 block(kTmaThreads, 1, 1);
  StepParams<T> sp = make_step_params<T>(c);
  if (c->tz == 0) persistent_plan(sp, c->nsm);  // one block per SM (shared memory)
  dim3 grid(sp.nblk, 1, 1);
  const S* fin = static_cast<const S*>(c->f[c->cur]);
  const RT* rin = static_cast<const RT*>(c->r[c->cur]);
  S* fout = static_cast<S*>(c->f[c->cur ^ 1]);
  RT* rout = static_cast<RT*>(c->r[c->cur ^ 1]);
  step_kernel_tma<L, T, S, RT, MODEL, WALLS, TX, TY><<<grid, block, smem, c->stream>>>(
      c->tma[c->cur], fin, rin, fout, rout, c->solid, &c->diag->status, sp);
  return cudaGetLastError();
}

// TMA-staged kernel with the x-halo exchanged inside a cluster of nx / 32 blocks.
template <class L, class T, class S, class RT, int MODEL, bool WALLS, int TX, int TY>
cudaError_t launch_tmac_t(lbm_ctx* c) {
  constexpr size_t smem = tmac_smem_bytes<L, T, S, RT, MODEL, WALLS, TX, TY>();
  auto kern = step_kernel_tmac<L, T, S, RT, MODEL, WALLS, TX, TY>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int C = c->p.nx / TX;
  StepParams<T> sp = make_step_params<T>(c);
  sp.ncx = C;                // blocks per cluster
  sp.ncol = c->p.ny / TY;    // tile rows: the work partition's columns
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(tmac_threads<MODEL, S, TX, TY>(), 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c->stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (c->tz > 0) {
    sp.nblk = sp.ncol * sp.nchunks;
  } else {
    const void* fn = reinterpret_cast<const void*>(kern);
    if (c->occ_fn != fn || c->occ_tx != -C) {
      int ncl = 0;
      cfg.gridDim = dim3(C, 1, 1);
      cudaError_t e = cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg);
      if (e != cudaSuccess) return e;
      c->occ_fn = fn;
      c->occ_tx = -C;
      c->occ_ty = 0;
      c->occ_blocks = ncl > 0 ? ncl : 1;
    }
    persistent_plan(sp, c->occ_blocks);  // clusters
  }
  cfg.gridDim = dim3(sp.nblk * C, 1, 1);
  S* fout = static_cast<S*>(c->f[c->cur ^ 1]);
  RT* rout = static_cast<RT*>(c->r[c->cur ^ 1]);
  return cudaLaunchKernelEx(&cfg, kern, c->tma[c->cur], fout, rout, c->solid, &c->diag->status, sp);
}

// Ring kernel (lbm_step_ring.cuh): 512-node tiles (one block per SM) or 256-node tiles
// (two), 2 to 4 raw plane buffers, clusters of nx / TX blocks.
template <class L, class T, class S, class RT, int MODEL, int TX, int TY>
cudaError_t launch_ring_t(lbm_ctx* c) {
  constexpr size_t smem = ring_smem_bytes<L, S, RT, MODEL, TX, TY>();
  auto kern = step_kernel_ring<L, T, S, RT, MODEL, TX, TY>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int C = c->p.nx / TX;
  StepParams<T> sp = make_step_params<T>(c);
  sp.ncx = C;               // blocks per cluster
  sp.ncol = c->p.ny / TY;   // tile rows: the work partition's columns
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(TX * TY, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c->stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (c->tz > 0) {
    sp.nblk = sp.ncol * sp.nchunks;  // one unit (tile row, tz planes) per cluster
  } else {
    const void* fn = reinterpret_cast<const void*>(kern);
    if (c->occ_fn != fn || c->occ_tx != -C) {
      int ncl = 0;
      cfg.gridDim = dim3(C, 1, 1);
      cudaError_t e = cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg);
      if (e != cudaSuccess) return e;
      c->occ_fn = fn;
      c->occ_tx = -C;
      c->occ_ty = 0;
      c->occ_blocks = ncl > 0 ? ncl : 1;
    }
    persistent_plan(sp, c->occ_blocks);  // clusters
  }
  cfg.gridDim = dim3(sp.nblk * C, 1, 1);
  S* fout = static_cast<S*>(c->f[c->cur ^ 1]);
  RT* rout = static_cast<RT*>(c->r[c->cur ^ 1]);
  return cudaLaunchKernelEx(&cfg, kern, c->tma[c->cur], fout, rout, &c->diag->status, sp);
}

// Whether the ring kernel runs this context with TX x TY tiles.
template <class L, class T, class S, class RT, int MODEL, bool WALLS, bool REP, int TX, int TY>
bool ring_eligible(const lbm_ctx* c) {
  if constexpr (L::D != 3 || sizeof(T) != 4 || WALLS || REP || !(MODEL == kCG || MODEL == kSCMP)) {
    return false;
  } else {
    if (ring_raw<L, S, RT, MODEL, TX, TY>() < 2) return false;  // two plane buffers do not fit
    // 64 x 4 and 32 x 8 tiles use the maps every TMA-eligible lattice has (64-column
    // maps where nx % 64 == 0)
    const bool maps = TX == 64 ? (TY == 8 ? c->tma[0].w_mid8 && c->tma[1].w_mid8 : c->p.nx % 64 == 0)
                               : (TY == 16 ? c->tma[0].mid16 && c->tma[1].mid16 : true);
    return c->tma_ok && maps && !c->aa && c->p.nx % TX == 0 && c->p.ny % TY == 0 &&
           c->p.nx / TX <= kMaxCluster && (long long)c->K * c->Q * c->N < (1LL << 31);
  }
}

// Field-pass step (in-place streaming, or the multirange model): the field pass, then the
// step kernel, both over all nodes.
template <class L, class T, class S, class RT, int MODEL, bool WALLS, bool REP, class I>
cudaError_t launch_fp_i(lbm_ctx* c) {
  if constexpr (REP) {
    cudaError_t e = launch_rep_prepass_t<L, T, S, RT>(c, c->cur);
    if (e != cudaSuccess) return e;
  }
  const StepParams<T> sp = make_step_params<T>(c);
  const int odd = c->aa ? (c->cur & 1) : 0;
  const int mode = c->aa ? 1 + odd : 0;
  const S* fin = static_cast<const S*>(c->f[c->cur]);
  S* fout = static_cast<S*>(c->f[c->cur ^ 1]);  // == fin in place
  const RT* rin = static_cast<const RT*>(c->r[c->cur]);
  RT* rout = static_cast<RT*>(c->r[c->cur ^ 1]);
  T* fld = reinterpret_cast<T*>(c->stage);  // [NF + K][N] of the compute type, fits 6N doubles
  const long long blocks = (c->N + 255) / 256;
  const int grid = (int)std::min<long long>(blocks, (long long)c->nsm * 16);
  fp_fields_kernel<L, T, S, RT, MODEL><<<grid, 256, 0, c->stream>>>(fin, rin, fld, WALLS ? c->solid : nullptr,
                                                                   &c->diag->status, sp, odd);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  c->launches += 1;
  if constexpr (L::D == 3 && MODEL == kSCMR) {
    // belt-2 fields staged in shared memory (halo 2): 2.7x faster than gathering the 92
    // neighbours through L1; for the halo-1 models the L1 gathers measured as fast or
    // faster (in-place SC-MP 128^3: 142 vs 162 us), so they keep fp_step_kernel
    constexpr int H = 2;
    constexpr size_t smem = fpt_smem_bytes<T, MODEL, WALLS, H>();
    auto kern = fpt_step_kernel<L, T, S, RT, MODEL, WALLS, REP, H, I>;
    static int occ = 0;  // resident blocks per SM of this instantiation
    if (occ == 0) {
      if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
      }
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kFpTX * kFpTY, smem);
      if (e != cudaSuccess) return e;
      occ = std::max(occ, 1);
    }
    StepParams<T> tp = sp;
    tp.ncx = (c->p.nx + kFpTX - 1) / kFpTX;
    tp.ncol = tp.ncx * ((c->p.ny + kFpTY - 1) / kFpTY);
    persistent_plan(tp, c->nsm * occ);
    kern<<<tp.nblk, kFpTX * kFpTY, smem, c->stream>>>(fin, fout, rin, rout, fld, c->solid, &c->diag->status, tp,
                                                      static_cast<const T*>(c->colour),
                                                      static_cast<const T*>(c->normals), rep_params(c), mode);
  } else {
    fp_step_kernel<L, T, S, RT, MODEL, WALLS, REP, I><<<grid, 256, 0, c->stream>>>(
        fin, fout, rin, rout, fld, c->solid, &c->diag->status, sp, static_cast<const T*>(c->colour),
        static_cast<const T*>(c->normals), rep_params(c), mode);
  }
  return cudaGetLastError();
}

// Field-pass step with 32-bit indices where every index fits (FP64 storage: 64-bit).
template <class L, class T, class S, class RT, int MODEL, bool WALLS, bool REP>
cudaError_t launch_fp_t(lbm_ctx* c) {
  if constexpr (sizeof(T) < 8) {
    if ((long long)c->K * c->Q * c->N < (1LL << 31)) return launch_fp_i<L, T, S, RT, MODEL, WALLS, REP, int>(c);
  }
  return launch_fp_i<L, T, S, RT, MODEL, WALLS, REP, long long>(c);
}

// Generic plane-marching step (step_kernel) with index type I.
template <class L, class T, class S, class RT, int MODEL, bool WALLS, bool REP, class I>
cudaError_t launch_generic_t(lbm_ctx* c) {
  const int tx = c->tx, ty = c->ty;
  const size_t smem = step_smem_bytes<L, T, MODEL, WALLS>(tx, ty);
  static size_t smem_set = 0;  // largest dynamic shared memory opted in so far
  if (smem > 48 * 1024 && smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(step_kernel<L, T, S, RT, MODEL, WALLS, REP, I>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    smem_set = smem;
  }
  dim3 block(tx, ty, 1);
  StepParams<T> sp = make_step_params<T>(c);
  if (c->tz == 0) {
    const void* fn = reinterpret_cast<const void*>(step_kernel<L, T, S, RT, MODEL, WALLS, REP, I>);
    if (c->occ_fn != fn || c->occ_tx != tx || c->occ_ty != ty) {
      int nb = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, step_kernel<L, T, S, RT, MODEL, WALLS, REP, I>,
                                                                    tx * ty, smem);
      if (e != cudaSuccess) return e;
      c->occ_fn = fn;
      c->occ_tx = tx;
      c->occ_ty = ty;
      c->occ_blocks = nb > 0 ? nb : 1;
    }
    persistent_plan(sp, c->nsm * c->occ_blocks);
  }
  dim3 grid(sp.nblk, 1, 1);
  const S* fin = static_cast<const S*>(c->f[c->cur]);
  S* fout = static_cast<S*>(c->f[c->cur ^ 1]);
  const RT* rin = static_cast<const RT*>(c->r[c->cur]);
  RT* rout = static_cast<RT*>(c->r[c->cur ^ 1]);
  step_kernel<L, T, S, RT, MODEL, WALLS, REP, I><<<grid, block, smem, c->stream>>>(
      fin, fout, rin, rout, c->solid, &c->diag->status, sp, static_cast<const T*>(c->colour),
      static_cast<const T*>(c->normals), rep_params(c));
  return cudaGetLastError();
}

template <class L, class T, class S, class RT, int MODEL, bool WALLS, bool REP>
cudaError_t launch_step_t(lbm_ctx* c) {
  if constexpr (MODEL == kSCMR) {
    return launch_fp_t<L, T, S, RT, MODEL, WALLS, REP>(c);
  } else {
  if (c->aa) return launch_fp_t<L, T, S, RT, MODEL, WALLS, REP>(c);
  if (c->tx * c->ty > 256) {
    // a ring tiling: the ring kernel where it applies, else the 32 x 8 persistent tiling
    if constexpr (L::D == 3 && sizeof(T) == 4 && !WALLS && !REP && (MODEL == kCG || MODEL == kSCMP)) {
      if constexpr (ring_raw<L, S, RT, MODEL, 32, 16>() >= 2)
        if (c->tx == 32 && ring_eligible<L, T, S, RT, MODEL, WALLS, REP, 32, 16>(c))
          return launch_ring_t<L, T, S, RT, MODEL, 32, 16>(c);
      if constexpr (ring_raw<L, S, RT, MODEL, 64, 8>() >= 2)
        if (c->tx == 64 && ring_eligible<L, T, S, RT, MODEL, WALLS, REP, 64, 8>(c))
          return launch_ring_t<L, T, S, RT, MODEL, 64, 8>(c);
    }
    const int tx = c->tx, ty = c->ty, tz = c->tz;
    c->tx = kTmaTX;
    c->ty = kTmaTY;
    c->tz = 0;
    const cudaError_t e = launch_step_t<L, T, S, RT, MODEL, WALLS, REP>(c);
    c->tx = tx;
    c->ty = ty;
    c->tz = tz;
    return e;
  }
  if constexpr (L::D == 3 && sizeof(T) == 4 && !WALLS && !REP && (MODEL == kCG || MODEL == kSCMP)) {
    // 64 x 4 tiles: the ring kernel (two blocks per SM) where two of its blocks fit an SM
    // (every storage type for SC multiphase, 16-bit storage for CG); it gives the same bits
    // as the cluster kernel, which keeps the other cases
    if constexpr (ring_raw<L, S, RT, MODEL, 64, 4>() >= 2)
      if (c->tx == 64 && c->ty == 4 && ring_eligible<L, T, S, RT, MODEL, WALLS, REP, 64, 4>(c))
        return launch_ring_t<L, T, S, RT, MODEL, 64, 4>(c);
  }
  if constexpr (L::D == 3 && sizeof(T) == 4 && !REP) {
    const bool small_index = (long long)c->K * c->Q * c->N < (1LL << 31);
    if (c->tma_ok && c->tx == 64 && c->ty == 4 && c->p.nx % 64 == 0 && c->p.nx / 64 <= kMaxCluster && small_index)
      return launch_tmac_t<L, T, S, RT, MODEL, WALLS, 64, 4>(c);
    if (c->tma_ok && c->tx == kTmaTX && c->ty == 4 && c->p.nx / kTmaTX <= kMaxCluster && small_index)
      return launch_tmac_t<L, T, S, RT, MODEL, WALLS, kTmaTX, 4>(c);
    if (c->tma_ok && c->tx == kTmaTX && c->ty == kTmaTY) {
      if (c->p.nx / kTmaTX <= kMaxCluster && (long long)c->K * c->Q * c->N < (1LL << 31))
        return launch_tmac_t<L, T, S, RT, MODEL, WALLS, kTmaTX, kTmaTY>(c);
      return launch_tma_t<L, T, S, RT, MODEL, WALLS>(c);
    }
  }
  if constexpr (REP) {
    cudaError_t e = launch_rep_prepass_t<L, T, S, RT>(c, c->cur);
    if (e != cudaSuccess) return e;
  }
  // 32-bit node and array indices where every index fits (FP64 storage keeps 64-bit ones:
  // its step is bound by the FP64 rate, not by index arithmetic)
  if constexpr (sizeof(T) < 8) {
    if ((long long)c->K * c->Q * c->N < (1LL << 31)) return launch_generic_t<L, T, S, RT, MODEL, WALLS, REP, int>(c);
  }
  return launch_generic_t<L, T, S, RT, MODEL, WALLS, REP, long long>(c);
  }
}

template <class L, class T, class S, class RT, int MODEL>
cudaError_t dispatch_walls(lbm_ctx* c) {
  const bool w = c->has_walls;
  if constexpr (MODEL == kCG) {
    if (c->rep) return w ? launch_step_t<L, T, S, RT, MODEL, true, true>(c) : launch_step_t<L, T, S, RT, MODEL, false, true>(c);
  }
  return w ? launch_step_t<L, T, S, RT, MODEL, true, false>(c) : launch_step_t<L, T, S, RT, MODEL, false, false>(c);
}

template <class T, class S, class RT, int MODEL>
cudaError_t dispatch_lattice(lbm_ctx* c) {
  if constexpr (MODEL == kSCMR) {
    return dispatch_walls<D3Q19, T, S, RT, MODEL>(c);  // D3Q19 only (lbm_create checks)
  } else {
    if (c->p.lattice == LBM_D3Q19) return dispatch_walls<D3Q19, T, S, RT, MODEL>(c);
    return dispatch_walls<D2Q9, T, S, RT, MODEL>(c);
  }
}

template <class T, class S, class RT>
cudaError_t dispatch_model(lbm_ctx* c) {
  if (c->p.model == LBM_MODEL_CG) return dispatch_lattice<T, S, RT, kCG>(c);
  if (c->p.model == LBM_MODEL_SC_MP) return dispatch_lattice<T, S, RT, kSCMP>(c);
  if (c->p.model == LBM_MODEL_SC_MR) return dispatch_lattice<T, S, RT, kSCMR>(c);
  return dispatch_lattice<T, S, RT, kSC2C>(c);
}


}  // namespace lbm
