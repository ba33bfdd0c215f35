// Host-side context and launcher declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/lbm.h"
#include "lbm_step.cuh"
#include "lbm_step_tma.cuh"

// Device-side diagnostics record: totals (LBM_NTOTALS doubles) then the blow-up status.
struct lbm_diag {
  double totals[LBM_NTOTALS];
  int status;       // 0 ok; bit 0 non-finite, bit 1 negative density, bit 2 |u| too large
  int trip_buf;     // population buffer (0/1) holding the state the check tripped on; after a
                    // trip the step kernels write nothing, so that buffer stays the state
  unsigned done;    // blocks of the running diagnostics pass that have written their partials
                    // (the last one reduces them and puts it back to 0)
  int pad;
};

struct lbm_ctx {
  lbm_params p;
  int K, Q;
  long long N;
  size_t elt;            // bytes per stored population
  size_t relt;           // bytes per reference density
  cudaStream_t stream;
  unsigned char* ws;
  size_t ws_bytes;
  void* f[2];            // A/B population buffers [K][Q][N], deviations from phi * r
  void* r[2];            // A/B reference densities [K][N] (paired with f[])
  int cur;               // index of the buffer pair holding the current state
  bool aa;               // in-place streaming: f[1] == f[0], r[1] == r[0], and cur is the
                         // layout parity of the state (lbm_step_aa.cuh)
  uint8_t* solid;        // [N] wall mask (all zero without walls)
  bool has_walls;
  double* stage;         // [6][N] FP64 staging ([7][N] for the multirange model in FP64):
                         // rho_r, rho_b, momentum then u (x, y, z), psi (SC multiphase) or
                         // the multirange Psi_s in the compute type;
                         // in-place streaming also uses it for the step's field pass
  double* partials;      // [nblk_diag][LBM_NTOTALS]
  int nblk_diag;
  lbm_diag* diag;        // device
  bool initialised;
  lbm_status sticky;
  unsigned long long launches;
  long long steps;
  int tx, ty, tz;        // step kernel tiling (tz = 0: persistent grid)
  int nsm;               // streaming multiprocessors of the device
  const void* occ_fn;    // step kernel variant whose occupancy occ_blocks holds
  int occ_tx, occ_ty, occ_blocks;
  bool rep;              // CG repulsion force enabled (rep_pi != 0)
  void* colour;          // [N] rho^N (step compute type), repulsion pre-pass
  void* normals;         // [3][N] unit colour gradients, repulsion pre-pass
  bool tma_ok;           // tensor maps built: the TMA-staged kernel can run this lattice
  lbm::TmaMaps tma[2];   // maps for reading buffer pair 0 / 1
};

namespace lbm {

constexpr int kDiagThreads = 256;
// Blow-up check: a density below -kNegDensityTol times the larger bulk density (at least 1)
// trips it.  Recolouring moves populations of a colour across a sharp interface with
// either sign, so that colour's density can dip a few 1e-6 below zero on the far side
// (seen at density ratio 12 with A = 0.3); a deficit of a percent only comes from a
// diverging run.
constexpr double kNegDensityTol = 1e-2;

// Workspace layout; returns the total size.  All regions 256-byte aligned.
size_t workspace_layout(const lbm_params& p, lbm_ctx* c /* may be null: size only */);

// Step launchers (one step: fin = f[cur] -> fout = f[cur^1]); return cudaSuccess or the
// launch error.
cudaError_t launch_step_f64(lbm_ctx* c);
cudaError_t launch_step_f32(lbm_ctx* c);
cudaError_t launch_step_f16(lbm_ctx* c);
cudaError_t launch_step_bf16(lbm_ctx* c);
size_t step_smem_for(const lbm_ctx* c, int tx, int ty);
// Encode the tensor maps of both buffer pairs when the lattice suits the TMA-staged
// kernel (D3Q19, FP32/FP16/BF16 storage, nx % 32 == 0, ny % 8 == 0); false otherwise.
bool build_tma_maps(lbm_ctx* c);

// Aux launchers (lbm_aux.cu)
cudaError_t launch_init_eq(lbm_ctx* c, const double* rr, const double* rb, const double* u);
// Checkpoint restore in two passes over the populations: accumulate the densities
// (acc [K][N] FP64), then write deviations relative to them.
cudaError_t launch_restore_accumulate(lbm_ctx* c, const double* plane, int k, double* acc, bool first);
cudaError_t launch_restore_plane(lbm_ctx* c, const double* plane, int k, int i, const double* acc);
cudaError_t launch_export_plane(lbm_ctx* c, double* plane, int k, int i);
cudaError_t launch_export_all(lbm_ctx* c, double* pops);
// In-place streaming at odd parity: stored plane (k, i) of the even layout into out [N]
// (storage type), i.e. slot opp(i) of node x - c_i for every x.
cudaError_t launch_aa_gather_plane(lbm_ctx* c, void* out, int k, int i);
// Densities into stage[0..2N), velocity into u_out (or stage[2N..5N) when null and
// want_u), block partials, then the fixed-order final reduction into c->diag.
cudaError_t launch_diagnostics(lbm_ctx* c, double* u_out, bool want_u);
// Repulsion pre-pass (colour and normal fields) of the current state, for the diagnostics.
cudaError_t launch_rep_prepass(lbm_ctx* c);

// Rest-state equilibrium weights per component and group: Eq. phi with alpha_k for CG
// (alpha_R from Eq. gamma), the lattice weights w for SC.
inline void rest_weights(const lbm_params& q, double phi[2][3]) {
  const bool d3 = q.lattice == LBM_D3Q19;
  for (int k = 0; k < 2; k++) {
    if (q.model == LBM_MODEL_CG) {
      const double alpha = k == 0 ? 1.0 - (1.0 - q.alpha_b) * q.rho_b0 / q.rho_r0 : q.alpha_b;
      phi[k][0] = alpha;
      phi[k][1] = (d3 ? D3Q19::phi_num(1) : D2Q9::phi_num(1)) * (1.0 - alpha);
      phi[k][2] = (d3 ? D3Q19::phi_num(2) : D2Q9::phi_num(2)) * (1.0 - alpha);
    } else {
      for (int g = 0; g < 3; g++) phi[k][g] = d3 ? D3Q19::w(g) : D2Q9::w(g);
    }
  }
}

template <class T>
StepParams<T> make_step_params(const lbm_ctx* c) {
  const lbm_params& q = c->p;
  StepParams<T> s{};
  s.nx = q.nx;
  s.ny = q.ny;
  s.nz = q.nz;
  s.ncx = (q.nx + c->tx - 1) / c->tx;
  s.ncol = s.ncx * ((q.ny + c->ty - 1) / c->ty);
  // chunked grid (tz > 0): one block per unit; a persistent grid (tz = 0) is sized by the
  // launcher (persistent_plan)
  s.nchunks = c->tz > 0 ? (q.nz + c->tz - 1) / c->tz : 1;
  s.nblk = s.ncol * s.nchunks;
  s.n = c->N;
  double phi[2][3];
  rest_weights(q, phi);
  for (int k = 0; k < 2; k++)
    for (int g = 0; g < 3; g++) s.phi[k][g] = T(phi[k][g]);
  s.inv_nu_r = T(3.0 / (q.tau_r - 0.5));
  s.inv_nu_b = T(3.0 / (q.tau_b - 0.5));
  s.A = T(q.A);
  s.beta = T(q.beta);
  s.grad_eps = T(q.grad_eps);
  s.inv_rho_r0 = T(1.0 / q.rho_r0);
  s.inv_rho_b0 = T(1.0 / q.rho_b0);
  s.enhanced = q.enhanced_eq;
  s.color_norm = q.color_norm;
  if (q.model == LBM_MODEL_SC_2C || q.model == LBM_MODEL_SC_MR)
    s.G = T(q.G / (q.rho0_psi * q.rho0_psi));
  else
    s.G = T(q.G);
  for (int k = 0; k < 2; k++) {
    s.Ga[k] = T(q.Ga[k]);
    s.Gr[k] = T(q.Gr[k]);
  }
  s.rho0 = T(q.rho0_psi);
  s.inv_rho0 = T(1.0 / q.rho0_psi);
  s.omega_r = T(1.0 / q.tau_r);
  s.omega_b = T(1.0 / q.tau_b);
  for (int a = 0; a < 3; a++) s.body[a] = T(q.body_force[a]);
  s.has_body = (q.body_force[0] != 0.0 || q.body_force[1] != 0.0 || q.body_force[2] != 0.0);
  return s;
}

}  // namespace lbm
