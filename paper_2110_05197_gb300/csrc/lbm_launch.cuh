// Launch helper for the fused step kernel (one instantiation per lattice, storage
// precision, model and wall variant).
#pragma once

#include "lbm_internal.cuh"

namespace lbm {

template <class L, class T, class S, class RT, int MODEL, bool WALLS>
cudaError_t launch_step_t(lbm_ctx* c) {
  const int tx = c->tx, ty = c->ty;
  const size_t smem = step_smem_bytes<L, T, MODEL, WALLS>(tx, ty);
  static size_t smem_set = 0;  // largest dynamic shared memory opted in so far
  if (smem > 48 * 1024 && smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(step_kernel<L, T, S, RT, MODEL, WALLS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    smem_set = smem;
  }
  dim3 block(tx, ty, 1);
  dim3 grid((c->p.nx + tx - 1) / tx, (c->p.ny + ty - 1) / ty, (c->p.nz + c->tz - 1) / c->tz);
  const StepParams<T> sp = make_step_params<T>(c);
  const S* fin = static_cast<const S*>(c->f[c->cur]);
  S* fout = static_cast<S*>(c->f[c->cur ^ 1]);
  const RT* rin = static_cast<const RT*>(c->r[c->cur]);
  RT* rout = static_cast<RT*>(c->r[c->cur ^ 1]);
  step_kernel<L, T, S, RT, MODEL, WALLS><<<grid, block, smem, c->stream>>>(fin, fout, rin, rout, c->solid,
                                                                          &c->diag->status, sp);
  return cudaGetLastError();
}

template <class T, class S, class RT, int MODEL>
cudaError_t dispatch_lattice(lbm_ctx* c) {
  const bool w = c->has_walls;
  if (c->p.lattice == LBM_D3Q19)
    return w ? launch_step_t<D3Q19, T, S, RT, MODEL, true>(c) : launch_step_t<D3Q19, T, S, RT, MODEL, false>(c);
  return w ? launch_step_t<D2Q9, T, S, RT, MODEL, true>(c) : launch_step_t<D2Q9, T, S, RT, MODEL, false>(c);
}

template <class T, class S, class RT>
cudaError_t dispatch_model(lbm_ctx* c) {
  if (c->p.model == LBM_MODEL_CG) return dispatch_lattice<T, S, RT, kCG>(c);
  if (c->p.model == LBM_MODEL_SC_MP) return dispatch_lattice<T, S, RT, kSCMP>(c);
  return dispatch_lattice<T, S, RT, kSC2C>(c);
}


}  // namespace lbm
