// C ABI of liblbm.so (declared in include/lbm.h): context creation over a caller-owned
// workspace, initial state, stepping and moments.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>

#include <cudaTypedefs.h>

#include "lbm_internal.cuh"

namespace {

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

bool params_ok(const lbm_params* p) {
  if (!p) return false;
  if (p->lattice != LBM_D2Q9 && p->lattice != LBM_D3Q19) return false;
  if (p->model < LBM_MODEL_CG || p->model > LBM_MODEL_SC_MR) return false;
  // the multirange model's repulsion reaches distance 2 (D3Q19 belts)
  if (p->model == LBM_MODEL_SC_MR && (p->lattice != LBM_D3Q19 || p->nx < 2 || p->ny < 2 || p->nz < 2)) return false;
  if (p->precision < LBM_FP64 || p->precision > LBM_BF16) return false;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return false;
  if (p->lattice == LBM_D2Q9 && p->nz != 1) return false;
  const long long n = (long long)p->nx * p->ny * p->nz;
  if (n > (1LL << 31)) return false;
  if (!(p->tau_r > 0.5)) return false;
  if (p->model != LBM_MODEL_SC_MP && !(p->tau_b > 0.5)) return false;
  if (p->model == LBM_MODEL_CG) {
    if (!(p->rho_r0 > 0) || !(p->rho_b0 > 0) || !(p->alpha_b >= 0 && p->alpha_b < 1)) return false;
    const double ar = 1.0 - (1.0 - p->alpha_b) * p->rho_b0 / p->rho_r0;
    if (!(ar >= 0 && ar < 1)) return false;
    if (!(p->grad_eps >= 0)) return false;
  } else {
    if (!(p->rho0_psi > 0)) return false;
  }
  if (p->diag_every < 0) return false;
  if (p->streaming != LBM_STREAM_AB && p->streaming != LBM_STREAM_AA) return false;
  return true;
}

bool is_device_ptr(const void* ptr) {
  if (!ptr) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

lbm_status fail(lbm_ctx* c, cudaError_t e) {
  if (e == cudaSuccess) return LBM_OK;
  if (c->sticky == LBM_OK) c->sticky = LBM_ECUDA;
  return LBM_ECUDA;
}

// Device view of a caller buffer of `bytes`: the pointer itself when it is device
// memory, otherwise `stage` after an H2D copy.
cudaError_t stage_in(lbm_ctx* c, const void* src, size_t bytes, void* stage, const void** dev, bool* host) {
  if (is_device_ptr(src)) {
    *dev = src;
    return cudaSuccess;
  }
  *host = true;
  *dev = stage;
  return cudaMemcpyAsync(stage, src, bytes, cudaMemcpyHostToDevice, c->stream);
}

cudaError_t copy_out(lbm_ctx* c, void* dst, const void* src, size_t bytes, bool* host) {
  if (!is_device_ptr(dst)) *host = true;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream);
}

}  // namespace

namespace lbm {

size_t workspace_layout(const lbm_params& p, lbm_ctx* c) {
  const int K = p.model == LBM_MODEL_SC_MP ? 1 : 2;
  const int Q = p.lattice == LBM_D3Q19 ? 19 : 9;
  const long long N = (long long)p.nx * p.ny * p.nz;
  const size_t elt = p.precision == LBM_FP64 ? 8 : (p.precision == LBM_FP32 ? 4 : 2);
  const size_t relt = p.precision == LBM_FP64 ? 8 : 4;
  const int nblk = (int)std::min<long long>((N + kDiagThreads - 1) / kDiagThreads, 1184);
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t o = off;
    off += align256(b);
    return o;
  };
  // in-place streaming: one population buffer and one reference field
  const bool aa = p.streaming == LBM_STREAM_AA;
  const size_t of0 = take((size_t)K * Q * N * elt);
  const size_t of1 = aa ? of0 : take((size_t)K * Q * N * elt);
  const size_t or0 = take((size_t)K * N * relt);
  const size_t or1 = aa ? or0 : take((size_t)K * N * relt);
  const size_t osol = take((size_t)N);
  // staging: rho_r, rho_b, momentum/velocity (3), then psi (SC multiphase) or the two
  // multirange Psi_s in the compute type (a seventh row for FP64 storage)
  const int stage_rows = (p.model == LBM_MODEL_SC_MR && p.precision == LBM_FP64) ? 7 : 6;
  const size_t ostg = take((size_t)stage_rows * N * sizeof(double));
  const size_t opar = take((size_t)nblk * LBM_NTOTALS * sizeof(double));
  const size_t odia = take(sizeof(lbm_diag));
  const bool rep = p.model == LBM_MODEL_CG && p.rep_pi != 0.0;
  const size_t tsz = p.precision == LBM_FP64 ? 8 : 4;  // step compute type
  const size_t ocol = rep ? take((size_t)N * tsz) : 0;
  const size_t onrm = rep ? take((size_t)3 * N * tsz) : 0;
  if (c) {
    c->K = K;
    c->Q = Q;
    c->N = N;
    c->elt = elt;
    c->relt = relt;
    c->aa = aa;
    c->f[0] = c->ws + of0;
    c->f[1] = c->ws + of1;
    c->r[0] = c->ws + or0;
    c->r[1] = c->ws + or1;
    c->solid = reinterpret_cast<uint8_t*>(c->ws + osol);
    c->stage = reinterpret_cast<double*>(c->ws + ostg);
    c->partials = reinterpret_cast<double*>(c->ws + opar);
    c->nblk_diag = nblk;
    c->diag = reinterpret_cast<lbm_diag*>(c->ws + odia);
    c->rep = rep;
    c->colour = rep ? c->ws + ocol : nullptr;
    c->normals = rep ? c->ws + onrm : nullptr;
  }
  return off;
}

size_t step_smem_for(const lbm_ctx* c, int tx, int ty) {
  const size_t ne = size_t(tx + 2) * (ty + 2), ni = size_t(tx) * ty;
  const int npl = c->p.lattice == LBM_D3Q19 ? 3 : 1;
  const int nf = c->p.model == LBM_MODEL_SC_MP ? 1 : 2;
  const size_t t = c->p.precision == LBM_FP64 ? 8 : 4;  // compute type
  return npl * (nf + c->K) * ne * t + 2 * c->K * (c->Q + 1) * ni * t + (c->has_walls ? npl * ne : 0);
}

static cudaError_t launch_step(lbm_ctx* c) {
  switch (c->p.precision) {
    case LBM_FP64: return launch_step_f64(c);
    case LBM_FP32: return launch_step_f32(c);
    case LBM_FP16: return launch_step_f16(c);
    default: return launch_step_bf16(c);
  }
}

using EncodeFn = PFN_cuTensorMapEncodeTiled_v12000;

static EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(f);
    else
      cudaGetLastError();
  }
  return fn;
}

// 4-D view (x, array, y, z) of a [arrays][z][y][x] buffer with boxes {bx, arrays, rows, 1}.
static bool encode4(EncodeFn fn, CUtensorMap* m, CUtensorMapDataType dt, size_t elt, void* base, int nx, int ny,
                    int nz, int arrays, long long n, int bx, int rows) {
  const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)arrays, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[3] = {(cuuint64_t)(n * elt), (cuuint64_t)nx * elt, (cuuint64_t)nx * ny * elt};
  const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)arrays, (cuuint32_t)rows, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(m, dt, 4, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool build_tma_maps(lbm_ctx* c) {
  const lbm_params& p = c->p;
  if (p.lattice != LBM_D3Q19 || p.precision == LBM_FP64 || c->aa) return false;
  if (p.nx % kTmaTX != 0 || p.ny % kTmaTY != 0) return false;
  const int K = c->K, Q = c->Q;
  if (K * Q > 256) return false;
  EncodeFn fn = encode_fn();
  if (!fn) return false;
  const CUtensorMapDataType dt = p.precision == LBM_FP32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : p.precision == LBM_FP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                           : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  for (int b = 0; b < 2; b++) {
    TmaMaps& m = c->tma[b];
    bool ok = encode4(fn, &m.pop_main_row, dt, c->elt, c->f[b], p.nx, p.ny, p.nz, K * Q, c->N, kTmaTX, 1) &&
              encode4(fn, &m.pop_main_mid, dt, c->elt, c->f[b], p.nx, p.ny, p.nz, K * Q, c->N, kTmaTX, kTmaTY) &&
              encode4(fn, &m.ref_main_row, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, c->relt, c->r[b], p.nx, p.ny, p.nz, K,
                      c->N, kTmaTX, 1) &&
              encode4(fn, &m.ref_main_mid, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, c->relt, c->r[b], p.nx, p.ny, p.nz, K,
                      c->N, kTmaTX, kTmaTY) &&
              encode4(fn, &m.pop_main_mid4, dt, c->elt, c->f[b], p.nx, p.ny, p.nz, K * Q, c->N, kTmaTX, 4) &&
              encode4(fn, &m.ref_main_mid4, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, c->relt, c->r[b], p.nx, p.ny, p.nz, K,
                      c->N, kTmaTX, 4);
    if (ok && p.nx % 64 == 0)
      ok = encode4(fn, &m.pop_w_row, dt, c->elt, c->f[b], p.nx, p.ny, p.nz, K * Q, c->N, 64, 1) &&
           encode4(fn, &m.pop_w_mid4, dt, c->elt, c->f[b], p.nx, p.ny, p.nz, K * Q, c->N, 64, 4) &&
           encode4(fn, &m.ref_w_row, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, c->relt, c->r[b], p.nx, p.ny, p.nz, K, c->N,
                   64, 1) &&
           encode4(fn, &m.ref_w_mid4, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, c->relt, c->r[b], p.nx, p.ny, p.nz, K, c->N,
                   64, 4);
    if (!ok) return false;
    // tiles of the ring kernel (lbm_step_ring.cuh); optional: without them that kernel is
    // not used
    m.mid16 = p.ny % 16 == 0 &&
              encode4(fn, &m.pop_main_mid16, dt, c->elt, c->f[b], p.nx, p.ny, p.nz, K * Q, c->N, kTmaTX, 16) &&
              encode4(fn, &m.ref_main_mid16, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, c->relt, c->r[b], p.nx, p.ny, p.nz, K,
                      c->N, kTmaTX, 16);
    m.w_mid8 = p.nx % 64 == 0 && p.ny % 8 == 0 &&
               encode4(fn, &m.pop_w_mid8, dt, c->elt, c->f[b], p.nx, p.ny, p.nz, K * Q, c->N, 64, 8) &&
               encode4(fn, &m.ref_w_mid8, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, c->relt, c->r[b], p.nx, p.ny, p.nz, K,
                       c->N, 64, 8);
  }
  return true;
}

}  // namespace lbm

extern "C" {

const char* lbm_status_string(lbm_status s) {
  switch (s) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "workspace too small";
    case LBM_ECUDA: return "CUDA error";
    case LBM_EUNSTABLE: return "simulation unstable (blow-up check tripped)";
    case LBM_ESTATE: return "call does not fit the context state or model";
    case LBM_ETIMEOUT: return "bounded device wait timed out";
  }
  return "unknown status";
}

lbm_status lbm_create(const lbm_params* p, void* ws, size_t* ws_bytes, void* stream, lbm_ctx** out) {
  if (!p || !ws_bytes || !params_ok(p)) return LBM_EINVAL;
  const size_t need = lbm::workspace_layout(*p, nullptr);
  if (!ws) {
    *ws_bytes = need;
    return LBM_OK;
  }
  if (!out) return LBM_EINVAL;
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return LBM_EINVAL;
  if (*ws_bytes < need) return LBM_ENOMEM;
  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_ENOMEM;
  c->p = *p;
  c->stream = static_cast<cudaStream_t>(stream);
  c->ws = static_cast<unsigned char*>(ws);
  c->ws_bytes = *ws_bytes;
  lbm::workspace_layout(*p, c);
  c->cur = 0;
  c->has_walls = false;
  c->initialised = false;
  c->sticky = LBM_OK;
  c->launches = 0;
  c->steps = 0;
  c->tx = 32;
  c->ty = 8;
  c->tz = p->lattice == LBM_D3Q19 ? (p->nz < 16 ? p->nz : 16) : 1;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    nsm = 0;
  c->nsm = nsm > 0 ? nsm : 1;
  c->occ_fn = nullptr;
  c->tma_ok = lbm::build_tma_maps(c);
  *out = c;
  return LBM_OK;
}

lbm_status lbm_set_tiling(lbm_ctx* c, int32_t tx, int32_t ty, int32_t tz) {
  if (!c) return LBM_EINVAL;
  // 512-node tiles (32 x 16, 64 x 8) select the ring kernel; where it does not apply the
  // step runs the 32 x 8 tiling instead
  const bool ring = (tx == 32 && ty == 16) || (tx == 64 && ty == 8);
  if (tx < 1 || ty < 1 || tz < 0 || (tx * ty > 256 && !ring) || (tx * ty) % 32 != 0) return LBM_EINVAL;
  if (ring && c->p.lattice != LBM_D3Q19) return LBM_EINVAL;
  if (c->p.lattice == LBM_D2Q9 && tz > 1) return LBM_EINVAL;
  c->tx = tx;
  c->ty = ty;
  c->tz = tz;
  return LBM_OK;
}

lbm_status lbm_init_fields(lbm_ctx* c, const double* rho_r, const double* rho_b, const double* u,
                           const uint8_t* solid, const double* pops) {
  if (!c) return LBM_EINVAL;
  if (c->sticky != LBM_OK) return c->sticky;
  if (!rho_r) return LBM_EINVAL;
  if (c->K == 2 && !rho_b && !pops) return LBM_EINVAL;
  const long long N = c->N;
  bool host = false;
  cudaError_t e;
  // wall mask
  if (solid) {
    if (is_device_ptr(solid))
      e = cudaMemcpyAsync(c->solid, solid, N, cudaMemcpyDeviceToDevice, c->stream);
    else {
      host = true;
      e = cudaMemcpyAsync(c->solid, solid, N, cudaMemcpyHostToDevice, c->stream);
    }
    c->has_walls = true;
  } else {
    e = cudaMemsetAsync(c->solid, 0, N, c->stream);
    c->has_walls = false;
  }
  if (e != cudaSuccess) return fail(c, e);
  if (pops) {
    // pass 1: component densities into stage[0, K*N); pass 2: deviations relative to them
    const bool dev = is_device_ptr(pops);
    double* acc = c->stage;
    double* buf = c->stage + 2 * N;
    for (int pass = 0; pass < 2; pass++)
      for (int k = 0; k < c->K; k++)
        for (int i = 0; i < c->Q; i++) {
          const double* src = pops + (size_t)(k * c->Q + i) * N;
          const double* plane = src;
          if (!dev) {
            host = true;
            e = cudaMemcpyAsync(buf, src, N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
            if (e != cudaSuccess) return fail(c, e);
            plane = buf;
          }
          e = pass == 0 ? lbm::launch_restore_accumulate(c, plane, k, acc, i == 0)
                        : lbm::launch_restore_plane(c, plane, k, i, acc);
          if (e != cudaSuccess) return fail(c, e);
        }
  } else {
    const void *drr = nullptr, *drb = nullptr, *du = nullptr;
    e = stage_in(c, rho_r, N * sizeof(double), c->stage, &drr, &host);
    if (e == cudaSuccess && c->K == 2) e = stage_in(c, rho_b, N * sizeof(double), c->stage + N, &drb, &host);
    if (e == cudaSuccess && u) e = stage_in(c, u, 3 * N * sizeof(double), c->stage + 2 * N, &du, &host);
    if (e != cudaSuccess) return fail(c, e);
    if (c->K == 1) drb = drr;  // unused by the multiphase equilibrium
    e = lbm::launch_init_eq(c, static_cast<const double*>(drr), static_cast<const double*>(drb),
                            static_cast<const double*>(du));
    if (e != cudaSuccess) return fail(c, e);
  }
  e = cudaMemsetAsync(c->diag, 0, sizeof(lbm_diag), c->stream);
  if (e != cudaSuccess) return fail(c, e);
  if (host) {
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, e);
  }
  c->cur = 0;
  c->steps = 0;
  c->initialised = true;
  return LBM_OK;
}

static lbm_status step_common(lbm_ctx* c, int32_t nsteps, bool cg) {
  if (!c || nsteps < 0) return LBM_EINVAL;
  if (c->sticky != LBM_OK) return c->sticky;
  if (!c->initialised) return LBM_ESTATE;
  if (cg != (c->p.model == LBM_MODEL_CG)) return LBM_ESTATE;
  for (int s = 0; s < nsteps; s++) {
    cudaError_t e = lbm::launch_step(c);
    if (e != cudaSuccess) return fail(c, e);
    c->launches += 1;
    c->cur ^= 1;
    c->steps += 1;
    if (c->p.diag_every > 0 && c->steps % c->p.diag_every == 0) {
      e = lbm::launch_diagnostics(c, nullptr, false);
      if (e != cudaSuccess) return fail(c, e);
    }
  }
  return LBM_OK;
}

lbm_status lbm_step_cg(lbm_ctx* c, int32_t nsteps) { return step_common(c, nsteps, true); }
lbm_status lbm_step_sc(lbm_ctx* c, int32_t nsteps) { return step_common(c, nsteps, false); }

lbm_status lbm_moments(lbm_ctx* c, double* rho_r, double* rho_b, double* u, double* pops, double* totals) {
  if (!c) return LBM_EINVAL;
  if (c->sticky != LBM_OK) return c->sticky;
  if (!c->initialised) return LBM_ESTATE;
  const long long N = c->N;
  bool host = false;
  cudaError_t e = cudaSuccess;
  const bool need_diag = rho_r || rho_b || u || totals;
  if (need_diag) {
    double* u_dev = (u && is_device_ptr(u)) ? u : nullptr;
    e = lbm::launch_diagnostics(c, u_dev, u != nullptr);
    if (e != cudaSuccess) return fail(c, e);
    if (rho_r) e = copy_out(c, rho_r, c->stage, N * sizeof(double), &host);
    if (e == cudaSuccess && rho_b) e = copy_out(c, rho_b, c->stage + N, N * sizeof(double), &host);
    if (e == cudaSuccess && u && !u_dev) e = copy_out(c, u, c->stage + 2 * N, 3 * N * sizeof(double), &host);
    if (e != cudaSuccess) return fail(c, e);
  }
  if (pops) {
    if (is_device_ptr(pops)) {
      e = lbm::launch_export_all(c, pops);
      if (e != cudaSuccess) return fail(c, e);
    } else {
      host = true;
      // the staged densities/velocity were already copied out (stream order)
      for (int k = 0; k < c->K; k++)
        for (int i = 0; i < c->Q; i++) {
          e = lbm::launch_export_plane(c, c->stage, k, i);
          if (e == cudaSuccess)
            e = cudaMemcpyAsync(pops + (size_t)(k * c->Q + i) * N, c->stage, N * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream);
          if (e != cudaSuccess) return fail(c, e);
        }
    }
  }
  lbm_diag hd;
  if (totals) {
    e = cudaMemcpyAsync(&hd, c->diag, sizeof(lbm_diag), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return fail(c, e);
    host = true;
  }
  if (host) {
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, e);
  }
  if (totals) {
    std::memcpy(totals, hd.totals, sizeof(hd.totals));
    if (hd.status & (lbm::kStatusTimeout | lbm::kStatusLayout)) return LBM_ETIMEOUT;
    if (hd.status != 0) return LBM_EUNSTABLE;
  }
  return LBM_OK;
}

lbm_status lbm_destroy(lbm_ctx* c) {
  delete c;
  return LBM_OK;
}

uint64_t lbm_launch_count(const lbm_ctx* c) { return c ? c->launches : 0; }

size_t lbm_state_bytes(const lbm_ctx* c) {
  if (!c) return 0;
  return (size_t)c->K * c->Q * c->N * c->elt + (size_t)c->K * c->N * c->relt;
}

lbm_status lbm_save_state(lbm_ctx* c, void* dst) {
  if (!c || !dst) return LBM_EINVAL;
  if (c->sticky != LBM_OK) return c->sticky;
  if (!c->initialised) return LBM_ESTATE;
  // the blow-up status decides which buffer pair is the state; read it first
  lbm_diag hd;
  cudaError_t e = cudaMemcpyAsync(&hd, c->diag, sizeof(lbm_diag), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, e);
  const int b = hd.status ? hd.trip_buf : c->cur;
  const size_t fb = (size_t)c->K * c->Q * c->N * c->elt;
  if (c->aa && (b & 1)) {
    // odd in-place layout: gather each population plane into the even (canonical slot)
    // layout through the staging buffer, so that a saved state always loads at parity 0
    const size_t pb = (size_t)c->N * c->elt;
    for (int k = 0; k < c->K && e == cudaSuccess; k++)
      for (int i = 0; i < c->Q && e == cudaSuccess; i++) {
        e = lbm::launch_aa_gather_plane(c, c->stage, k, i);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(static_cast<char*>(dst) + (size_t)(k * c->Q + i) * pb, c->stage, pb, cudaMemcpyDefault,
                              c->stream);
      }
  } else {
    e = cudaMemcpyAsync(dst, c->f[b], fb, cudaMemcpyDefault, c->stream);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(static_cast<char*>(dst) + fb, c->r[b], (size_t)c->K * c->N * c->relt, cudaMemcpyDefault,
                        c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, e);
  return hd.status ? LBM_EUNSTABLE : LBM_OK;
}

size_t lbm_state_planes_bytes(const lbm_ctx* c, int32_t nplanes) {
  if (!c || nplanes < 1) return 0;
  const size_t per = (size_t)nplanes * c->p.nx * c->p.ny;
  return per * ((size_t)c->K * c->Q * c->elt + (size_t)c->K * c->relt);
}

namespace {
// Copies between the current buffer pair's planes [z0, z0 + np) and a packed buffer:
// every population array's planes, then every reference array's (to_buf: state -> buf).
lbm_status copy_planes(lbm_ctx* c, int32_t z0, int32_t np, void* buf, bool to_buf) {
  if (!c || !buf || z0 < 0 || np < 1 || z0 + np > c->p.nz) return LBM_EINVAL;
  if (c->sticky != LBM_OK) return c->sticky;
  if (!c->initialised || c->aa) return LBM_ESTATE;
  const size_t plane = (size_t)c->p.nx * c->p.ny;
  const size_t pb = np * plane * c->elt, rb = np * plane * c->relt;
  unsigned char* f = static_cast<unsigned char*>(c->f[c->cur]);
  unsigned char* r = static_cast<unsigned char*>(c->r[c->cur]);
  unsigned char* b = static_cast<unsigned char*>(buf);
  cudaError_t e = cudaSuccess;
  for (int a = 0; a < c->K * c->Q && e == cudaSuccess; a++) {
    unsigned char* st = f + ((size_t)a * c->N + z0 * plane) * c->elt;
    unsigned char* bb = b + a * pb;
    e = to_buf ? cudaMemcpyAsync(bb, st, pb, cudaMemcpyDefault, c->stream)
               : cudaMemcpyAsync(st, bb, pb, cudaMemcpyDefault, c->stream);
  }
  for (int k = 0; k < c->K && e == cudaSuccess; k++) {
    unsigned char* st = r + ((size_t)k * c->N + z0 * plane) * c->relt;
    unsigned char* bb = b + (size_t)c->K * c->Q * pb + k * rb;
    e = to_buf ? cudaMemcpyAsync(bb, st, rb, cudaMemcpyDefault, c->stream)
               : cudaMemcpyAsync(st, bb, rb, cudaMemcpyDefault, c->stream);
  }
  return e == cudaSuccess ? LBM_OK : fail(c, e);
}
}  // namespace

lbm_status lbm_get_state_planes(lbm_ctx* c, int32_t z0, int32_t nplanes, void* buf) {
  return copy_planes(c, z0, nplanes, buf, true);
}

lbm_status lbm_set_state_planes(lbm_ctx* c, int32_t z0, int32_t nplanes, const void* buf) {
  return copy_planes(c, z0, nplanes, const_cast<void*>(buf), false);
}

lbm_status lbm_load_state(lbm_ctx* c, const void* src, const uint8_t* solid) {
  if (!c || !src) return LBM_EINVAL;
  if (c->sticky != LBM_OK) return c->sticky;
  const long long N = c->N;
  cudaError_t e;
  if (solid) {
    e = cudaMemcpyAsync(c->solid, solid, N, cudaMemcpyDefault, c->stream);
    c->has_walls = true;
  } else {
    e = cudaMemsetAsync(c->solid, 0, N, c->stream);
    c->has_walls = false;
  }
  const size_t fb = (size_t)c->K * c->Q * N * c->elt;
  const size_t rb = (size_t)c->K * N * c->relt;
  for (int b = 0; b < (c->aa ? 1 : 2) && e == cudaSuccess; b++) {
    e = cudaMemcpyAsync(c->f[b], src, fb, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->r[b], static_cast<const char*>(src) + fb, rb, cudaMemcpyDefault, c->stream);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(c->diag, 0, sizeof(lbm_diag), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, e);
  c->cur = 0;
  c->steps = 0;
  c->initialised = true;
  return LBM_OK;
}

}  // extern "C"
