// C ABI of batched stepping (include/lbm.h, "Batched stepping"): job table upload, one
// persistent launch per step, optional CUDA-graph replay of a multi-step call.
#include <map>
#include <new>
#include <vector>

#include "lbm_batch.cuh"

namespace lbm {
const BatchOps* batch_ops(int precision) {
  switch (precision) {
    case LBM_FP32: return batch_ops_f32();
    case LBM_FP16: return batch_ops_f16();
    case LBM_BF16: return batch_ops_bf16();
    default: return nullptr;
  }
}
}  // namespace lbm

struct lbm_batch {
  int precision;
  const lbm::BatchOps* ops;
  int max_jobs, max_units;
  unsigned char* ws;
  cudaStream_t stream;
  lbm::BatchHeader* d_hdr;
  unsigned char* d_jobs;
  lbm::BatchUnit* d_units;
  size_t smem[2];  // [w]: kernel variant for job lists without / with wall lattices
  int grid[2];
  int walls;       // the current job list holds a lattice with walls
  std::vector<lbm_ctx*> ctxs;
  std::vector<int> remaining;
  std::vector<unsigned char> host_jobs;
  std::vector<lbm::BatchUnit> host_units;
  lbm::BatchHeader host_hdr;
  std::map<int, cudaGraphExec_t> graphs;  // by 2 * nsteps + walls
  unsigned long long launches;
  lbm_status sticky;
};

namespace {

lbm_status bfail(lbm_batch* b, cudaError_t e) {
  if (e == cudaSuccess) return LBM_OK;
  if (b->sticky == LBM_OK) b->sticky = LBM_ECUDA;
  return LBM_ECUDA;
}

int units_of(const lbm_ctx* c) {
  const int ncol = ((c->p.nx + lbm::kBatchTX - 1) / lbm::kBatchTX) * ((c->p.ny + lbm::kBatchTY - 1) / lbm::kBatchTY);
  const int nch = c->p.lattice == LBM_D3Q19 ? (c->p.nz + lbm::batch_chunk(c) - 1) / lbm::batch_chunk(c) : 1;
  return ncol * nch;
}

// Graph of n launches in a chain; node s carries the step index s.
cudaError_t build_graph(lbm_batch* b, int n, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  cudaGraphNode_t prev = nullptr;
  for (int s = 0; s < n && e == cudaSuccess; s++) {
    const lbm::BatchHeader* hdr = b->d_hdr;
    const void* jobs = b->d_jobs;
    const lbm::BatchUnit* units = b->d_units;
    int sv = s;
    void* args[4] = {&hdr, &jobs, &units, &sv};
    cudaKernelNodeParams kp = {};
    kp.func = const_cast<void*>(b->ops->kernel[b->walls]);
    kp.gridDim = dim3(b->grid[b->walls], 1, 1);
    kp.blockDim = dim3(lbm::kBatchTX, lbm::kBatchTY, 1);
    kp.sharedMemBytes = (unsigned)b->smem[b->walls];
    kp.kernelParams = args;
    cudaGraphNode_t node;
    e = cudaGraphAddKernelNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
    prev = node;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return e;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(int32_t precision, int32_t max_jobs, int32_t max_units, void* ws, size_t* ws_bytes,
                            void* stream, lbm_batch** out) {
  const lbm::BatchOps* ops = lbm::batch_ops(precision);
  if (!ops || !ws_bytes || max_jobs < 1 || max_units < 1) return LBM_EINVAL;
  const size_t need = ops->ws_bytes(max_jobs, max_units);
  if (!ws) {
    *ws_bytes = need;
    return LBM_OK;
  }
  if (!out || (reinterpret_cast<uintptr_t>(ws) & 255) != 0) return LBM_EINVAL;
  if (*ws_bytes < need) return LBM_ENOMEM;
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_ENOMEM;
  b->precision = precision;
  b->ops = ops;
  b->max_jobs = max_jobs;
  b->max_units = max_units;
  b->ws = static_cast<unsigned char*>(ws);
  b->stream = static_cast<cudaStream_t>(stream);
  b->d_hdr = reinterpret_cast<lbm::BatchHeader*>(b->ws);
  b->d_jobs = b->ws + lbm::align256b(sizeof(lbm::BatchHeader));
  b->d_units = reinterpret_cast<lbm::BatchUnit*>(b->d_jobs + lbm::align256b(ops->job_bytes * size_t(max_jobs)));
  b->smem[0] = ops->smem_bytes(false);
  b->smem[1] = ops->smem_bytes(true);
  b->walls = 0;
  b->launches = 0;
  b->sticky = LBM_OK;
  b->host_hdr = {0, 0};
  int dev = 0, nsm = 1, per_sm[2] = {1, 1};
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = ops->prepare(false, b->smem[0], &per_sm[0]);
  if (e == cudaSuccess) e = ops->prepare(true, b->smem[1], &per_sm[1]);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_hdr, &b->host_hdr, sizeof(lbm::BatchHeader), cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) {
    delete b;
    return LBM_ECUDA;
  }
  for (int w = 0; w < 2; w++) b->grid[w] = std::max(1, nsm * std::max(1, per_sm[w]));
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_units(const lbm_ctx* c, int32_t* units) {
  if (!c || !units) return LBM_EINVAL;
  *units = units_of(c);
  return LBM_OK;
}

lbm_status lbm_batch_set(lbm_batch* b, lbm_ctx* const* ctxs, const int32_t* nsteps, int32_t njobs) {
  if (!b || njobs < 0 || njobs > b->max_jobs || (njobs > 0 && (!ctxs || !nsteps))) return LBM_EINVAL;
  if (b->sticky != LBM_OK) return b->sticky;
  long long nunits = 0;
  for (int j = 0; j < njobs; j++) {
    const lbm_ctx* c = ctxs[j];
    if (!c || nsteps[j] < 0) return LBM_EINVAL;
    if (c->sticky != LBM_OK || !c->initialised) return LBM_ESTATE;
    if (c->p.precision != b->precision || c->rep || c->aa || c->p.model == LBM_MODEL_SC_MR ||
        c->stream != b->stream)
      return LBM_EINVAL;
    // the batched kernel indexes in 32 bits
    if ((long long)c->K * c->Q * c->N >= (1LL << 31)) return LBM_EINVAL;
    nunits += units_of(c);
  }
  if (nunits > b->max_units) return LBM_EINVAL;
  b->walls = 0;
  for (int j = 0; j < njobs; j++) b->walls |= ctxs[j]->has_walls ? 1 : 0;
  b->ctxs.assign(ctxs, ctxs + njobs);
  b->remaining.assign(nsteps, nsteps + njobs);
  b->host_jobs.assign(b->ops->job_bytes * size_t(njobs), 0);
  b->host_units.clear();
  for (int j = 0; j < njobs; j++) {
    b->ops->fill_job(ctxs[j], nsteps[j], b->host_jobs.data() + b->ops->job_bytes * j);
    const int nu = units_of(ctxs[j]);
    const int ncol = ((ctxs[j]->p.nx + lbm::kBatchTX - 1) / lbm::kBatchTX) *
                     ((ctxs[j]->p.ny + lbm::kBatchTY - 1) / lbm::kBatchTY);
    for (int u = 0; u < nu; u++) b->host_units.push_back(lbm::BatchUnit{j, u % ncol, u / ncol});
  }
  b->host_hdr = {njobs, (int)nunits};
  cudaError_t e = cudaSuccess;
  if (nunits > 0)
    e = cudaMemcpyAsync(b->d_units, b->host_units.data(), sizeof(lbm::BatchUnit) * nunits, cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess && njobs > 0)
    e = cudaMemcpyAsync(b->d_jobs, b->host_jobs.data(), b->host_jobs.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_hdr, &b->host_hdr, sizeof(lbm::BatchHeader), cudaMemcpyHostToDevice, b->stream);
  return bfail(b, e);
}

lbm_status lbm_batch_step(lbm_batch* b, int32_t nsteps, int32_t use_graph) {
  if (!b || nsteps < 0) return LBM_EINVAL;
  if (b->sticky != LBM_OK) return b->sticky;
  const int njobs = (int)b->ctxs.size();
  if (nsteps == 0 || njobs == 0) return LBM_OK;
  for (int j = 0; j < njobs; j++)
    if (b->ctxs[j]->sticky != LBM_OK) return LBM_ESTATE;
  // per-job buffer pair and step count of this call
  for (int j = 0; j < njobs; j++) {
    const int take = std::min(nsteps, b->remaining[j]);
    b->ops->fill_job(b->ctxs[j], take, b->host_jobs.data() + b->ops->job_bytes * j);
  }
  cudaError_t e = cudaMemcpyAsync(b->d_jobs, b->host_jobs.data(), b->host_jobs.size(), cudaMemcpyHostToDevice,
                                  b->stream);
  if (e != cudaSuccess) return bfail(b, e);
  if (use_graph) {
    const int key = 2 * nsteps + b->walls;
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
      cudaGraphExec_t ex = nullptr;
      e = build_graph(b, nsteps, &ex);
      if (e != cudaSuccess) return bfail(b, e);
      it = b->graphs.emplace(key, ex).first;
    }
    e = cudaGraphLaunch(it->second, b->stream);
  } else {
    for (int s = 0; s < nsteps && e == cudaSuccess; s++) {
      const lbm::BatchHeader* hdr = b->d_hdr;
      const void* jobs = b->d_jobs;
      const lbm::BatchUnit* units = b->d_units;
      int sv = s;
      void* args[4] = {&hdr, &jobs, &units, &sv};
      e = cudaLaunchKernel(b->ops->kernel[b->walls], dim3(b->grid[b->walls], 1, 1),
                           dim3(lbm::kBatchTX, lbm::kBatchTY, 1), args, b->smem[b->walls], b->stream);
    }
  }
  if (e != cudaSuccess) return bfail(b, e);
  b->launches += (unsigned long long)nsteps;
  for (int j = 0; j < njobs; j++) {
    const int take = std::min(nsteps, b->remaining[j]);
    b->remaining[j] -= take;
    lbm_ctx* c = b->ctxs[j];
    c->cur ^= (take & 1);
    c->steps += take;
  }
  return LBM_OK;
}

uint64_t lbm_batch_launch_count(const lbm_batch* b) { return b ? b->launches : 0; }

lbm_status lbm_batch_destroy(lbm_batch* b) {
  if (!b) return LBM_OK;
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  delete b;
  return LBM_OK;
}

}  // extern "C"
