// Batched stepping: many lattices advance in one persistent launch driven by a job table.
//
// Every lattice of a batch (a "job": one lbm_ctx) is cut into work units of 32 x 8 node
// columns and z-chunks of at most tz planes (the job's tiling; 16 by default); the unit
// list of all jobs sits in device
// memory beside the job descriptors (array pointers, StepParams, the buffer pair holding
// the state, the steps the job still takes).  One launch advances every job by one step:
// a persistent grid walks the unit list with a stride, loads the unit's job descriptor
// into shared memory and marches the unit with the same per-node code as the generic
// step kernel (march_segment), dispatching on the job's lattice, model and wall mask.  A job's result
// is therefore bitwise the same alone or in any mix.  Launch s of a multi-step call reads
// the pair cur0 ^ (s & 1) and skips jobs with fewer than s + 1 steps left, so a whole call
// can be replayed as one CUDA graph whose nodes differ only in s.
#pragma once

#include <algorithm>

#include "lbm_internal.cuh"

struct lbm_batch;

namespace lbm {

constexpr int kBatchTX = 32, kBatchTY = 8;  // block shape of the batched kernel
constexpr int kBatchChunk = 16;            // default z planes per work unit (3-D lattices)

// z planes per work unit of a job: the context's own tz (lbm_set_tiling) when it is set,
// else kBatchChunk.  Shorter chunks give small lattices more units (more of the GPU) at
// the price of two halo planes per unit.
inline int batch_chunk(const lbm_ctx* c) { return c->tz > 0 ? c->tz : kBatchChunk; }

template <class T, class S, class RT>
struct BatchJob {
  S* f[2];         // population buffer pair
  RT* r[2];        // reference density pair (written by the step that reads the other)
  const int* status;
  const uint8_t* solid;  // wall mask [N] (halfway bounce-back), or nullptr
  int lattice, model;
  int walls;       // solid != nullptr
  int cur0;        // pair holding the state when the call starts
  int nsteps;      // steps this job takes in the call
  StepParams<T> p;
};

struct BatchUnit {
  int job, col, chunk;
};

struct BatchHeader {
  int njobs, nunits;
};

// Workspace: header, then jobs[max_jobs], then units[max_units] (256-byte aligned parts).
inline size_t align256b(size_t b) { return (b + 255) & ~size_t(255); }
template <class T, class S, class RT>
size_t batch_ws_bytes(int max_jobs, int max_units) {
  return align256b(sizeof(BatchHeader)) + align256b(sizeof(BatchJob<T, S, RT>) * size_t(max_jobs)) +
         align256b(sizeof(BatchUnit) * size_t(max_units));
}

template <class T, class S, class RT, bool WALLS>
__device__ __forceinline__ void batch_march_w(const BatchJob<T, S, RT>& job, const StepArrays<S, RT>& a,
                                              const Segment& sg, unsigned char* smem) {
  const RepParams rp{};
  if (job.lattice == LBM_D3Q19) {
    if (job.model == LBM_MODEL_CG)
      march_segment<D3Q19, T, S, RT, kCG, WALLS, false, int>(a, job.p, nullptr, nullptr, rp, sg, smem);
    else if (job.model == LBM_MODEL_SC_MP)
      march_segment<D3Q19, T, S, RT, kSCMP, WALLS, false, int>(a, job.p, nullptr, nullptr, rp, sg, smem);
    else
      march_segment<D3Q19, T, S, RT, kSC2C, WALLS, false, int>(a, job.p, nullptr, nullptr, rp, sg, smem);
  } else {
    if (job.model == LBM_MODEL_CG)
      march_segment<D2Q9, T, S, RT, kCG, WALLS, false, int>(a, job.p, nullptr, nullptr, rp, sg, smem);
    else if (job.model == LBM_MODEL_SC_MP)
      march_segment<D2Q9, T, S, RT, kSCMP, WALLS, false, int>(a, job.p, nullptr, nullptr, rp, sg, smem);
    else
      march_segment<D2Q9, T, S, RT, kSC2C, WALLS, false, int>(a, job.p, nullptr, nullptr, rp, sg, smem);
  }
}

// ANYWALLS: the job list may hold lattices with walls (the kernel then carries both
// variants of the per-node code; without wall jobs the smaller kernel runs).
template <class T, class S, class RT, bool ANYWALLS>
__device__ __forceinline__ void batch_march(const BatchJob<T, S, RT>& job, const StepArrays<S, RT>& a,
                                            const Segment& sg, unsigned char* smem) {
  if (ANYWALLS && job.walls)
    batch_march_w<T, S, RT, ANYWALLS>(job, a, sg, smem);
  else
    batch_march_w<T, S, RT, false>(job, a, sg, smem);
}

template <class T, class S, class RT, bool ANYWALLS>
__global__ void __launch_bounds__(kBatchTX * kBatchTY, min_blocks<T>())
    batch_step_kernel(const BatchHeader* __restrict__ hdr, const BatchJob<T, S, RT>* __restrict__ jobs,
                      const BatchUnit* __restrict__ units, int s) {
  using Job = BatchJob<T, S, RT>;
  static_assert(sizeof(Job) % 4 == 0, "job descriptors are copied as 32-bit words");
  __shared__ __align__(16) unsigned char job_raw[sizeof(Job)];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Job& job = *reinterpret_cast<const Job*>(job_raw);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nunits = hdr->nunits;
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const BatchUnit un = units[u];
    const uint32_t* src = reinterpret_cast<const uint32_t*>(jobs + un.job);
    for (int w = tid; w < int(sizeof(Job) / 4); w += blockDim.x * blockDim.y)
      reinterpret_cast<uint32_t*>(job_raw)[w] = src[w];
    __syncthreads();
    // the job's status word is written only by the diagnostics kernels, never during this
    // launch, so every thread of the block takes the same branch
    if (s < job.nsteps && *job.status == 0) {
      const int cur = job.cur0 ^ (s & 1);
      Segment sg;
      sg.col = un.col;
      sg.z0 = (int)(((long long)un.chunk * job.p.nz) / job.p.nchunks);
      sg.z1 = (int)(((long long)(un.chunk + 1) * job.p.nz) / job.p.nchunks);
      const StepArrays<S, RT> a{job.f[cur], job.f[cur ^ 1], job.r[cur], job.r[cur ^ 1], job.solid};
      batch_march<T, S, RT, ANYWALLS>(job, a, sg, smem_raw);
    }
    __syncthreads();  // the descriptor slot is rewritten for the next unit
  }
}

// Host side, per storage precision (lbm_batch_{f32,f16,bf16}.cu).
struct BatchOps {
  size_t job_bytes;                                                  // sizeof(BatchJob<...>)
  size_t (*ws_bytes)(int max_jobs, int max_units);
  void (*fill_job)(const lbm_ctx* c, int nsteps, void* dst);         // host descriptor
  // [w]: the kernel for job lists without (w = 0) or with (w = 1) lattices with walls
  size_t (*smem_bytes)(bool walls);                                  // dynamic shared memory
  cudaError_t (*prepare)(bool walls, size_t smem, int* blocks_per_sm);  // opt-in + occupancy
  const void* kernel[2];                                             // batch_step_kernel<...>
};
const BatchOps* batch_ops(int precision);  // nullptr when the precision has no batch kernel

template <class T, class S, class RT>
void batch_fill_job(const lbm_ctx* c, int nsteps, void* dst) {
  BatchJob<T, S, RT> j{};
  j.f[0] = static_cast<S*>(c->f[0]);
  j.f[1] = static_cast<S*>(c->f[1]);
  j.r[0] = static_cast<RT*>(c->r[0]);
  j.r[1] = static_cast<RT*>(c->r[1]);
  j.status = &c->diag->status;
  j.solid = c->has_walls ? c->solid : nullptr;
  j.walls = c->has_walls ? 1 : 0;
  j.lattice = c->p.lattice;
  j.model = c->p.model;
  j.cur0 = c->cur;
  j.nsteps = nsteps;
  j.p = make_step_params<T>(c);
  j.p.ncx = (c->p.nx + kBatchTX - 1) / kBatchTX;
  j.p.ncol = j.p.ncx * ((c->p.ny + kBatchTY - 1) / kBatchTY);
  j.p.nchunks = c->p.lattice == LBM_D3Q19 ? (c->p.nz + batch_chunk(c) - 1) / batch_chunk(c) : 1;
  j.p.nblk = 0;  // unused: the batch's unit list replaces the per-lattice partition
  *static_cast<BatchJob<T, S, RT>*>(dst) = j;
}

template <class T, class S, class RT>
size_t batch_smem_bytes(bool walls) {
  size_t m = 0;
  m = std::max(m, step_smem_bytes<D3Q19, T, kCG, false>(kBatchTX, kBatchTY));
  m = std::max(m, step_smem_bytes<D3Q19, T, kSCMP, false>(kBatchTX, kBatchTY));
  m = std::max(m, step_smem_bytes<D3Q19, T, kSC2C, false>(kBatchTX, kBatchTY));
  m = std::max(m, step_smem_bytes<D2Q9, T, kCG, false>(kBatchTX, kBatchTY));
  m = std::max(m, step_smem_bytes<D2Q9, T, kSCMP, false>(kBatchTX, kBatchTY));
  m = std::max(m, step_smem_bytes<D2Q9, T, kSC2C, false>(kBatchTX, kBatchTY));
  if (walls) {
    m = std::max(m, step_smem_bytes<D3Q19, T, kCG, true>(kBatchTX, kBatchTY));
    m = std::max(m, step_smem_bytes<D3Q19, T, kSCMP, true>(kBatchTX, kBatchTY));
    m = std::max(m, step_smem_bytes<D3Q19, T, kSC2C, true>(kBatchTX, kBatchTY));
    m = std::max(m, step_smem_bytes<D2Q9, T, kCG, true>(kBatchTX, kBatchTY));
    m = std::max(m, step_smem_bytes<D2Q9, T, kSCMP, true>(kBatchTX, kBatchTY));
    m = std::max(m, step_smem_bytes<D2Q9, T, kSC2C, true>(kBatchTX, kBatchTY));
  }
  return m;
}

template <class T, class S, class RT>
cudaError_t batch_prepare(bool walls, size_t smem, int* blocks_per_sm) {
  auto k = walls ? batch_step_kernel<T, S, RT, true> : batch_step_kernel<T, S, RT, false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, kBatchTX * kBatchTY, smem);
}

template <class T, class S, class RT>
const BatchOps* make_batch_ops() {
  static const BatchOps ops = {sizeof(BatchJob<T, S, RT>),
                               &batch_ws_bytes<T, S, RT>,
                               &batch_fill_job<T, S, RT>,
                               &batch_smem_bytes<T, S, RT>,
                               &batch_prepare<T, S, RT>,
                               {reinterpret_cast<const void*>(&batch_step_kernel<T, S, RT, false>),
                                reinterpret_cast<const void*>(&batch_step_kernel<T, S, RT, true>)}};
  return &ops;
}

const BatchOps* batch_ops_f32();
const BatchOps* batch_ops_f16();
const BatchOps* batch_ops_bf16();

}  // namespace lbm
