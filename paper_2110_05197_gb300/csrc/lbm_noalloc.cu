// Allocation-free totals reduction (lbm_totals_noalloc in include/lbm.h).
//
// Some callers cannot call cudaMalloc: a plugin inside a host application whose caching
// allocator has reserved the device memory (a cudaMalloc beside it fails or fragments the
// pool the host accounts for), or a latency-bound monitoring loop that must never enter
// the driver's allocation path.  They can still own the populations they hand in and the
// totals they read back.  For them this entry point computes the same FP64 totals as
// lbm_moments from caller-owned canonical populations, and keeps its scratch -- the
// per-node densities the force stencil needs, the per-block partial sums and the result
// record -- in one file-scope __device__ array of fixed size instead of a workspace.
//
// The array exists once per device for the life of the process.  Every call shares it
// and it keeps the previous call's contents; calls whose work overlaps on the GPU (two
// streams, or two host threads) race on it and must be serialised by the caller.
#include <algorithm>
#include <mutex>

#include "lbm_internal.cuh"

namespace {

constexpr long long kMaxNodes = 1LL << 20;        // 16 MiB of FP64 densities (2 per node)
constexpr int kBlocks = 1184;                      // partial sums: 1184 x LBM_NTOTALS doubles
constexpr int kThreads = 256;
constexpr size_t kDensBytes = size_t(kMaxNodes) * 2 * sizeof(double);
constexpr size_t kPartBytes = size_t(kBlocks) * LBM_NTOTALS * sizeof(double);
constexpr size_t kScratchBytes = kDensBytes + kPartBytes + 256;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct Record {
  double totals[LBM_NTOTALS];
  int status;
};
static_assert(sizeof(Record) <= 256, "record slot");

struct TotParams {
  int nx, ny, nz, lattice, model, K;
  long long n;
  double G, rho0, body[3], umax, neg_tol;
};

__device__ __forceinline__ long long wrapped(int x, int y, int z, const TotParams& a) {
  x = x < 0 ? x + a.nx : (x >= a.nx ? x - a.nx : x);
  y = y < 0 ? y + a.ny : (y >= a.ny ? y - a.ny : y);
  z = z < 0 ? z + a.nz : (z >= a.nz ? z - a.nz : z);
  return x + (long long)a.nx * (y + (long long)a.ny * z);
}

template <class L>
__global__ void dens_kernel(const double* __restrict__ f, double* __restrict__ rr, double* __restrict__ rb,
                            TotParams a) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < a.n; m += (long long)gridDim.x * blockDim.x) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = 0; i < L::Q; i++) s0 += f[(long long)i * a.n + m];
    if (a.K == 2)
      for (int i = 0; i < L::Q; i++) s1 += f[(long long)(L::Q + i) * a.n + m];
    rr[m] = s0;
    rb[m] = s1;
  }
}

// slots: 0 mass_r 1 mass_b 2-4 momentum 5 E_kin 6 max|u| 7 non-finite 8 min rho_r 9 min rho_b
__device__ __forceinline__ void merge(double* a, const double* b) {
  for (int s = 0; s < 6; s++) a[s] += b[s];
  a[6] = fmax(a[6], b[6]);
  a[7] += b[7];
  a[8] = fmin(a[8], b[8]);
  a[9] = fmin(a[9], b[9]);
}

__device__ void reduce_block(double* v) {
  __shared__ double sh[kThreads / 32][LBM_NTOTALS];
  for (int off = 16; off > 0; off >>= 1) {
    double o[LBM_NTOTALS];
    for (int s = 0; s < LBM_NTOTALS; s++) o[s] = __shfl_xor_sync(0xffffffffu, v[s], off);
    merge(v, o);
  }
  if ((threadIdx.x & 31) == 0)
    for (int s = 0; s < LBM_NTOTALS; s++) sh[threadIdx.x >> 5][s] = v[s];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) merge(v, sh[w]);
}

template <class L>
__global__ void __launch_bounds__(kThreads) part_kernel(const double* __restrict__ f, const double* __restrict__ rr,
                                                        const double* __restrict__ rb,
                                                        const uint8_t* __restrict__ solid,
                                                        double* __restrict__ partials, TotParams a) {
  using namespace lbm;
  double acc[LBM_NTOTALS] = {0, 0, 0, 0, 0, 0, 0, 0, INFINITY, INFINITY};
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < a.n; n += (long long)gridDim.x * blockDim.x) {
    if (solid && solid[n]) continue;
    // momentum as opposite-pair differences f_i - f_opp(i), as lbm_moments sums it: the
    // symmetric (rest-state) part of each pair cancels exactly before it is accumulated
    double j[3] = {0.0, 0.0, 0.0};
    int bad = 0;
    for (int k = 0; k < a.K; k++) {
      if (!isfinite(f[(long long)(k * L::Q) * a.n + n])) bad = 1;
      for (int q = 0; q < L::NP; q++) {
        const double vp = f[(long long)(k * L::Q + 2 * q + 1) * a.n + n];
        const double vm = f[(long long)(k * L::Q + 2 * q + 2) * a.n + n];
        if (!isfinite(vp) || !isfinite(vm)) bad = 1;
        const double d = vp - vm;
        j[0] += L::pcx(q) * d;
        j[1] += L::pcy(q) * d;
        j[2] += L::pcz(q) * d;
      }
    }
    const double r = rr[n], b = rb[n], rho = r + b;
    double F[3] = {a.body[0], a.body[1], a.body[2]};
    if (a.model != LBM_MODEL_CG) {
      // SC force: Eq. interactionforceMP (psi of Eq. pseudopotential) or the cross force of
      // Eq. doublebeltrepulsionforce2; a wall neighbour takes the centre value
      int x, y, z;
      node_coords(n, a.nx, a.ny, a.n, x, y, z);
      const double psic = a.rho0 * (1.0 - exp(-r / a.rho0));
      double s1[3] = {0.0, 0.0, 0.0}, s2[3] = {0.0, 0.0, 0.0};
      for (int i = 1; i < L::Q; i++) {
        const long long m = wrapped(x + cx<L>(i), y + cy<L>(i), z + cz<L>(i), a);
        const bool sw = solid && solid[m];
        const double w = L::w(grp<L>(i));
        const double v1 = a.model == LBM_MODEL_SC_MP ? (sw ? psic : a.rho0 * (1.0 - exp(-rr[m] / a.rho0)))
                                                     : (sw ? b : rb[m]);
        const double v2 = sw ? r : rr[m];
        s1[0] += w * v1 * cx<L>(i);
        s1[1] += w * v1 * cy<L>(i);
        s1[2] += w * v1 * cz<L>(i);
        s2[0] += w * v2 * cx<L>(i);
        s2[1] += w * v2 * cy<L>(i);
        s2[2] += w * v2 * cz<L>(i);
      }
      for (int d = 0; d < 3; d++)
        F[d] = a.model == LBM_MODEL_SC_MP ? -a.G * psic * s1[d] + a.body[d]
                                          : -a.G * r * s1[d] - a.G * b * s2[d] + a.body[d];
    }
    double u[3];
    for (int d = 0; d < 3; d++) u[d] = (j[d] + 0.5 * F[d]) / rho;
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    acc[0] += r;
    acc[1] += b;
    acc[2] += j[0];
    acc[3] += j[1];
    acc[4] += j[2];
    acc[5] += 0.5 * rho * uu;
    acc[6] = fmax(acc[6], sqrt(uu));
    acc[7] += bad;
    acc[8] = fmin(acc[8], r);
    acc[9] = fmin(acc[9], b);
  }
  reduce_block(acc);
  if (threadIdx.x == 0)
    for (int s = 0; s < LBM_NTOTALS; s++) partials[blockIdx.x * LBM_NTOTALS + s] = acc[s];
}

__global__ void __launch_bounds__(kThreads) final_kernel(const double* __restrict__ partials, int nblk,
                                                         Record* __restrict__ rec, TotParams a) {
  double acc[LBM_NTOTALS] = {0, 0, 0, 0, 0, 0, 0, 0, INFINITY, INFINITY};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) merge(acc, partials + b * LBM_NTOTALS);
  reduce_block(acc);
  if (threadIdx.x == 0) {
    int st = 0;
    if (acc[7] > 0 || !isfinite(acc[0]) || !isfinite(acc[1])) st |= 1;
    if (acc[8] < -a.neg_tol || acc[9] < -a.neg_tol) st |= 2;
    if (!(acc[6] <= a.umax)) st |= 4;
    for (int s = 0; s < LBM_NTOTALS; s++) rec->totals[s] = acc[s];
    rec->status = st;  // written whole on every call: nothing carries over
  }
}

// Device address of g_scratch, looked up once per device (with that device current).
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

cudaError_t scratch_on_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// True for managed memory and for device memory of device `dev` (the current device, on
// which the kernels run); a device pointer of another GPU would be read without peer
// access, so it is refused like a host pointer.
bool is_device(const void* ptr, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" lbm_status lbm_totals_noalloc(const lbm_params* p, const double* pops, const uint8_t* solid,
                                         double* totals, void* stream) {
  if (!p || !pops || !totals) return LBM_EINVAL;
  if (p->lattice != LBM_D2Q9 && p->lattice != LBM_D3Q19) return LBM_EINVAL;
  if (p->model < LBM_MODEL_CG || p->model > LBM_MODEL_SC_2C) return LBM_EINVAL;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || (p->lattice == LBM_D2Q9 && p->nz != 1)) return LBM_EINVAL;
  const long long n = (long long)p->nx * p->ny * p->nz;
  if (n > kMaxNodes) return LBM_EINVAL;  // beyond the fixed scratch (LBM_NOALLOC_MAX_NODES)
  if (p->model != LBM_MODEL_CG && !(p->rho0_psi > 0)) return LBM_EINVAL;
  // the CG repulsion force (Sec. 2.3) enters u and E_kin; this entry point does not
  // compute it, so such a state is refused rather than given different totals
  if (p->model == LBM_MODEL_CG && p->rep_pi != 0.0) return LBM_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ECUDA;
  if (!is_device(pops, dev) || (solid && !is_device(solid, dev))) return LBM_EINVAL;
  const bool dev_totals = is_device(totals, dev);

  unsigned char* base = nullptr;
  cudaError_t e = scratch_on_current_device(&base);
  if (e != cudaSuccess) return LBM_ECUDA;
  double* rr = reinterpret_cast<double*>(base);
  double* rb = rr + n;
  double* partials = reinterpret_cast<double*>(base + kDensBytes);
  Record* rec = reinterpret_cast<Record*>(base + kDensBytes + kPartBytes);

  TotParams a{};
  a.nx = p->nx;
  a.ny = p->ny;
  a.nz = p->nz;
  a.lattice = p->lattice;
  a.model = p->model;
  a.K = p->model == LBM_MODEL_SC_MP ? 1 : 2;
  a.n = n;
  a.G = p->model == LBM_MODEL_SC_2C ? p->G / (p->rho0_psi * p->rho0_psi) : p->G;
  a.rho0 = p->rho0_psi;
  for (int d = 0; d < 3; d++) a.body[d] = p->body_force[d];
  a.umax = p->umax_unstable > 0 ? p->umax_unstable : 0.5;
  a.neg_tol = lbm::kNegDensityTol * (p->model == LBM_MODEL_CG ? fmax(1.0, fmax(p->rho_r0, p->rho_b0)) : 1.0);

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int g1 = (int)std::min<long long>((n + kThreads - 1) / kThreads, 8192);
  const int g2 = (int)std::min<long long>((n + kThreads - 1) / kThreads, kBlocks);
  if (p->lattice == LBM_D3Q19) {
    dens_kernel<lbm::D3Q19><<<g1, kThreads, 0, s>>>(pops, rr, rb, a);
    part_kernel<lbm::D3Q19><<<g2, kThreads, 0, s>>>(pops, rr, rb, solid, partials, a);
  } else {
    dens_kernel<lbm::D2Q9><<<g1, kThreads, 0, s>>>(pops, rr, rb, a);
    part_kernel<lbm::D2Q9><<<g2, kThreads, 0, s>>>(pops, rr, rb, solid, partials, a);
  }
  final_kernel<<<1, kThreads, 0, s>>>(partials, g2, rec, a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return LBM_ECUDA;
  Record host;
  if (dev_totals) {
    e = cudaMemcpyAsync(totals, rec->totals, sizeof(host.totals), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host.status, &rec->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  } else {
    e = cudaMemcpyAsync(&host, rec, sizeof(Record), cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return LBM_ECUDA;
  if (!dev_totals)
    for (int k = 0; k < LBM_NTOTALS; k++) totals[k] = host.totals[k];
  return host.status ? LBM_EUNSTABLE : LBM_OK;
}
