// D3Q19 step kernel with TMA-staged planes and the x-halo exchanged inside a thread-block
// cluster (16-bit and FP32 storage).
//
// Same step and per-node code as step_kernel_tma (lbm_step_tma.cuh), which fetches the two
// x-halo columns of every plane from global memory: one element per row and population
// array, i.e. as many small requests per plane as the whole interior needs in 128-byte
// rows.  Here a cluster of C = nx / TX blocks covers a full x-row of tiles (the periodic
// wrap in x stays inside the cluster), all blocks of a cluster march the same y-tile and z
// range in step, and no block reads a halo column at all: the stencil fields (densities,
// colour or psi, reference densities) of a block's first and last interior column are
// written by the staging warps straight into the x-neighbours' field slots in distributed
// shared memory (st.shared::cluster), and announced with a remote mbarrier arrival.
//
// Per plane J (slots J % RS raw, J % FS fields; RS = tmac_raw_slots, FS = kClusterFieldSlots)
// the barriers of one block are
//   raw_full  : the producer's tensor copies of the TX interior columns (+ y-halo rows);
//   raw_free  : the staging warps (tmac_stage_warps) and the W = TX*TY/32 collision warps are done
//               with the raw plane;
//   fld_full  : the local staging warps and, from each x-neighbour, the staging warp that
//               wrote its edge column have written their part of the field slot (two
//               remote arrivals; those release at cluster scope, the waits acquire at
//               cluster scope);
//   fld_free  : the W local collision warps are done with the field slot;
//   nbr_free  : the W collision warps of each x-neighbour are done with their field slot
//               (2W arrivals), so that this block may write its edge columns into them.
//               These arrivals are relaxed: they follow the last use of every value read
//               from the slot, and a release at cluster scope would make the collision warp
//               wait for its own outstanding global stores.
// Staging of plane J waits fld_free(J-FS) and nbr_free(J-FS); collision of plane J waits
// fld_full of J-1, J, J+1.  No wait is on an earlier plane's event of the same block than
// the waiter's own, so the pipeline cannot deadlock; every wait is bounded, a timeout sets
// the status word and the thread skips to the final cluster barrier, which every thread
// of every block reaches (a block's shared memory must outlive its neighbours' accesses).
#pragma once

#include "lbm_step_tma.cuh"

namespace lbm {

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// shared::cluster address of the same shared-memory offset in block `rank` of the cluster
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
  uint32_t d;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(addr), "r"(rank));
  return d;
}
__device__ __forceinline__ void st_cluster_f32(uint32_t addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// Relaxed remote arrival: no fence.  Used where the arrival only releases shared-memory
// entries this thread has already read and consumed (a release at cluster scope would
// also wait for the thread's outstanding global stores).
__device__ __forceinline__ void mbar_arrive_remote_relaxed(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_try_wait_cluster_suspend(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}
// As mbar_wait_bounded, with cluster-scope acquire.
__device__ __forceinline__ bool mbar_wait_bounded_cluster(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait_cluster(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (long long it = 0; it < kWaitLimit; ++it) {
    if (mbar_try_wait_cluster_suspend(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::
          : "memory");
}

constexpr int kClusterHeader = 256;  // mbarriers (up to 24 x 8 bytes), 128-byte aligned after it
constexpr int kMaxCluster = 8;       // portable cluster size: nx <= 8 * TX
// Field slots: the collision of plane J reads J-1, J, J+1; the others let the staging run
// ahead by two planes.
constexpr int kClusterFieldSlots = 5;

// Blocks per SM: more where the plane buffers are smaller (one population set, 16-bit
// storage, 32 x 4 tiles); the step is latency bound, so more resident warps pay even with
// a few spilled registers.  With 32 x 4 tiles two blocks of half the size share an SM:
// each cluster's lockstep stalls are then covered by the other cluster's work, which pays
// where clusters are large (nx = 256: C = 8).
template <int MODEL, class S, int TX, int TY>
__host__ __device__ constexpr int tmac_min_blocks() {
  return TX * TY <= 128 ? 2 : ((ModelTraits<MODEL>::K == 1 || sizeof(S) == 2) ? 2 : 1);  // 3 measured no faster
}

// Raw plane buffers: as many as the block's share of shared memory holds, 2 to 6.  The
// copy of plane J+RS-1 can be issued once plane J's collision has loaded its nodes, so
// more buffers hide more of the copy latency.
template <class L, class T, class S, class RT, int MODEL, bool WALLS, int TX, int TY>
__host__ __device__ constexpr int tmac_raw_slots() {
  using Lay = TmaLayout<L, S, RT, MODEL, TX, TY>;
  constexpr int NV = ModelTraits<MODEL>::NF + ModelTraits<MODEL>::K;
  // per-block share of the SM's 228 KB (1 KB of it reserved per block), 227 KB at most
  constexpr size_t budget = tmac_min_blocks<MODEL, S, TX, TY>() == 1 ? 232448 : (233472 / tmac_min_blocks<MODEL, S, TX, TY>() - 1024);
  constexpr size_t fixed = kClusterHeader + kClusterFieldSlots * NV * Lay::NE * sizeof(T) + (WALLS ? kClusterFieldSlots * Lay::NE : 0);
  constexpr size_t n = (budget - fixed) / Lay::BUF_MAIN;
  return n > 6 ? 6 : int(n);
}

// Tensor maps of the tile shape: main columns of one row (halo rows) or of the TY rows.
template <int TX, int TY>
__device__ __forceinline__ const CUtensorMap* tmac_pop_map(const TmaMaps& m, bool mid) {
  if constexpr (TX == 64) return mid ? &m.pop_w_mid4 : &m.pop_w_row;
  return mid ? (TY == 4 ? &m.pop_main_mid4 : &m.pop_main_mid) : &m.pop_main_row;
}
template <int TX, int TY>
__device__ __forceinline__ const CUtensorMap* tmac_ref_map(const TmaMaps& m, bool mid) {
  if constexpr (TX == 64) return mid ? &m.ref_w_mid4 : &m.ref_w_row;
  return mid ? (TY == 4 ? &m.ref_main_mid4 : &m.ref_main_mid) : &m.ref_main_row;
}

template <class L, class T, class S, class RT, int MODEL, bool WALLS, int TX, int TY>
__host__ __device__ constexpr size_t tmac_smem_bytes() {
  using Lay = TmaLayout<L, S, RT, MODEL, TX, TY>;
  constexpr int NV = ModelTraits<MODEL>::NF + ModelTraits<MODEL>::K;
  constexpr int RS = tmac_raw_slots<L, T, S, RT, MODEL, WALLS, TX, TY>();
  return kClusterHeader + RS * Lay::BUF_MAIN + kClusterFieldSlots * NV * Lay::NE * sizeof(T) +
         (WALLS ? kClusterFieldSlots * Lay::NE : 0);
}

// Launch: cluster dims (C, 1, 1) with C = p.ncx = nx / TX; grid = p.nblk clusters * C
// blocks; p.ncol = ny / TY tile rows (the work partition's columns); cluster c takes the
// work units (tile row, z-chunk) c, c + nblk, c + 2 nblk, ... (WorkRange).
// Staging warps: 8 for two population sets (the staging of plane J+1 gates the collision
// of plane J; 6 measured the same, 4 11% slower), 4 where two blocks share an SM.
template <int MODEL, class S, int TX, int TY>
__host__ __device__ constexpr int tmac_stage_warps() { return tmac_min_blocks<MODEL, S, TX, TY>() == 1 ? 8 : 4; }
template <int MODEL, class S, int TX, int TY>
__host__ __device__ constexpr int tmac_threads() { return TX * TY + 32 * (tmac_stage_warps<MODEL, S, TX, TY>() + 1); }

template <class L, class T, class S, class RT, int MODEL, bool WALLS, int TX, int TY>
__global__ void __launch_bounds__(tmac_threads<MODEL, S, TX, TY>(), tmac_min_blocks<MODEL, S, TX, TY>())
    step_kernel_tmac(const __grid_constant__ TmaMaps maps, S* __restrict__ fout, RT* __restrict__ rout,
                     const uint8_t* __restrict__ solid, int* __restrict__ status, StepParams<T> p) {
  constexpr int kCollideWarps = TX * TY / 32;  // one collision thread per tile node
  static_assert(TX * TY % 32 == 0, "whole collision warps");
  static_assert(sizeof(T) == 4, "fields are exchanged as 32-bit words");
  static_assert(2 * (TY + 2) <= 32, "both edge columns fit the first staging warp's first pass");
  using Lay = TmaLayout<L, S, RT, MODEL, TX, TY>;
  constexpr int Q = L::Q, K = Lay::K;
  constexpr int NF = ModelTraits<MODEL>::NF, NV = NF + K;
  constexpr int EX = Lay::EX, NE = Lay::NE;
  constexpr int kRawSlots = tmac_raw_slots<L, T, S, RT, MODEL, WALLS, TX, TY>();
  constexpr int kStageWarps = tmac_stage_warps<MODEL, S, TX, TY>();
  static_assert(kRawSlots >= 2, "at least two raw plane buffers");
  static_assert(2 * kRawSlots + 3 * kClusterFieldSlots <= kClusterHeader / 8, "mbarriers fit the header");
  // A blown-up (or timed-out) state stops stepping.  Blocks of one cluster may read the
  // word at different times, so none returns here: a skipping block still passes both
  // cluster barriers (its neighbours' waits on it then run out and set the status too).
  const bool skip = *status != 0;

  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* raw_full = reinterpret_cast<uint64_t*>(smem);  // [RS]
  uint64_t* raw_free = raw_full + kRawSlots;                // [RS]
  uint64_t* fld_full = raw_free + kRawSlots;                // [kClusterFieldSlots]
  uint64_t* fld_free = fld_full + kClusterFieldSlots;              // [kClusterFieldSlots]
  uint64_t* nbr_free = fld_free + kClusterFieldSlots;              // [kClusterFieldSlots]
  unsigned char* bufs = smem + kClusterHeader;              // [RS][BUF_MAIN]
  T* fld = reinterpret_cast<T*>(bufs + kRawSlots * Lay::BUF_MAIN);        // [kClusterFieldSlots][NV][NE]
  uint8_t* msk = reinterpret_cast<uint8_t*>(fld + kClusterFieldSlots * NV * NE);  // [kClusterFieldSlots][NE]

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const long long N = p.n;
  const int C = p.ncx;
  const uint32_t rank = cluster_ctarank();
  const uint32_t left = (rank + C - 1) % C, right = (rank + 1) % C;
  const int x0 = (int)rank * TX;
  const int cid = blockIdx.x / C;

  if (smem_addr(bufs) & 127u) {  // copy destinations must be 128-byte aligned
    if (tid == 0) atomicOr(status, kStatusLayout);
  }
  if (tid == 0) {
    for (int s = 0; s < kRawSlots; s++) {
      mbar_init(&raw_full[s], 1);
      mbar_init(&raw_free[s], kCollideWarps + kStageWarps);
    }
    for (int s = 0; s < kClusterFieldSlots; s++) {
      mbar_init(&fld_full[s], kStageWarps + 2);  // local staging warps + one per x-neighbour
      mbar_init(&fld_free[s], kCollideWarps);
      mbar_init(&nbr_free[s], 2 * kCollideWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  cluster_sync_all();  // barriers of every block initialised before any remote arrival
  const bool layout_ok = (smem_addr(bufs) & 127u) == 0;

  auto give_up = [&]() { atomicOr(status, kStatusTimeout); };

  if (skip || !layout_ok) {
    // nothing to do; fall through to the final cluster barrier
  } else if (warp == kCollideWarps + kStageWarps) {
    // ---------------- producer ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(&maps.pop_main_mid) : "memory");
      WorkRange work(cid, p.nblk, p.ncol, p.nz, p.nchunks);
      Segment sg;
      int J = 0;
      bool ok = true;
      while (ok && work.pop(sg)) {
        const int y0 = sg.col * TY;
        const int yt = y0 == 0 ? p.ny - 1 : y0 - 1, yb = y0 + TY == p.ny ? 0 : y0 + TY;
        for (int z = sg.z0 - 1; z <= sg.z1; z++, J++) {
          const int s = J % kRawSlots;
          if (J >= kRawSlots && !mbar_wait_bounded(&raw_free[s], ((J / kRawSlots) - 1) & 1)) {
            give_up();
            ok = false;
            break;
          }
          const int gz = wrap(z, p.nz);
          unsigned char* b = bufs + s * Lay::BUF_MAIN;
          uint64_t* bar = &raw_full[s];
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive_expect_tx(bar, Lay::TX_BYTES);
#pragma unroll
          for (int g = 0; g < 3; g++) {
            const bool mid = g == 1;
            const int y = g == 0 ? yt : (g == 1 ? y0 : yb);
            tma_load_4d(b + Lay::PM::group(g), tmac_pop_map<TX, TY>(maps, mid), x0, 0, y, gz, bar);
            tma_load_4d(b + Lay::OFF_RM + Lay::RMR::group(g), tmac_ref_map<TX, TY>(maps, mid), x0, 0,
                        y, gz, bar);
          }
        }
      }
      // wait (bounded) until the copies this block issued have landed
      for (int j = J - kRawSlots; j < J; j++)
        if (j >= 0) mbar_wait_bounded(&raw_full[j % kRawSlots], (j / kRawSlots) & 1);
    }
  } else if (warp >= kCollideWarps) {
    // ---------------- staging ----------------
    const int stid = tid - 32 * kCollideWarps;
    WorkRange work(cid, p.nblk, p.ncol, p.nz, p.nchunks);
    Segment sg;
    int J = 0;
    bool ok = true;
    while (ok && work.pop(sg)) {
      const int y0 = sg.col * TY;
      for (int z = sg.z0 - 1; z <= sg.z1; z++, J++) {
        const int s = J % kRawSlots, fs = J % kClusterFieldSlots;
        ok = mbar_wait_bounded(&raw_full[s], (J / kRawSlots) & 1);
        if (ok && J >= kClusterFieldSlots)
          ok = mbar_wait_bounded(&fld_free[fs], ((J / kClusterFieldSlots) - 1) & 1) &&
               mbar_wait_bounded_cluster(&nbr_free[fs], ((J / kClusterFieldSlots) - 1) & 1);
        ok = __all_sync(0xffffffffu, ok);  // one decision per warp
        if (!ok) {
          give_up();
          break;
        }
        const unsigned char* b = bufs + s * Lay::BUF_MAIN;
        const int gz = wrap(z, p.nz);
        if (WALLS) {
          for (int e = stid; e < NE; e += 32 * kStageWarps) {
            const int ey = e / EX, ex = e - ey * EX;
            const int gxn = wrap(x0 - 1 + ex, p.nx), gyn = wrap(y0 - 1 + ey, p.ny);
            msk[fs * NE + e] = solid[gxn + (long long)p.nx * (gyn + (long long)p.ny * gz)];
          }
        }
        // Interior columns of all EY rows (the halo columns come from the x-neighbours).  The
        // two edge columns go first, to staging warp 0, which writes them into the
        // neighbours' slots early: its release at the end of the plane then finds those
        // remote stores long completed.
        for (int it = stid; it < TX * Lay::EY; it += 32 * kStageWarps) {
          int ex, ey;
          if (it < 2 * Lay::EY) {
            ex = it < Lay::EY ? 1 : TX;
            ey = it < Lay::EY ? it : it - Lay::EY;
          } else {
            const int j = it - 2 * Lay::EY;
            ey = j / (TX - 2);
            ex = 2 + (j - ey * (TX - 2));
          }
          const int e = ey * EX + ex;
          const S* pop = reinterpret_cast<const S*>(b + Lay::PM::row(ey)) + (ex - 1);
          const RT* ref = reinterpret_cast<const RT*>(b + Lay::OFF_RM + Lay::RMR::row(ey)) + (ex - 1);
          T val[NV];
          T rho[2] = {T(0), T(0)};
#pragma unroll
          for (int k = 0; k < K; k++) {
            T g[Q];
#pragma unroll
            for (int i = 0; i < Q; i++) g[i] = ld_s<S, T>(pop[(k * Q + i) * TX]);
            const CompState<T> c = comp_state<L, T, RT>(g, T(ref[k * TX]));
            rho[k] = c.rho;
            val[NF + k] = c.q;
          }
          node_fields<MODEL, T>(p, rho[0], rho[1], val);
#pragma unroll
          for (int f = 0; f < NV; f++) fld[(fs * NV + f) * NE + e] = val[f];
          if (it < 2 * Lay::EY) {
            // edge column: it is the halo column ex' = TX+1 of the left neighbour (ex == 1)
            // or ex' = 0 of the right neighbour (ex == TX)
            const uint32_t peer = ex == 1 ? left : right;
            const int ed = ey * EX + (ex == 1 ? TX + 1 : 0);
#pragma unroll
            for (int f = 0; f < NV; f++)
              st_cluster_f32(mapa_shared(smem_addr(&fld[(fs * NV + f) * NE + ed]), peer), val[f]);
          }
        }
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&fld_full[fs]);  // local readers: CTA-scope release
          if (warp == kCollideWarps) {  // the warp that wrote the neighbours' halo columns
            mbar_arrive_remote(mapa_shared(smem_addr(&fld_full[fs]), left));
            mbar_arrive_remote(mapa_shared(smem_addr(&fld_full[fs]), right));
          }
          mbar_arrive(&raw_free[s]);
        }
      }
    }
  } else {
    // ---------------- collision ----------------
    const int tx = tid % TX, ty = tid / TX;
    const int e0 = (ty + 1) * EX + (tx + 1);
    // 32-bit node indices: the launcher guarantees K * Q * N < 2^31
    const int nxl = p.nx;
    const int plane_n = p.nx * p.ny;
    const int N32 = (int)N;
    const int gx = x0 + tx;
    const int xm = gx == 0 ? p.nx - 1 : gx - 1, xp = gx + 1 >= p.nx ? 0 : gx + 1;
    WorkRange work(cid, p.nblk, p.ncol, p.nz, p.nchunks);
    Segment sg;
    int J = 0;  // global index of the segment's first (halo) plane
    bool ok = true;
    // fields of plane Jf are no longer read here: release the local slot and tell both
    // x-neighbours that their edge columns may be written again
    auto release_fields = [&](int Jf) {
      __syncwarp();
      if (lane == 0) {
        const int fs = Jf % kClusterFieldSlots;
        mbar_arrive(&fld_free[fs]);
        mbar_arrive_remote_relaxed(mapa_shared(smem_addr(&nbr_free[fs]), left));
        mbar_arrive_remote_relaxed(mapa_shared(smem_addr(&nbr_free[fs]), right));
      }
    };
    auto release_raw = [&](int Jr) {  // a plane whose raw data this warp does not read
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(&raw_full[Jr % kRawSlots], (Jr / kRawSlots) & 1)))
        return false;
      if (lane == 0) mbar_arrive(&raw_free[Jr % kRawSlots]);
      return true;
    };
    while (ok && work.pop(sg)) {
      const int y0 = sg.col * TY;
      const int gy = y0 + ty;
      const int ym = gy == 0 ? p.ny - 1 : gy - 1, yp = gy + 1 >= p.ny ? 0 : gy + 1;
      const int rowm = ym * nxl, row0 = gy * nxl, rowp = yp * nxl;
      const int np = sg.z1 - sg.z0 + 2;  // planes z0-1 .. z1
      if (!release_raw(J)) {              // leading halo plane: nothing to collide
        ok = false;
        break;
      }
      for (int c = 1; c <= np - 2 && ok; c++) {
        const int Jc = J + c;
        if (c == 1)
          ok = mbar_wait_bounded_cluster(&fld_full[(Jc - 1) % kClusterFieldSlots], ((Jc - 1) / kClusterFieldSlots) & 1) &&
               mbar_wait_bounded_cluster(&fld_full[Jc % kClusterFieldSlots], (Jc / kClusterFieldSlots) & 1);
        ok = ok && mbar_wait_bounded_cluster(&fld_full[(Jc + 1) % kClusterFieldSlots], ((Jc + 1) / kClusterFieldSlots) & 1);
        ok = ok && mbar_wait_bounded(&raw_full[Jc % kRawSlots], (Jc / kRawSlots) & 1);
        ok = __all_sync(0xffffffffu, ok);  // one decision per warp
        if (!ok) break;
        const int slm = (Jc - 1) % kClusterFieldSlots, sl0 = Jc % kClusterFieldSlots, slp = (Jc + 1) % kClusterFieldSlots;
        const int z = sg.z0 - 1 + c;
        const bool live = !(WALLS && msk[sl0 * NE + e0]);
        T g[K][Q];
        CompState<T> cs[K];
        if (live) {
          const unsigned char* b = bufs + (Jc % kRawSlots) * Lay::BUF_MAIN;
          const S* pop = reinterpret_cast<const S*>(b + Lay::PM::row(ty + 1)) + tx;
          const RT* ref = reinterpret_cast<const RT*>(b + Lay::OFF_RM + Lay::RMR::row(ty + 1)) + tx;
#pragma unroll
          for (int k = 0; k < K; k++) {
#pragma unroll
            for (int i = 0; i < Q; i++) g[k][i] = ld_s<S, T>(pop[(k * Q + i) * TX]);
            cs[k] = comp_state<L, T, RT>(g[k], T(ref[k * TX]));
          }
        }
        // the raw plane is no longer read: hand its buffer back to the producer before the
        // collision arithmetic, so that the next copy is in flight meanwhile
        __syncwarp();
        if (lane == 0) mbar_arrive(&raw_free[Jc % kRawSlots]);
        if (live) {
          auto slot_of = [&](int czv) { return czv == 0 ? sl0 : (czv > 0 ? slp : slm); };
          auto nbr = [&](int fi, int i) -> T {
            const int sl = slot_of(cz<L>(i));
            const int e = e0 + cy<L>(i) * EX + cx<L>(i);
            if (WALLS && msk[sl * NE + e]) return fld[(sl0 * NV + fi) * NE + e0];
            return fld[(sl * NV + fi) * NE + e];
          };
          if constexpr (MODEL == kCG) {
            const T Fx[3] = {T(0), T(0), T(0)};  // the repulsion force runs on the generic kernel
            cg_collide<L, T>(p, g, cs[0], cs[1], nbr, Fx);
          } else if constexpr (MODEL == kSCMP) {
            scmp_collide<L, T>(p, g, cs[0], nbr);
          } else {
            sc2c_collide<L, T>(p, g, cs[0], cs[1], nbr);
          }
          const int zz = z, zm = zz == 0 ? p.nz - 1 : zz - 1, zpp = zz + 1 >= p.nz ? 0 : zz + 1;
          const int pm = zm * plane_n, p0 = zz * plane_n, pp = zpp * plane_n;
          const int n0 = gx + row0 + p0;
#pragma unroll
          for (int k = 0; k < K; k++) rout[k * N32 + n0] = RT(cs[k].q);
#pragma unroll
          for (int i = 0; i < Q; i++) {
            const int dxv = cx<L>(i), dyv = cy<L>(i), dzv = cz<L>(i);
            const int X = dxv == 0 ? gx : (dxv > 0 ? xp : xm);
            const int Y = dyv == 0 ? row0 : (dyv > 0 ? rowp : rowm);
            const int Z = dzv == 0 ? p0 : (dzv > 0 ? pp : pm);
            int nd = X + Y + Z;
            int id = i;
            const int sl = slot_of(dzv);
            const int ed = e0 + dyv * EX + dxv;
            bool bounce = false;
            if (WALLS && i != 0 && msk[sl * NE + ed]) {
              nd = n0;
              id = opp<L>(i);
              bounce = true;
            }
#pragma unroll
            for (int k = 0; k < K; k++) {
              T val = g[k][i];
              if (i != 0 && !bounce) val += p.phi[k][grp<L>(i)] * (cs[k].q - fld[(sl * NV + NF + k) * NE + ed]);
              fout[(k * Q + id) * N32 + nd] = st_s<S, T>(val);
            }
          }
        }
        release_fields(Jc - 1);
      }
      if (!ok) break;
      // segment end: the last interior plane's fields and the trailing halo plane are done
      const int Je = J + np - 1;
      release_fields(Je - 1);
      release_fields(Je);
      if (!release_raw(Je)) {
        ok = false;
        break;
      }
      J += np;
    }
    if (!ok) give_up();
  }
  __syncwarp();
  cluster_sync_all();  // no block leaves while a neighbour may still write to it
}

}  // namespace lbm
