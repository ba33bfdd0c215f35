// D3Q19 step kernel with TMA-staged planes (16-bit and FP32 storage).
//
// Same step as step_kernel (lbm_step.cuh): identical staging sums, collision and push, so
// the two agree to the last few ulps.  What differs is how a plane reaches shared memory.
// One producer warp fetches the extended (TX+2) x (TY+2) plane -- every population array
// and both reference densities -- into a three-deep ring of plane buffers, completing on
// an mbarrier per buffer; plane z+2 is in flight while plane z+1 is reduced to its
// stencil fields and plane z collides.
//
// The TX interior columns of every row come as 4-D tensor copies (cp.async.bulk.tensor)
// of 128-byte rows: a tensor map views a population buffer [k][i][z][y][x] as a tensor
// with dimensions (x, array, y, z), so a box {TX, K*Q, rows, 1} lands in shared memory as
// [rows][array][x].  The two x-halo columns are one element per row and array; as tensor
// boxes they would be 16-byte requests that cost as much copy-engine time as a full row,
// so the producer warp's 32 lanes fetch them instead with 4-byte cp.async copies (the
// aligned 4-byte word holding the element for 16-bit storage), wrapped periodically,
// whose completion is counted on the same mbarrier (cp.async.mbarrier.arrive.noinc).
// The launcher requires nx % TX == 0 and ny % TY == 0.
#pragma once

#include <cuda.h>

#include "lbm_step.cuh"

namespace lbm {

// Tensor maps for one population buffer and its reference field: main-column boxes of
// a single row and of TY rows.
struct TmaMaps {
  CUtensorMap pop_main_row, pop_main_mid, pop_main_mid4;  // 32 columns, rows 1, 8, 4
  CUtensorMap ref_main_row, ref_main_mid, ref_main_mid4;
  CUtensorMap pop_w_row, pop_w_mid4, ref_w_row, ref_w_mid4;  // 64 columns, rows 1, 4 (nx % 64 == 0)
  CUtensorMap pop_main_mid16, ref_main_mid16;                  // 32 columns, 16 rows (ny % 16 == 0)
  CUtensorMap pop_w_mid8, ref_w_mid8;                          // 64 columns, 8 rows (nx % 64 == 0)
  bool mid16, w_mid8;                                          // which of the last two pairs are encoded
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  uint64_t state;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
               : "=l"(state)
               : "r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  (void)state;
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_addr(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
      : "memory");
}

// 4-byte asynchronous copy global -> shared, and an mbarrier arrival once this thread's
// earlier cp.async copies have landed (the arrival is one of the barrier's expected count).
__device__ __forceinline__ void cp_async_4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(__cvta_generic_to_global(src))
               : "memory");
}
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Bounded wait on an mbarrier phase (the copies complete on their own; the bound keeps a
// lost completion from hanging the GPU).  After one plain test, each try_wait carries a
// suspend-time hint, so a waiting warp sleeps until the phase completes (or the hint
// elapses) instead of re-polling: the producer and staging warps of the cluster kernel
// wait for most of each plane, and their polling took issue slots from the collision
// warps (128^3 CG FP32 cluster kernel 183 -> 179 us, 16-bit CG 159 -> 154 us).  The wait
// gives up after kWaitNs of global time or kWaitLimit tries, whichever comes first.
constexpr long long kWaitLimit = 1LL << 22;
constexpr uint32_t kSuspendNs = 20000;
constexpr uint64_t kWaitNs = 2000000000ull;
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (long long it = 0; it < kWaitLimit; ++it) {
    if (mbar_try_wait_suspend(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

constexpr int kStatusTimeout = 0x100;  // diag status bit: a bounded device wait gave up

// Tile of the TMA-staged kernel (compile-time: every shared-memory offset is an immediate).
constexpr int kTmaTX = 32, kTmaTY = 8;

// A tensor copy's shared-memory destination must be 128-byte aligned.  The main-column
// region of a plane buffer (populations, and the same for the reference densities) is
// therefore three slabs -- top halo row, TY interior rows, bottom halo row -- each starting
// on a 128-byte boundary; rows inside the interior slab are contiguous, as the copy writes
// them.
template <int ROW_BYTES, int TY>
struct Region {
  static constexpr size_t al(size_t b) { return (b + 127) & ~size_t(127); }
  static constexpr size_t S1 = al(ROW_BYTES);                  // start of the interior slab
  static constexpr size_t S2 = S1 + al(size_t(TY) * ROW_BYTES);  // start of the bottom slab
  static constexpr size_t BYTES = S2 + al(ROW_BYTES);
  // byte offset of extended row ey (0 .. TY+1)
  __host__ __device__ static constexpr size_t row(int ey) {
    return ey == 0 ? 0 : (ey <= TY ? S1 + size_t(ey - 1) * ROW_BYTES : S2);
  }
  // byte offset where row group g (0 top, 1 interior, 2 bottom) lands
  __host__ __device__ static constexpr size_t group(int g) { return g == 0 ? 0 : (g == 1 ? S1 : S2); }
};

// Plane buffer: population main columns, reference main columns (tensor copies), then
// the x-halo words [side][row][array] of populations and of reference densities.
template <class L, class S, class RT, int MODEL, int TX, int TY>
struct TmaLayout {
  static constexpr int K = ModelTraits<MODEL>::K, Q = L::Q, KQ = K * Q;
  static constexpr int EPW = 4 / int(sizeof(S));    // population elements per 4-byte halo word
  static_assert(sizeof(RT) == 4, "reference densities are 4-byte words here");
  static constexpr int EX = TX + 2, EY = TY + 2, NE = EX * EY, NI = TX * TY;
  using PM = Region<KQ * TX * int(sizeof(S)), TY>;   // population main columns
  using RMR = Region<K * TX * int(sizeof(RT)), TY>;  // reference main columns
  static constexpr size_t OFF_RM = PM::BYTES;        // reference main columns
  static constexpr size_t OFF_H = OFF_RM + RMR::BYTES;  // halo words: [2][EY][KQ + K]
  static constexpr int HW = KQ + K;                  // halo words per side and row
  static constexpr int NH = 2 * EY * HW;             // halo words per plane
  static constexpr size_t BUF = (OFF_H + size_t(NH) * 4 + 127) & ~size_t(127);
  static constexpr size_t BUF_MAIN = OFF_H;          // without the halo words (cluster kernel)
  static_assert(BUF % 128 == 0 && OFF_RM % 128 == 0, "tensor-copy destinations must be 128-byte aligned");
  // bytes the tensor copies of one plane deliver (the alignment padding is not written)
  static constexpr uint32_t TX_BYTES = uint32_t(EY) * (KQ * TX * sizeof(S) + K * TX * sizeof(RT));
};

constexpr int kStatusLayout = 0x200;  // diag status bit: shared-memory base not 128-byte aligned

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  uint64_t state;
  asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(smem_addr(bar)) : "memory");
  (void)state;
}

// Warp roles of the TMA-staged kernel.
constexpr int kCollideWarps = 8;  // one node per thread of the TX x TY = 32 x 8 tile
constexpr int kStageWarps = 4;    // reduce each staged plane to its stencil fields
constexpr int kTmaThreads = 32 * (kCollideWarps + kStageWarps + 1);  // + one producer warp
constexpr int kRawSlots = 3, kFieldSlots = 4;

// Shared memory: [0, 128) the mbarriers; then the raw plane buffers (128-byte aligned);
// then the stencil-field slots; then the wall-mask slots.
template <class L, class T, class S, class RT, int MODEL, bool WALLS, int TX, int TY>
__host__ __device__ constexpr size_t tma_smem_bytes() {
  using Lay = TmaLayout<L, S, RT, MODEL, TX, TY>;
  constexpr int NV = ModelTraits<MODEL>::NF + ModelTraits<MODEL>::K;
  return 128 + kRawSlots * Lay::BUF + kFieldSlots * NV * Lay::NE * sizeof(T) + (WALLS ? kFieldSlots * Lay::NE : 0);
}

// Pipeline.  A block marches the segments of its work range (WorkRange) one after the
// other; a segment [z0, z1) of column col needs the planes z0-1 .. z1 (the first and last
// are halo planes).  All roles walk the same global sequence of planes J = 0, 1, ... over
// the segments, so ring slots (J % 3 raw, J % 4 fields) and mbarrier phases carry on from
// one segment to the next:
//   producer : raw_full[J%3] <- tensor copies of plane J, after raw_free[J%3] reports
//              plane J-3 finished by every consumer warp;
//   staging  : waits raw_full(J), and fld_free(J-4); writes the fields of plane J into
//              slot J%4; arrives fld_full(J) and raw_free(J);
//   collision: for each interior plane waits the fields of J-1, J, J+1 and raw_full(J);
//              loads its node, arrives raw_free(J), collides and pushes, arrives
//              fld_free(J-1).  A halo plane gets raw_free after raw_full (its data is not
//              read); at a segment's end the last two planes' fields are released.
// Every arrival on a ring barrier for plane J comes after that warp has observed
// plane J's copy (raw) or fields (fld) complete, so no arrival can land in the phase of
// plane J-3 (J-4).  No block-wide barrier inside the loop; every wait is bounded and a
// timeout sets the status word, so no thread can hang.
template <class L, class T, class S, class RT, int MODEL, bool WALLS, int TX, int TY>
__global__ void __launch_bounds__(kTmaThreads, 1)
    step_kernel_tma(const __grid_constant__ TmaMaps maps, const S* __restrict__ fin, const RT* __restrict__ rin,
                    S* __restrict__ fout, RT* __restrict__ rout,
                    const uint8_t* __restrict__ solid, int* __restrict__ status, StepParams<T> p) {
  static_assert(TX * TY == 32 * kCollideWarps, "one collision thread per tile node");
  using Lay = TmaLayout<L, S, RT, MODEL, TX, TY>;
  constexpr int Q = L::Q, K = Lay::K, KQ = Lay::KQ, EPW = Lay::EPW, HW = Lay::HW;
  constexpr int NF = ModelTraits<MODEL>::NF, NV = NF + K;
  constexpr int EX = Lay::EX, NE = Lay::NE;
  if (*status != 0) return;  // blown-up (or timed-out) state: stop stepping

  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* raw_full = reinterpret_cast<uint64_t*>(smem);  // [3]
  uint64_t* raw_free = raw_full + kRawSlots;                // [3]
  uint64_t* fld_full = raw_free + kRawSlots;                // [4]
  uint64_t* fld_free = fld_full + kFieldSlots;              // [4]
  unsigned char* bufs = smem + 128;                         // [3][BUF]
  T* fld = reinterpret_cast<T*>(bufs + kRawSlots * Lay::BUF);      // [4][NV][NE]
  uint8_t* msk = reinterpret_cast<uint8_t*>(fld + kFieldSlots * NV * NE);  // [4][NE]

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const long long N = p.n;

  if (smem_addr(bufs) & 127u) {  // copy destinations must be 128-byte aligned
    if (tid == 0) atomicOr(status, kStatusLayout);
    return;
  }
  if (tid == 0) {
    for (int s = 0; s < kRawSlots; s++) {
      mbar_init(&raw_full[s], 1 + 32);  // the producer's expect-tx arrival + one cp.async arrival per lane
      mbar_init(&raw_free[s], kCollideWarps + kStageWarps);
    }
    for (int s = 0; s < kFieldSlots; s++) {
      mbar_init(&fld_full[s], kStageWarps);
      mbar_init(&fld_free[s], kCollideWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();  // the only block-wide barrier: barriers initialised

  auto give_up = [&]() { atomicOr(status, kStatusTimeout); };

  // Ext-node views into a plane buffer: base pointers and strides of the node's arrays.
  struct View {
    const S* pop;
    int ps;
    const RT* ref;
    int rs;
  };
  auto view = [&](const unsigned char* b, int ex, int ey) -> View {
    View v;
    if (ex == 0 || ex == TX + 1) {
      // halo word of side 0 (left, x0-1) or 1 (right, x0+TX); for 16-bit storage the left
      // element is the word's upper half
      const int side = ex == 0 ? 0 : 1;
      const uint32_t* w = reinterpret_cast<const uint32_t*>(b + Lay::OFF_H) + (side * Lay::EY + ey) * HW;
      v.pop = reinterpret_cast<const S*>(w) + (side == 0 ? EPW - 1 : 0);
      v.ps = EPW;
      v.ref = reinterpret_cast<const RT*>(w + KQ);
      v.rs = 1;
    } else {
      v.pop = reinterpret_cast<const S*>(b + Lay::PM::row(ey)) + (ex - 1);
      v.ps = TX;
      v.ref = reinterpret_cast<const RT*>(b + Lay::OFF_RM + Lay::RMR::row(ey)) + (ex - 1);
      v.rs = TX;
    }
    return v;
  };

  if (warp == kCollideWarps + kStageWarps) {
    // ---------------- producer ----------------
    if (lane == 0) asm volatile("prefetch.tensormap [%0];" ::"l"(&maps.pop_main_mid) : "memory");
    WorkRange work(blockIdx.x, p.nblk, p.ncol, p.nz, p.nchunks);
    Segment sg;
    int J = 0;
    bool ok = true;
    const long long plane_n = (long long)p.nx * p.ny;
    while (ok && work.pop(sg)) {
      const int x0 = (sg.col % p.ncx) * TX, y0 = (sg.col / p.ncx) * TY;
      const int yt = y0 == 0 ? p.ny - 1 : y0 - 1, yb = y0 + TY == p.ny ? 0 : y0 + TY;
      // x of the 4-byte halo words: the word holding x0-1 (periodic) and the one at x0+TX;
      // reference densities are one 4-byte element per word
      const int xl = (x0 == 0 ? p.nx : x0) - EPW, xr = x0 + TX == p.nx ? 0 : x0 + TX;
      const int xl_ref = (x0 == 0 ? p.nx : x0) - 1;
      for (int z = sg.z0 - 1; z <= sg.z1; z++, J++) {
        const int s = J % kRawSlots;
        if (J >= kRawSlots &&
            !__all_sync(0xffffffffu, mbar_wait_bounded(&raw_free[s], ((J / kRawSlots) - 1) & 1))) {
          if (lane == 0) give_up();
          ok = false;
          break;
        }
        const int gz = wrap(z, p.nz);
        unsigned char* b = bufs + s * Lay::BUF;
        uint64_t* bar = &raw_full[s];
        if (lane == 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive_expect_tx(bar, Lay::TX_BYTES);
#pragma unroll
          for (int g = 0; g < 3; g++) {
            const bool mid = g == 1;
            const int y = g == 0 ? yt : (g == 1 ? y0 : yb);
            tma_load_4d(b + Lay::PM::group(g), mid ? &maps.pop_main_mid : &maps.pop_main_row, x0, 0, y, gz, bar);
            tma_load_4d(b + Lay::OFF_RM + Lay::RMR::group(g), mid ? &maps.ref_main_mid : &maps.ref_main_row, x0, 0,
                        y, gz, bar);
          }
        }
        // halo words: h = (side * EY + ey) * HW + a, a < KQ a population array, else a
        // reference density
        uint32_t* hw = reinterpret_cast<uint32_t*>(b + Lay::OFF_H);
        const long long zoff = gz * plane_n;
        for (int h = lane; h < Lay::NH; h += 32) {
          const int a = h % HW, r = h / HW;
          const int ey = r % Lay::EY, side = r / Lay::EY;
          const int gy = ey == 0 ? yt : (ey == TY + 1 ? yb : y0 + ey - 1);
          const long long row = zoff + (long long)gy * p.nx;
          const void* src = a < KQ ? static_cast<const void*>(fin + (long long)a * N + row + (side == 0 ? xl : xr))
                                   : static_cast<const void*>(rin + (long long)(a - KQ) * N + row +
                                                              (side == 0 ? xl_ref : xr));
          cp_async_4(hw + h, src);
        }
        cp_async_arrive_noinc(bar);
      }
    }
    // wait (bounded) until the copies this block issued have landed before exiting
    for (int j = J - kRawSlots; j < J; j++)
      if (j >= 0) mbar_wait_bounded(&raw_full[j % kRawSlots], (j / kRawSlots) & 1);
    return;
  }

  if (warp >= kCollideWarps) {
    // ---------------- staging ----------------
    const int stid = tid - 32 * kCollideWarps;
    WorkRange work(blockIdx.x, p.nblk, p.ncol, p.nz, p.nchunks);
    Segment sg;
    int J = 0;
    while (work.pop(sg)) {
      const int x0 = (sg.col % p.ncx) * TX, y0 = (sg.col / p.ncx) * TY;
      for (int z = sg.z0 - 1; z <= sg.z1; z++, J++) {
        const int s = J % kRawSlots, fs = J % kFieldSlots;
        bool ok = mbar_wait_bounded(&raw_full[s], (J / kRawSlots) & 1);
        if (ok && J >= kFieldSlots) ok = mbar_wait_bounded(&fld_free[fs], ((J / kFieldSlots) - 1) & 1);
        ok = __all_sync(0xffffffffu, ok);  // one decision per warp
        if (!ok) {
          give_up();
          return;
        }
        const unsigned char* b = bufs + s * Lay::BUF;
        const int gz = wrap(z, p.nz);
        for (int e = stid; e < NE; e += 32 * kStageWarps) {
          const int ey = e / EX, ex = e - ey * EX;
          const View v = view(b, ex, ey);
          T rho[2] = {T(0), T(0)};
#pragma unroll
          for (int k = 0; k < K; k++) {
            T g[Q];
#pragma unroll
            for (int i = 0; i < Q; i++) g[i] = ld_s<S, T>(v.pop[(k * Q + i) * v.ps]);
            const CompState<T> c = comp_state<L, T, RT>(g, T(v.ref[k * v.rs]));
            rho[k] = c.rho;
            fld[(fs * NV + NF + k) * NE + e] = c.q;
          }
          T out[2];
          node_fields<MODEL, T>(p, rho[0], rho[1], out);
#pragma unroll
          for (int f = 0; f < NF; f++) fld[(fs * NV + f) * NE + e] = out[f];
          if (WALLS) {
            const int gxn = wrap(x0 - 1 + ex, p.nx), gyn = wrap(y0 - 1 + ey, p.ny);
            msk[fs * NE + e] = solid[gxn + (long long)p.nx * (gyn + (long long)p.ny * gz)];
          }
        }
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&fld_full[fs]);
          mbar_arrive(&raw_free[s]);
        }
      }
    }
    return;
  }

  // ---------------- collision ----------------
  const int tx = tid % TX, ty = tid / TX;
  const int e0 = (ty + 1) * EX + (tx + 1);
  const long long nxl = p.nx;
  const long long plane_n = (long long)p.nx * p.ny;
  WorkRange work(blockIdx.x, p.nblk, p.ncol, p.nz, p.nchunks);
  Segment sg;
  int J = 0;  // global index of the segment's first (halo) plane
  auto release_raw = [&](int Jr) {  // a plane whose raw data this warp does not read
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(&raw_full[Jr % kRawSlots], (Jr / kRawSlots) & 1)))
      return false;
    if (lane == 0) mbar_arrive(&raw_free[Jr % kRawSlots]);
    return true;
  };
  while (work.pop(sg)) {
    const int x0 = (sg.col % p.ncx) * TX, y0 = (sg.col / p.ncx) * TY;
    const int gx = x0 + tx, gy = y0 + ty;
    const int xm = gx == 0 ? p.nx - 1 : gx - 1, xp = gx + 1 >= p.nx ? 0 : gx + 1;
    const int ym = gy == 0 ? p.ny - 1 : gy - 1, yp = gy + 1 >= p.ny ? 0 : gy + 1;
    const long long rowm = ym * nxl, row0 = gy * nxl, rowp = yp * nxl;
    const int np = sg.z1 - sg.z0 + 2;  // planes z0-1 .. z1
    if (!release_raw(J)) {              // leading halo plane: nothing to collide
      give_up();
      return;
    }
    for (int c = 1; c <= np - 2; c++) {
      const int Jc = J + c;
      bool ok = true;
      if (c == 1)
        ok = mbar_wait_bounded(&fld_full[(Jc - 1) % kFieldSlots], ((Jc - 1) / kFieldSlots) & 1) &&
             mbar_wait_bounded(&fld_full[Jc % kFieldSlots], (Jc / kFieldSlots) & 1);
      ok = ok && mbar_wait_bounded(&fld_full[(Jc + 1) % kFieldSlots], ((Jc + 1) / kFieldSlots) & 1);
      ok = ok && mbar_wait_bounded(&raw_full[Jc % kRawSlots], (Jc / kRawSlots) & 1);
      ok = __all_sync(0xffffffffu, ok);  // one decision per warp
      if (!ok) {
        give_up();
        return;
      }
      const int slm = (Jc - 1) % kFieldSlots, sl0 = Jc % kFieldSlots, slp = (Jc + 1) % kFieldSlots;
      const int z = sg.z0 - 1 + c;
      const bool live = !(WALLS && msk[sl0 * NE + e0]);
      T g[K][Q];
      CompState<T> cs[K];
      if (live) {
        const View v = view(bufs + (Jc % kRawSlots) * Lay::BUF, tx + 1, ty + 1);
#pragma unroll
        for (int k = 0; k < K; k++) {
#pragma unroll
          for (int i = 0; i < Q; i++) g[k][i] = ld_s<S, T>(v.pop[(k * Q + i) * TX]);
          cs[k] = comp_state<L, T, RT>(g[k], T(v.ref[k * TX]));
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
        const long long pm = zm * plane_n, p0 = zz * plane_n, pp = zpp * plane_n;
        const long long n0 = gx + row0 + p0;
#pragma unroll
        for (int k = 0; k < K; k++) rout[(long long)k * N + n0] = RT(cs[k].q);
#pragma unroll
        for (int i = 0; i < Q; i++) {
          const int dxv = cx<L>(i), dyv = cy<L>(i), dzv = cz<L>(i);
          const long long X = dxv == 0 ? gx : (dxv > 0 ? xp : xm);
          const long long Y = dyv == 0 ? row0 : (dyv > 0 ? rowp : rowm);
          const long long Z = dzv == 0 ? p0 : (dzv > 0 ? pp : pm);
          long long nd = X + Y + Z;
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
            fout[(long long)(k * Q + id) * N + nd] = st_s<S, T>(val);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&fld_free[(Jc - 1) % kFieldSlots]);
    }
    // segment end: the last interior plane's fields and the trailing halo plane are done
    const int Je = J + np - 1;
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&fld_free[(Je - 1) % kFieldSlots]);
      mbar_arrive(&fld_free[Je % kFieldSlots]);
    }
    if (!release_raw(Je)) {
      give_up();
      return;
    }
    J += np;
  }
}

}  // namespace lbm
