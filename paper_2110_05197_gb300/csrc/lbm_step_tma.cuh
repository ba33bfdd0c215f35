// D3Q19 step kernel with TMA-staged planes (16-bit and FP32 storage).
//
// Same step as step_kernel (lbm_step.cuh): identical staging sums, collision and push, so
// the two give bitwise identical results.  What differs is how a plane reaches shared
// memory.  One thread issues 4-D tensor copies (cp.async.bulk.tensor) of the extended
// (TX+2) x (TY+2) plane -- every population array and both reference densities -- into
// a three-deep ring of plane buffers, completing on an mbarrier per buffer; plane z+2 is
// in flight while plane z+1 is reduced to its stencil fields and plane z collides.  No
// thread computes a global load address for staging, and the copy latency is off the
// critical path.
//
// Tensor maps view a population buffer [k][i][z][y][x] as a 4-D tensor with dimensions
// (x, array, y, z), so a box {TX, K*Q, rows, 1} lands in shared memory as
// [rows][array][x]: row groups (top halo row, TY interior rows, bottom halo row) stack in
// y.  The x halo columns come as 16-byte strips at x0-SW and x0+TX, wrapped to the far side
// of the periodic box by choosing the strip's start coordinate; every coordinate is in
// range and 16-byte aligned (the launcher requires nx % TX == 0 and ny % TY == 0).
#pragma once

#include <cuda.h>

#include "lbm_step.cuh"

namespace lbm {

// Tensor maps for one population buffer and its reference field: main-x boxes and
// x-strip boxes, each for a single row and for TY rows.
struct TmaMaps {
  CUtensorMap pop_main_row, pop_main_mid, pop_strip_row, pop_strip_mid;
  CUtensorMap ref_main_row, ref_main_mid, ref_strip_row, ref_strip_mid;
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

// Bounded wait on an mbarrier phase (the copies complete on their own; the bound keeps a
// lost completion from hanging the GPU).
constexpr long long kWaitLimit = 1LL << 22;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

constexpr int kStatusTimeout = 0x100;  // diag status bit: a bounded device wait gave up

// Tile of the TMA-staged kernel (compile-time: every shared-memory offset is an immediate).
constexpr int kTmaTX = 32, kTmaTY = 8;

// A tensor copy's shared-memory destination must be 128-byte aligned.  Each region of a
// plane buffer (population main columns, left/right strips, and the same for the
// reference densities) is therefore three slabs -- top halo row, TY interior rows, bottom
// halo row -- each starting on a 128-byte boundary; rows inside the interior slab are
// contiguous, as the copy writes them.
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

template <class L, class S, class RT, int MODEL, int TX, int TY>
struct TmaLayout {
  static constexpr int K = ModelTraits<MODEL>::K, Q = L::Q, KQ = K * Q;
  static constexpr int SW = 16 / int(sizeof(S));    // strip width (elements) of populations
  static constexpr int RSW = 16 / int(sizeof(RT));  // strip width of reference densities
  static constexpr int EX = TX + 2, EY = TY + 2, NE = EX * EY, NI = TX * TY;
  using PM = Region<KQ * TX * int(sizeof(S)), TY>;   // population main columns
  using PS = Region<KQ * SW * int(sizeof(S)), TY>;   // population strip (one side)
  using RMR = Region<K * TX * int(sizeof(RT)), TY>;  // reference main columns
  using RSR = Region<K * RSW * int(sizeof(RT)), TY>; // reference strip (one side)
  static constexpr size_t OFF_L = PM::BYTES, OFF_R = OFF_L + PS::BYTES, OFF_RM = OFF_R + PS::BYTES,
                          OFF_RL = OFF_RM + RMR::BYTES, OFF_RR = OFF_RL + RSR::BYTES;
  static constexpr size_t BUF = OFF_RR + RSR::BYTES;
  static_assert(BUF % 128 == 0 && OFF_L % 128 == 0 && OFF_R % 128 == 0 && OFF_RM % 128 == 0 &&
                    OFF_RL % 128 == 0 && OFF_RR % 128 == 0,
                "tensor-copy destinations must be 128-byte aligned");
  // bytes the copies of one plane deliver (the alignment padding is not written)
  static constexpr uint32_t TX_BYTES =
      uint32_t(EY) * (KQ * (TX + 2 * SW) * sizeof(S) + K * (TX + 2 * RSW) * sizeof(RT));
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

// Pipeline over the planes j = 0 .. n-1 of a block's z-chunk (plane z = z0 - 1 + j; j = 0
// and j = n-1 are the halo planes):
//   producer : raw_full[j%3] <- tensor copies of plane j, after raw_free[j%3] reports
//              plane j-3 finished (staging and collision);
//   staging  : waits raw_full, and fld_free[j%4] for plane j-4's fields; writes the fields of
//              plane j into slot j%4; arrives fld_full[j%4] and raw_free[j%3];
//   collision: for planes c = 1 .. n-2 waits fld_full of c+1 (c-1, c were waited earlier)
//              and raw_full of c; collides and pushes; arrives raw_free[c%3] and
//              fld_free[(c-1)%4] (the last use of plane c-1's fields).
// No block-wide barrier inside the loop; every wait is bounded and a timeout sets the
// status word, so no thread can hang.
template <class L, class T, class S, class RT, int MODEL, bool WALLS, int TX, int TY>
__global__ void __launch_bounds__(kTmaThreads, 1)
    step_kernel_tma(const __grid_constant__ TmaMaps maps, S* __restrict__ fout, RT* __restrict__ rout,
                    const uint8_t* __restrict__ solid, int* __restrict__ status, StepParams<T> p) {
  static_assert(TX * TY == 32 * kCollideWarps, "one collision thread per tile node");
  using Lay = TmaLayout<L, S, RT, MODEL, TX, TY>;
  constexpr int Q = L::Q, K = Lay::K, KQ = Lay::KQ, SW = Lay::SW, RSW = Lay::RSW;
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
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = (int)(((long long)blockIdx.z * p.nz) / p.nchunks);
  const int z1 = (int)(((long long)(blockIdx.z + 1) * p.nz) / p.nchunks);
  const int np = z1 - z0 + 2;  // planes z0-1 .. z1
  const long long N = p.n;

  if (smem_addr(bufs) & 127u) {  // copy destinations must be 128-byte aligned
    if (tid == 0) atomicOr(status, kStatusLayout);
    return;
  }
  if (tid == 0) {
    for (int s = 0; s < kRawSlots; s++) {
      mbar_init(&raw_full[s], 1);
      mbar_init(&raw_free[s], kCollideWarps + kStageWarps);
    }
    for (int s = 0; s < kFieldSlots; s++) {
      mbar_init(&fld_full[s], kStageWarps);
      mbar_init(&fld_free[s], kCollideWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();  // the only block-wide barrier: barriers initialised

  auto plane_z = [&](int j) { return wrap(z0 - 1 + j, p.nz); };
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
    if (ex == 0) {
      v.pop = reinterpret_cast<const S*>(b + Lay::OFF_L + Lay::PS::row(ey)) + (SW - 1);
      v.ps = SW;
      v.ref = reinterpret_cast<const RT*>(b + Lay::OFF_RL + Lay::RSR::row(ey)) + (RSW - 1);
      v.rs = RSW;
    } else if (ex == TX + 1) {
      v.pop = reinterpret_cast<const S*>(b + Lay::OFF_R + Lay::PS::row(ey));
      v.ps = SW;
      v.ref = reinterpret_cast<const RT*>(b + Lay::OFF_RR + Lay::RSR::row(ey));
      v.rs = RSW;
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
    if (lane != 0) return;
    asm volatile("prefetch.tensormap [%0];" ::"l"(&maps.pop_main_mid) : "memory");
    const int yt = y0 == 0 ? p.ny - 1 : y0 - 1, yb = y0 + TY == p.ny ? 0 : y0 + TY;
    const int xl = x0 == 0 ? p.nx - SW : x0 - SW, xr = x0 + TX == p.nx ? 0 : x0 + TX;
    const int xlr = x0 == 0 ? p.nx - RSW : x0 - RSW, xrr = x0 + TX == p.nx ? 0 : x0 + TX;
    int issued = 0;
    for (int j = 0; j < np; j++) {
      const int s = j % kRawSlots;
      if (j >= kRawSlots && !mbar_wait_bounded(&raw_free[s], ((j / kRawSlots) - 1) & 1)) {
        give_up();
        break;
      }
      const int gz = plane_z(j);
      unsigned char* b = bufs + s * Lay::BUF;
      uint64_t* bar = &raw_full[s];
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive_expect_tx(bar, Lay::TX_BYTES);
#pragma unroll
      for (int g = 0; g < 3; g++) {
        const bool mid = g == 1;
        const int y = g == 0 ? yt : (g == 1 ? y0 : yb);
        tma_load_4d(b + Lay::PM::group(g), mid ? &maps.pop_main_mid : &maps.pop_main_row, x0, 0, y, gz, bar);
        tma_load_4d(b + Lay::OFF_L + Lay::PS::group(g), mid ? &maps.pop_strip_mid : &maps.pop_strip_row, xl, 0, y,
                    gz, bar);
        tma_load_4d(b + Lay::OFF_R + Lay::PS::group(g), mid ? &maps.pop_strip_mid : &maps.pop_strip_row, xr, 0, y,
                    gz, bar);
        tma_load_4d(b + Lay::OFF_RM + Lay::RMR::group(g), mid ? &maps.ref_main_mid : &maps.ref_main_row, x0, 0, y,
                    gz, bar);
        tma_load_4d(b + Lay::OFF_RL + Lay::RSR::group(g), mid ? &maps.ref_strip_mid : &maps.ref_strip_row, xlr, 0,
                    y, gz, bar);
        tma_load_4d(b + Lay::OFF_RR + Lay::RSR::group(g), mid ? &maps.ref_strip_mid : &maps.ref_strip_row, xrr, 0,
                    y, gz, bar);
      }
      issued = j + 1;
    }
    // wait (bounded) until the copies this block issued have landed before exiting
    for (int j = issued - kRawSlots; j < issued; j++)
      if (j >= 0) mbar_wait_bounded(&raw_full[j % kRawSlots], (j / kRawSlots) & 1);
    return;
  }

  if (warp >= kCollideWarps) {
    // ---------------- staging ----------------
    const int stid = tid - 32 * kCollideWarps;
    for (int j = 0; j < np; j++) {
      const int s = j % kRawSlots, fs = j % kFieldSlots;
      bool ok = mbar_wait_bounded(&raw_full[s], (j / kRawSlots) & 1);
      if (ok && j >= kFieldSlots) ok = mbar_wait_bounded(&fld_free[fs], ((j / kFieldSlots) - 1) & 1);
      if (!ok) {
        give_up();
        return;
      }
      const unsigned char* b = bufs + s * Lay::BUF;
      const int gz = plane_z(j);
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
    return;
  }

  // ---------------- collision ----------------
  const int tx = tid % TX, ty = tid / TX;
  const int gx = x0 + tx, gy = y0 + ty;
  const int e0 = (ty + 1) * EX + (tx + 1);
  const int xm = gx == 0 ? p.nx - 1 : gx - 1, xp = gx + 1 >= p.nx ? 0 : gx + 1;
  const int ym = gy == 0 ? p.ny - 1 : gy - 1, yp = gy + 1 >= p.ny ? 0 : gy + 1;
  const long long nxl = p.nx;
  const long long plane_n = (long long)p.nx * p.ny;
  const long long rowm = ym * nxl, row0 = gy * nxl, rowp = yp * nxl;
  if (lane == 0) mbar_arrive(&raw_free[0]);  // plane 0 is a halo plane: nothing to collide

  for (int c = 1; c <= np - 2; c++) {
    bool ok = true;
    if (c == 1) {
      ok = mbar_wait_bounded(&fld_full[0], 0) && mbar_wait_bounded(&fld_full[1], 0);
    }
    ok = ok && mbar_wait_bounded(&fld_full[(c + 1) % kFieldSlots], ((c + 1) / kFieldSlots) & 1);
    ok = ok && mbar_wait_bounded(&raw_full[c % kRawSlots], (c / kRawSlots) & 1);
    if (!ok) {
      give_up();
      return;
    }
    const int slm = (c - 1) % kFieldSlots, sl0 = c % kFieldSlots, slp = (c + 1) % kFieldSlots;
    const int z = z0 - 1 + c;
    const bool live = !(WALLS && msk[sl0 * NE + e0]);
    if (live) {
      const View v = view(bufs + (c % kRawSlots) * Lay::BUF, tx + 1, ty + 1);
      T g[K][Q];
      CompState<T> cs[K];
#pragma unroll
      for (int k = 0; k < K; k++) {
#pragma unroll
        for (int i = 0; i < Q; i++) g[k][i] = ld_s<S, T>(v.pop[(k * Q + i) * TX]);
        cs[k] = comp_state<L, T, RT>(g[k], T(v.ref[k * TX]));
      }
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
      const int zz = wrap(z, p.nz), zm = zz == 0 ? p.nz - 1 : zz - 1, zpp = zz + 1 >= p.nz ? 0 : zz + 1;
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
    if (lane == 0) {
      mbar_arrive(&raw_free[c % kRawSlots]);
      mbar_arrive(&fld_free[(c - 1) % kFieldSlots]);
    }
  }
}

}  // namespace lbm
