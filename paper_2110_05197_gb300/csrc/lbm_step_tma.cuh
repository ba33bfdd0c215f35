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

// Shared memory: [0, 128) the three mbarriers; then three plane buffers (128-byte
// aligned); then the rotating stencil-field planes; then the wall masks.
template <class L, class T, class S, class RT, int MODEL, bool WALLS, int TX, int TY>
__host__ __device__ constexpr size_t tma_smem_bytes() {
  using Lay = TmaLayout<L, S, RT, MODEL, TX, TY>;
  constexpr int NV = ModelTraits<MODEL>::NF + ModelTraits<MODEL>::K;
  return 128 + 3 * Lay::BUF + 3 * NV * Lay::NE * sizeof(T) + (WALLS ? 3 * Lay::NE : 0);
}

template <class L, class T, class S, class RT, int MODEL, bool WALLS, int TX, int TY>
__global__ void __launch_bounds__(TX* TY, 1)
    step_kernel_tma(const __grid_constant__ TmaMaps maps, S* __restrict__ fout, RT* __restrict__ rout,
                    const uint8_t* __restrict__ solid, int* __restrict__ status, StepParams<T> p) {
  using Lay = TmaLayout<L, S, RT, MODEL, TX, TY>;
  constexpr int Q = L::Q, K = Lay::K, KQ = Lay::KQ, SW = Lay::SW, RSW = Lay::RSW;
  constexpr int NF = ModelTraits<MODEL>::NF, NV = NF + K;
  constexpr int EX = Lay::EX, NE = Lay::NE, NI = Lay::NI;
  if (*status != 0) return;  // blown-up (or timed-out) state: stop stepping

  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);           // [3]
  unsigned char* bufs = smem + 128;                              // [3][BUF]
  T* fld = reinterpret_cast<T*>(bufs + 3 * Lay::BUF);           // [3][NV][NE]
  uint8_t* msk = reinterpret_cast<uint8_t*>(fld + 3 * NV * NE);  // [3][NE]

  const int tid = threadIdx.y * TX + threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * p.tz;
  const int z1 = min(z0 + p.tz, p.nz);
  const long long N = p.n;

  // the plane buffers start 128 bytes into dynamic shared memory; refuse to issue any copy
  // if the base is not 128-byte aligned (uniform over the block)
  if (smem_addr(bufs) & 127u) {
    if (tid == 0) atomicOr(status, kStatusLayout);
    return;
  }
  if (tid == 0) {
    for (int b = 0; b < 3; b++) mbar_init(&bars[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&maps.pop_main_mid) : "memory");
  }
  __syncthreads();

  // plane p -> ring slot (buffers and field planes rotate together)
  auto slot = [&](int pl) { return (pl - z0 + 1) % 3; };
  const int yt = y0 == 0 ? p.ny - 1 : y0 - 1, yb = y0 + TY == p.ny ? 0 : y0 + TY;
  const int xl = x0 == 0 ? p.nx - SW : x0 - SW, xr = x0 + TX == p.nx ? 0 : x0 + TX;
  const int xlr = x0 == 0 ? p.nx - RSW : x0 - RSW, xrr = x0 + TX == p.nx ? 0 : x0 + TX;
  bool pending[3] = {false, false, false};  // thread 0: copies issued, not yet waited for
  auto issue = [&](int pl) {  // thread 0 only
    const int gz = wrap(pl, p.nz);
    const int s = slot(pl);
    pending[s] = true;
    unsigned char* b = bufs + s * Lay::BUF;
    uint64_t* bar = &bars[s];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(bar, Lay::TX_BYTES);
    const int rows_y[3] = {yt, y0, yb};
    for (int g = 0; g < 3; g++) {
      const bool mid = g == 1;
      const int y = rows_y[g];
      tma_load_4d(b + Lay::PM::group(g), mid ? &maps.pop_main_mid : &maps.pop_main_row, x0, 0, y, gz, bar);
      tma_load_4d(b + Lay::OFF_L + Lay::PS::group(g), mid ? &maps.pop_strip_mid : &maps.pop_strip_row, xl, 0, y, gz,
                  bar);
      tma_load_4d(b + Lay::OFF_R + Lay::PS::group(g), mid ? &maps.pop_strip_mid : &maps.pop_strip_row, xr, 0, y, gz,
                  bar);
      tma_load_4d(b + Lay::OFF_RM + Lay::RMR::group(g), mid ? &maps.ref_main_mid : &maps.ref_main_row, x0, 0, y, gz,
                  bar);
      tma_load_4d(b + Lay::OFF_RL + Lay::RSR::group(g), mid ? &maps.ref_strip_mid : &maps.ref_strip_row, xlr, 0, y,
                  gz, bar);
      tma_load_4d(b + Lay::OFF_RR + Lay::RSR::group(g), mid ? &maps.ref_strip_mid : &maps.ref_strip_row, xrr, 0, y,
                  gz, bar);
    }
  };

  // Ext-node views into a plane buffer: (base, stride) such that array a of the node is
  // base[a * stride]; populations and reference densities.
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

  const int tx = threadIdx.x, ty = threadIdx.y;
  // ring task of this thread (84 ring nodes for 32 x 8, spread three threads apart)
  constexpr int NRING = 2 * EX + 2 * TY;
  constexpr int RSTRIDE = NI / NRING > 0 ? NI / NRING : 1;
  const bool has_ring = (tid % RSTRIDE == 0) && (tid / RSTRIDE < NRING);
  int rex = 0, rey = 0;
  if (has_ring) {
    const int r = tid / RSTRIDE;
    if (r < EX) {
      rex = r;
      rey = 0;
    } else if (r < 2 * EX) {
      rex = r - EX;
      rey = TY + 1;
    } else if (r < 2 * EX + TY) {
      rex = 0;
      rey = 1 + (r - 2 * EX);
    } else {
      rex = TX + 1;
      rey = 1 + (r - 2 * EX - TY);
    }
  }
  const int rgx = wrap(x0 - 1 + rex, p.nx), rgy = wrap(y0 - 1 + rey, p.ny);

  // densities and stencil fields of one ext node from a plane buffer
  auto stage_node = [&](const unsigned char* b, int ex, int ey, int sl, int gxn, int gyn, int gz) {
    const View v = view(b, ex, ey);
    const int e = ey * EX + ex;
    T rho[2] = {T(0), T(0)};
#pragma unroll
    for (int k = 0; k < K; k++) {
      T g[Q];
#pragma unroll
      for (int i = 0; i < Q; i++) g[i] = ld_s<S, T>(v.pop[(k * Q + i) * v.ps]);
      const CompState<T> c = comp_state<L, T, RT>(g, T(v.ref[k * v.rs]));
      rho[k] = c.rho;
      fld[(sl * NV + NF + k) * NE + e] = c.q;
    }
    T out[2];
    node_fields<MODEL, T>(p, rho[0], rho[1], out);
#pragma unroll
    for (int f = 0; f < NF; f++) fld[(sl * NV + f) * NE + e] = out[f];
    if (WALLS) msk[sl * NE + e] = solid[gxn + (long long)p.nx * (gyn + (long long)p.ny * gz)];
  };

  const int gx = x0 + tx, gy = y0 + ty;
  auto stage_plane = [&](int pl) {
    const int s = slot(pl);
    const unsigned char* b = bufs + s * Lay::BUF;
    const int gz = wrap(pl, p.nz);
    stage_node(b, tx + 1, ty + 1, s, gx, gy, gz);
    if (has_ring) stage_node(b, rex, rey, s, rgx, rgy, gz);
  };

  uint32_t phase[3] = {0, 0, 0};
  auto wait_plane = [&](int pl) -> bool {
    const int s = slot(pl);
    const bool ok = mbar_wait_bounded(&bars[s], phase[s]);
    phase[s] ^= 1;
    pending[s] = false;
    return ok;
  };
  // a wait gave up: flag it, and let thread 0 wait (bounded again) for the copies still
  // in flight into this block's shared memory before the block exits
  auto give_up = [&]() {
    if (tid == 0) {
      atomicOr(status, kStatusTimeout);
      for (int s = 0; s < 3; s++)
        if (pending[s]) mbar_wait_bounded(&bars[s], phase[s]);
    }
  };

  const int e0 = (ty + 1) * EX + (tx + 1);
  const int xm = gx == 0 ? p.nx - 1 : gx - 1, xp = gx + 1 >= p.nx ? 0 : gx + 1;
  const int ym = gy == 0 ? p.ny - 1 : gy - 1, yp = gy + 1 >= p.ny ? 0 : gy + 1;
  const long long nxl = p.nx;
  const long long plane_n = (long long)p.nx * p.ny;
  const long long rowm = ym * nxl, row0 = gy * nxl, rowp = yp * nxl;

  auto collide = [&](int z) {
    const int slm = slot(z - 1), sl0 = slot(z), slp = slot(z + 1);
    if (WALLS && msk[sl0 * NE + e0]) return;
    const View v = view(bufs + sl0 * Lay::BUF, tx + 1, ty + 1);
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
  };

  // prologue: planes z0-1, z0, z0+1 in flight; reduce z0-1, refill its buffer with z0+2
  if (tid == 0) {
    issue(z0 - 1);
    issue(z0);
    if (z0 + 1 <= z1) issue(z0 + 1);
  }
  bool ok = wait_plane(z0 - 1);
  if (ok) stage_plane(z0 - 1);
  if (__syncthreads_or(!ok)) {
    give_up();
    return;
  }
  if (tid == 0 && z0 + 2 <= z1) issue(z0 + 2);
  ok = wait_plane(z0);
  if (ok) stage_plane(z0);
  if (__syncthreads_or(!ok)) {
    give_up();
    return;
  }
  for (int z = z0; z < z1; z++) {
    ok = wait_plane(z + 1);
    if (ok) stage_plane(z + 1);
    if (__syncthreads_or(!ok)) {
      give_up();
      return;
    }
    collide(z);
    __syncthreads();
    if (tid == 0 && z + 3 <= z1) issue(z + 3);  // refill the buffer plane z used
  }
}

}  // namespace lbm
