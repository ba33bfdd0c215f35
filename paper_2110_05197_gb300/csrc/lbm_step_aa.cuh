// Field-pass steps: in-place streaming (AA pattern) with one population buffer, and the
// multirange Shan-Chen model, whose repulsive force reaches distance 2.
//
// Storage.  After an even number of steps the canonical population f^k_i(x) sits in slot i
// of node x; after an odd number, in slot opp(i) of node x - c_i.  An even step reads the
// node's own slots and writes post-collision f*_i to slot opp(i) of the same node; an odd
// step reads slot opp(i) of x - c_i and writes f*_i to slot i of x + c_i.  In both steps a
// node reads and writes the same Q locations per component and no other node touches them,
// so the update is race-free in place.  Halfway bounce-back (Eq. streaming with walls:
// f_opp(i)(x, t+1) = f*_i(x) when x + c_i is a wall node) goes, in an even step, to slot i
// of the wall node x + c_i (whence the next odd step reads it back as f_opp(i)(x)), and in
// an odd step to slot opp(i) of x; both locations belong to no other fluid node.
// Deviations (g = f - phi_i q) are re-referenced to the destination node's q exactly as in
// the two-buffer scheme; the reference densities are read and rewritten by their own node
// only, so they are updated in place as well.
//
// The stencils need the densities of the 18 neighbours at time t, which a neighbour may
// already have overwritten in place.  A first pass therefore writes every node's stencil
// fields and reference densities (NF + K values of the compute type) into a field array,
// and the step kernel reads its neighbours' values from there: 2*K*Q populations plus
// K*Q more per node for the pass, i.e. 1.5x the bytes of a two-buffer step, for half the
// population memory.
//
// The multirange SC model (Eq. benziforces) needs Psi at distance 2, beyond the halo of the
// plane-marching kernels, so it runs on the same two kernels in either storage mode: the
// field pass stores rho_s, Psi_s and q_s of every node, the step kernel reads the 92
// neighbours of belts 1 and 2 from there (L1/L2 serve the re-reads).
#pragma once

#include "lbm_step.cuh"

namespace lbm {

// Index of the canonical population f^k_i at node n = x + nx (y + ny z) in the in-place
// buffer after an even (odd == false) or odd number of steps.
template <class L>
__device__ __forceinline__ long long aa_index(int k, int i, long long n, int x, int y, int z, int nx, int ny, int nz,
                                              long long N, bool odd) {
  if (!odd || i == 0) return (long long)(k * L::Q + i) * N + n;
  return (long long)(k * L::Q + opp<L>(i)) * N + wrap_index(x - cx<L>(i), y - cy<L>(i), z - cz<L>(i), nx, ny, nz);
}

// The same in index type I (int when K Q N < 2^31).
template <class L, class I>
__device__ __forceinline__ I aa_index_nt(int k, int i, I n, int nx, int ny, int nz, I N, bool odd) {
  if (!odd || i == 0) return I(k * L::Q + i) * N + n;
  int x, y, z;
  node_coords(n, nx, ny, N, x, y, z);
  const int X = x - cx<L>(i), Y = y - cy<L>(i), Z = z - cz<L>(i);
  const int Xw = X < 0 ? X + nx : (X >= nx ? X - nx : X);
  const int Yw = Y < 0 ? Y + ny : (Y >= ny ? Y - ny : Y);
  const int Zw = Z < 0 ? Z + nz : (Z >= nz ? Z - nz : Z);
  return I(k * L::Q + opp<L>(i)) * N + (Xw + I(nx) * (Yw + I(ny) * Zw));
}

template <class L>
__device__ __forceinline__ long long aa_index_n(int k, int i, long long n, int nx, int ny, int nz, long long N,
                                                bool odd) {
  if (!odd || i == 0) return (long long)(k * L::Q + i) * N + n;
  int x, y, z;
  node_coords(n, nx, ny, N, x, y, z);
  return aa_index<L>(k, i, n, x, y, z, nx, ny, nz, N, odd);
}

// Field pass: fld[NF + K][N] = the stencil fields (node_fields) and the new reference
// densities q_k of every fluid node, from the state at t (layout parity `odd`).
template <class L, class T, class S, class RT, int MODEL>
__global__ void __launch_bounds__(256) fp_fields_kernel(const S* __restrict__ f, const RT* __restrict__ r,
                                                        T* __restrict__ fld, const uint8_t* __restrict__ solid,
                                                        const int* __restrict__ status, const StepParams<T> p,
                                                        int odd) {
  if (*status != 0) return;  // blown-up state: stop stepping
  constexpr int Q = L::Q, K = ModelTraits<MODEL>::K, NF = ModelTraits<MODEL>::NF;
  const long long N = p.n;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
    if (solid && solid[n]) continue;  // wall values are never read: the stencil substitutes the centre
    int x, y, z;
    node_coords(n, p.nx, p.ny, N, x, y, z);
    T rho[2] = {T(0), T(0)};
#pragma unroll
    for (int k = 0; k < K; k++) {
      T v[Q];
#pragma unroll
      for (int i = 0; i < Q; i++) v[i] = ld_s<S, T>(f[aa_index<L>(k, i, n, x, y, z, p.nx, p.ny, p.nz, N, odd)]);
      const CompState<T> c = comp_state<L, T, RT>(v, T(r[(long long)k * N + n]));
      rho[k] = c.rho;
      fld[(long long)(NF + k) * N + n] = c.q;
    }
    T out[NF > 2 ? NF : 2];
    node_fields<MODEL, T>(p, rho[0], rho[1], out);
#pragma unroll
    for (int fi = 0; fi < NF; fi++) fld[(long long)fi * N + n] = out[fi];
  }
}

// One step, one thread per node: moments, stencil from the field pass, collision (the same
// per-node code as the plane-marching kernels), streaming.  mode 0: two buffers (read fin,
// rin; push into fout, rout); mode 1 / 2: in place at even / odd layout parity (fin == fout,
// rin == rout; the pointers may alias, so none is restrict-qualified).
template <class L, class T, class S, class RT, int MODEL, bool WALLS, bool REP, class I = long long>
__global__ void __launch_bounds__(256, min_blocks<T>())
    fp_step_kernel(const S* fin, S* fout, const RT* rin, RT* rout, const T* __restrict__ fld,
                   const uint8_t* __restrict__ solid, const int* __restrict__ status,
                   const __grid_constant__ StepParams<T> p, const T* __restrict__ colour,
                   const T* __restrict__ normals, const __grid_constant__ RepParams rp, int mode) {
  if (*status != 0) return;
  const bool inplace = mode != 0, odd = mode == 2;
  constexpr int Q = L::Q, K = ModelTraits<MODEL>::K, NF = ModelTraits<MODEL>::NF;
  const I N = I(p.n);
  for (I n = blockIdx.x * I(blockDim.x) + threadIdx.x; n < N; n += I(gridDim.x) * blockDim.x) {
    if (WALLS && solid[n]) continue;
    int x, y, z;
    node_coords(n, p.nx, p.ny, N, x, y, z);
    const int xm = x == 0 ? p.nx - 1 : x - 1, xp = x + 1 >= p.nx ? 0 : x + 1;
    const int ym = y == 0 ? p.ny - 1 : y - 1, yp = y + 1 >= p.ny ? 0 : y + 1;
    const int zm = z == 0 ? p.nz - 1 : z - 1, zp = z + 1 >= p.nz ? 0 : z + 1;
    auto nb = [&](int i) -> I {
      const int X = cx<L>(i) == 0 ? x : (cx<L>(i) > 0 ? xp : xm);
      const int Y = cy<L>(i) == 0 ? y : (cy<L>(i) > 0 ? yp : ym);
      const int Z = cz<L>(i) == 0 ? z : (cz<L>(i) > 0 ? zp : zm);
      return X + I(p.nx) * (Y + I(p.ny) * Z);
    };
    // x - c_i = the neighbour in direction opp(i)
    T g[K][Q];
    CompState<T> cs[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
#pragma unroll
      for (int i = 0; i < Q; i++) {
        const I src = (odd && i != 0) ? I(k * Q + opp<L>(i)) * N + nb(opp<L>(i))
                                              : I(k * Q + i) * N + n;
        g[k][i] = ld_s<S, T>(fin[src]);
      }
      cs[k] = comp_state<L, T, RT>(g[k], T(rin[I(k) * N + n]));
    }
    auto nbr = [&](int fi, int i) -> T {
      const I m = nb(i);
      if (WALLS && solid[m]) return fld[I(fi) * N + n];
      return fld[I(fi) * N + m];
    };
    if constexpr (MODEL == kCG) {
      T Fx[3] = {T(0), T(0), T(0)};
      if constexpr (REP) rep_force<L, T, I>(normals, colour, WALLS ? solid : nullptr, x, y, z, rp, Fx);
      cg_collide<L, T>(p, g, cs[0], cs[1], nbr, Fx);
    } else if constexpr (MODEL == kSCMR) {
      auto far = [&](int fi, int dx, int dy, int dz) -> T {
        const I m = (I)wrap_index(x + dx, y + dy, z + dz, p.nx, p.ny, p.nz);
        if (WALLS && solid[m]) return fld[I(fi) * N + n];
        return fld[I(fi) * N + m];
      };
      scmr_collide<L, T>(p, g, cs[0], cs[1], nbr, far);
    } else if constexpr (MODEL == kSCMP) {
      scmp_collide<L, T>(p, g, cs[0], nbr);
    } else {
      sc2c_collide<L, T>(p, g, cs[0], cs[1], nbr);
    }
#pragma unroll
    for (int k = 0; k < K; k++) rout[I(k) * N + n] = RT(cs[k].q);
#pragma unroll
    for (int i = 0; i < Q; i++) {
      const I d = nb(i);
      const bool bounce = WALLS && i != 0 && solid[d];
#pragma unroll
      for (int k = 0; k < K; k++) {
        T v = g[k][i];
        if (i != 0 && !bounce) v += p.phi[k][grp<L>(i)] * (cs[k].q - fld[I(NF + k) * N + d]);
        I dst;
        if (i == 0)
          dst = I(k * Q) * N + n;
        else if (!inplace || odd)  // push to x + c_i; bounce-back into opp(i) of x
          dst = bounce ? I(k * Q + opp<L>(i)) * N + n : I(k * Q + i) * N + d;
        else                       // even in-place step: back into opp(i) of x
          dst = bounce ? I(k * Q + i) * N + d : I(k * Q + opp<L>(i)) * N + n;
        fout[dst] = st_s<S, T>(v);
      }
    }
  }
}

// The same step for D3Q19 with the neighbours' fields staged in shared memory (used for the
// multirange model): a block of
// TX x TY = 32 x 8 threads takes work units (column tile, z-chunk) as the plane-marching
// kernels do and marches z; a ring of 2H+1 planes holds the fields (and wall mask) of the
// (TX+2H) x (TY+2H) extended tile, H = 2 for the multirange model (belt 2) and 1 otherwise,
// loaded with coalesced rows from the field pass's array.  Populations move as in
// fp_step_kernel (mode 0 two buffers, 1 / 2 in place at even / odd parity).
constexpr int kFpTX = 32, kFpTY = 8;

template <class T, int MODEL, bool WALLS, int H>
__host__ __device__ constexpr size_t fpt_smem_bytes() {
  constexpr int NV = ModelTraits<MODEL>::NF + ModelTraits<MODEL>::K;
  constexpr size_t ne = size_t(kFpTX + 2 * H) * (kFpTY + 2 * H);
  return (((2 * H + 1) * (NV * ne * sizeof(T) + (WALLS ? ne : 0))) + 15) & ~size_t(15);
}

template <class L, class T, class S, class RT, int MODEL, bool WALLS, bool REP, int H, class I = long long>
__global__ void __launch_bounds__(kFpTX * kFpTY, min_blocks<T>())
    fpt_step_kernel(const S* fin, S* fout, const RT* rin, RT* rout, const T* __restrict__ fld,
                    const uint8_t* __restrict__ solid, const int* __restrict__ status,
                    const __grid_constant__ StepParams<T> p, const T* __restrict__ colour,
                    const T* __restrict__ normals, const __grid_constant__ RepParams rp, int mode) {
  if (*status != 0) return;
  static_assert(L::D == 3, "plane marching");
  constexpr int TX = kFpTX, TY = kFpTY;
  constexpr int EX = TX + 2 * H, NE = EX * (TY + 2 * H), NS = 2 * H + 1;
  constexpr int Q = L::Q, K = ModelTraits<MODEL>::K, NF = ModelTraits<MODEL>::NF, NV = NF + K;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sf = reinterpret_cast<T*>(smem_raw);                      // [NS][NV][NE]
  uint8_t* sm = reinterpret_cast<uint8_t*>(sf + NS * NV * NE);  // [NS][NE] (walls)
  const bool inplace = mode != 0, odd = mode == 2;
  const I N = I(p.n);
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  auto slot = [](int z) { return ((z % NS) + NS) % NS; };
  WorkRange work(blockIdx.x, p.nblk, p.ncol, p.nz, p.nchunks);
  Segment sg;
  while (work.pop(sg)) {
    const int x0 = (sg.col % p.ncx) * TX, y0 = (sg.col / p.ncx) * TY;
    auto load = [&](int z) {
      const int sl = slot(z);
      const int gz = wrap(z, p.nz);
      for (int e = tid; e < NE; e += TX * TY) {
        const int ey = e / EX, ex = e - ey * EX;
        const I m = wrap(x0 - H + ex, p.nx) + I(p.nx) * (wrap(y0 - H + ey, p.ny) + I(p.ny) * gz);
#pragma unroll
        for (int fi = 0; fi < NV; fi++) sf[(sl * NV + fi) * NE + e] = fld[I(fi) * N + m];
        if (WALLS) sm[sl * NE + e] = solid[m];
      }
    };
    for (int z = sg.z0 - H; z < sg.z0 + H; z++) load(z);
    for (int z = sg.z0; z < sg.z1; z++) {
      load(z + H);
      __syncthreads();
      const int x = x0 + tx, y = y0 + ty;
      const int e0 = (ty + H) * EX + (tx + H);
      const int sl0 = slot(z);
      if (x < p.nx && y < p.ny && !(WALLS && sm[sl0 * NE + e0])) {
        const I n = x + I(p.nx) * (y + I(p.ny) * z);
        const int xm = x == 0 ? p.nx - 1 : x - 1, xp = x + 1 >= p.nx ? 0 : x + 1;
        const int ym = y == 0 ? p.ny - 1 : y - 1, yp = y + 1 >= p.ny ? 0 : y + 1;
        const int zm = z == 0 ? p.nz - 1 : z - 1, zp = z + 1 >= p.nz ? 0 : z + 1;
        auto nb = [&](int i) -> I {
          const int X = cx<L>(i) == 0 ? x : (cx<L>(i) > 0 ? xp : xm);
          const int Y = cy<L>(i) == 0 ? y : (cy<L>(i) > 0 ? yp : ym);
          const int Z = cz<L>(i) == 0 ? z : (cz<L>(i) > 0 ? zp : zm);
          return X + I(p.nx) * (Y + I(p.ny) * Z);
        };
        T g[K][Q];
        CompState<T> cs[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
#pragma unroll
          for (int i = 0; i < Q; i++) {
            const I src = (odd && i != 0) ? I(k * Q + opp<L>(i)) * N + nb(opp<L>(i))
                                                  : I(k * Q + i) * N + n;
            g[k][i] = ld_s<S, T>(fin[src]);
          }
          cs[k] = comp_state<L, T, RT>(g[k], T(rin[I(k) * N + n]));
        }
        auto at = [&](int fi, int dx, int dy, int dz) -> T {
          const int sl = slot(z + dz), e = e0 + dy * EX + dx;
          if (WALLS && sm[sl * NE + e]) return sf[(sl0 * NV + fi) * NE + e0];
          return sf[(sl * NV + fi) * NE + e];
        };
        auto nbr = [&](int fi, int i) -> T { return at(fi, cx<L>(i), cy<L>(i), cz<L>(i)); };
        if constexpr (MODEL == kCG) {
          T Fx[3] = {T(0), T(0), T(0)};
          if constexpr (REP) rep_force<L, T, I>(normals, colour, WALLS ? solid : nullptr, x, y, z, rp, Fx);
          cg_collide<L, T>(p, g, cs[0], cs[1], nbr, Fx);
        } else if constexpr (MODEL == kSCMR) {
          scmr_collide<L, T>(p, g, cs[0], cs[1], nbr, at);
        } else if constexpr (MODEL == kSCMP) {
          scmp_collide<L, T>(p, g, cs[0], nbr);
        } else {
          sc2c_collide<L, T>(p, g, cs[0], cs[1], nbr);
        }
#pragma unroll
        for (int k = 0; k < K; k++) rout[I(k) * N + n] = RT(cs[k].q);
#pragma unroll
        for (int i = 0; i < Q; i++) {
          const I d = nb(i);
          const int sl = slot(z + cz<L>(i)), ed = e0 + cy<L>(i) * EX + cx<L>(i);
          const bool bounce = WALLS && i != 0 && sm[sl * NE + ed];
#pragma unroll
          for (int k = 0; k < K; k++) {
            T v = g[k][i];
            if (i != 0 && !bounce) v += p.phi[k][grp<L>(i)] * (cs[k].q - sf[(sl * NV + NF + k) * NE + ed]);
            I dst;
            if (i == 0)
              dst = I(k * Q) * N + n;
            else if (!inplace || odd)
              dst = bounce ? I(k * Q + opp<L>(i)) * N + n : I(k * Q + i) * N + d;
            else
              dst = bounce ? I(k * Q + i) * N + d : I(k * Q + opp<L>(i)) * N + n;
            fout[dst] = st_s<S, T>(v);
          }
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace lbm
