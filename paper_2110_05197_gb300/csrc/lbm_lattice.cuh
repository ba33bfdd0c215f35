// Lattice traits for the device code: D3Q19 (Eqs. speeds, weights) and D2Q9.
//
// Direction order: rest, then opposite pairs (2p+1, 2p+2) with c_{2p+2} = -c_{2p+1}:
//   D3Q19 pairs: x, y, z, (1,1,0), (1,-1,0), (1,0,1), (1,0,-1), (0,1,1), (0,1,-1)
//   D2Q9  pairs: x, y, (1,1), (1,-1)
// Per-group constants (rest / axis / diagonal):
//   w   : D3Q19 1/3, 1/18, 1/36 (Eq. weights);         D2Q9 4/9, 1/9, 1/36
//   B   : D3Q19 -2/9, 1/54, 1/27 (after Eq. perturbationOp); D2Q9 -4/27, 2/27, 5/108
//   psi : D3Q19 -5/2, -1/6, 1/24 (after Eq. phi);       D2Q9 -8/3, -1/6, 1/12
//   xi  : D3Q19 0, 1/4, 1/8;                            D2Q9 0, 1/2, 1/8
//   phi : D3Q19 alpha, (1-alpha)/12, (1-alpha)/24 (Eq. phi); D2Q9 alpha, (1-alpha)/5, (1-alpha)/20
// The D2Q9 constants are not in the paper; they satisfy the same moment identities as the
// D3Q19 set (sum B = 1/3, sum B cc = I/3, sum psi + 2 sum xi c_x^2 = 0, sum psi cc = 0,
// sum xi c^4 = (1/2)(dd+dd+dd), c_s^2 = 3(1-alpha)/5).
#pragma once

#include <cstdint>

namespace lbm {

struct D3Q19 {
  static constexpr int D = 3;
  static constexpr int Q = 19;
  static constexpr int NP = 9;  // opposite pairs
  // components of the positive member of each pair
  __host__ __device__ static constexpr int pcx(int p) {
    return p == 0 ? 1 : p == 1 ? 0 : p == 2 ? 0 : p == 3 ? 1 : p == 4 ? 1 : p == 5 ? 1 : p == 6 ? 1 : 0;
  }
  __host__ __device__ static constexpr int pcy(int p) {
    return p == 0 ? 0 : p == 1 ? 1 : p == 2 ? 0 : p == 3 ? 1 : p == 4 ? -1 : p == 5 ? 0 : p == 6 ? 0 : p == 7 ? 1 : 1;
  }
  __host__ __device__ static constexpr int pcz(int p) {
    return p == 0 ? 0 : p == 1 ? 0 : p == 2 ? 1 : p == 3 ? 0 : p == 4 ? 0 : p == 5 ? 1 : p == 6 ? -1 : p == 7 ? 1 : -1;
  }
  __host__ __device__ static constexpr int pgrp(int p) { return p < 3 ? 1 : 2; }
  __host__ __device__ static constexpr double w(int g) { return g == 0 ? 1.0 / 3.0 : g == 1 ? 1.0 / 18.0 : 1.0 / 36.0; }
  __host__ __device__ static constexpr double B(int g) { return g == 0 ? -2.0 / 9.0 : g == 1 ? 1.0 / 54.0 : 1.0 / 27.0; }
  __host__ __device__ static constexpr double psi(int g) { return g == 0 ? -2.5 : g == 1 ? -1.0 / 6.0 : 1.0 / 24.0; }
  __host__ __device__ static constexpr double xi(int g) { return g == 0 ? 0.0 : g == 1 ? 0.25 : 0.125; }
  __host__ __device__ static constexpr double phi_num(int g) { return g == 0 ? 1.0 : g == 1 ? 1.0 / 12.0 : 1.0 / 24.0; }
};

struct D2Q9 {
  static constexpr int D = 2;
  static constexpr int Q = 9;
  static constexpr int NP = 4;
  __host__ __device__ static constexpr int pcx(int p) { return p == 1 ? 0 : 1; }
  __host__ __device__ static constexpr int pcy(int p) { return p == 0 ? 0 : p == 3 ? -1 : 1; }
  __host__ __device__ static constexpr int pcz(int) { return 0; }
  __host__ __device__ static constexpr int pgrp(int p) { return p < 2 ? 1 : 2; }
  __host__ __device__ static constexpr double w(int g) { return g == 0 ? 4.0 / 9.0 : g == 1 ? 1.0 / 9.0 : 1.0 / 36.0; }
  __host__ __device__ static constexpr double B(int g) { return g == 0 ? -4.0 / 27.0 : g == 1 ? 2.0 / 27.0 : 5.0 / 108.0; }
  __host__ __device__ static constexpr double psi(int g) { return g == 0 ? -8.0 / 3.0 : g == 1 ? -1.0 / 6.0 : 1.0 / 12.0; }
  __host__ __device__ static constexpr double xi(int g) { return g == 0 ? 0.0 : g == 1 ? 0.5 : 0.125; }
  __host__ __device__ static constexpr double phi_num(int g) { return g == 0 ? 1.0 : g == 1 ? 0.2 : 0.05; }
};

// Direction i (0..Q-1) helpers built on the pair tables.
template <class L>
__host__ __device__ constexpr int cx(int i) { return i == 0 ? 0 : ((i & 1) ? L::pcx((i - 1) >> 1) : -L::pcx((i - 1) >> 1)); }
template <class L>
__host__ __device__ constexpr int cy(int i) { return i == 0 ? 0 : ((i & 1) ? L::pcy((i - 1) >> 1) : -L::pcy((i - 1) >> 1)); }
template <class L>
__host__ __device__ constexpr int cz(int i) { return i == 0 ? 0 : ((i & 1) ? L::pcz((i - 1) >> 1) : -L::pcz((i - 1) >> 1)); }
template <class L>
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
template <class L>
__host__ __device__ constexpr int grp(int i) { return i == 0 ? 0 : L::pgrp((i - 1) >> 1); }

// Coordinates (x, y, z) of node n = x + nx (y + ny z) of a lattice of N nodes, in 32-bit
// arithmetic whenever N allows it (64-bit integer division is a long instruction sequence).
__device__ __forceinline__ void node_coords(long long n, int nx, int ny, long long N, int& x, int& y, int& z) {
  if (N < (1LL << 31)) {
    const unsigned m = (unsigned)n, row = m / (unsigned)nx;
    x = (int)(m - row * (unsigned)nx);
    z = (int)(row / (unsigned)ny);
    y = (int)(row - (unsigned)z * (unsigned)ny);
  } else {
    x = (int)(n % nx);
    y = (int)((n / nx) % ny);
    z = (int)(n / ((long long)nx * ny));
  }
}

}  // namespace lbm
