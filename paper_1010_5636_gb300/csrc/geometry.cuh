// Site geometry on the device: even-odd index <-> coordinates and neighbours, computed
// arithmetically (no neighbour tables are read by the operator kernels).
//
//   lex(x) = x3 + L3*(x2 + L2*(x1 + L1*x0)),  p(x) = (x0+x1+x2+x3) mod 2,
//   eo(x)  = p(x)*Vh + floor(lex/2),  Vh = V/2, all extents even.
// For a site (p, h): q = floor(2h / L3) fixes (x0, x1, x2); since L3 is even, the parity of
// x3 equals lex mod 2 = b with b = (p + x0 + x1 + x2) mod 2, so x3 = (2h mod L3) + b and
// lex = 2h + b.  A neighbour x +- mu differs in lex by +-stride_mu (or wraps by
// -+(L_mu - 1)*stride_mu) and has the other parity; its half index is floor(lex'/2).
#pragma once
#include <stdint.h>

namespace nd {

struct Geom {
  int L[4];        // extents T, L1, L2, L3
  int stride[4];   // lex strides: L1*L2*L3, L2*L3, L3, 1
  int Vh;          // sites per parity
  int apbc;        // 1: antiperiodic in time
  int even_only;   // BLAS-1 kernels: 1 = fields of the even sites only (parity 0), 0 = whole lattice
  // division by L[1], L[2], L[3] as a multiply-high (set by geom_set_divisors): for a divisor d
  // with l = ceil(log2 d), n / d = (t + ((n - t) >> 1)) >> (l - 1), t = umulhi(n, div_m),
  // div_m = floor(2^32 (2^l - d) / d) + 1, exact for every 32-bit n (Granlund and Montgomery, 1994)
  unsigned div_m[4];
  int div_l[4];
};

// Fill the division constants of g for L[1..3] (all extents are even, so every l >= 1).
__host__ inline void geom_set_divisors(Geom& g) {
  for (int k = 1; k < 4; ++k) {
    const unsigned d = (unsigned)g.L[k];
    int l = 0;
    while ((1ull << l) < d) ++l;
    g.div_l[k] = l;
    g.div_m[k] = (unsigned)((((1ull << l) - d) << 32) / d + 1);
  }
  g.div_l[0] = 0;
  g.div_m[0] = 0;
}

__device__ __forceinline__ unsigned geom_div(unsigned n, const Geom& g, int k) {
  const unsigned t = __umulhi(n, g.div_m[k]);
  return (t + ((n - t) >> 1)) >> (g.div_l[k] - 1);
}

// Sites a BLAS-1 launch covers: parity 0 comes first in every field layout, so an even-site field
// is the first half of a whole-lattice one.
__host__ __device__ inline int blas_sites(const Geom& g) { return g.even_only ? g.Vh : 2 * g.Vh; }

struct Site {
  int x[4];
  int lex;
};

__device__ __forceinline__ Site site_of(const Geom& g, int p, int h) {
  Site s;
  unsigned twoh = 2u * (unsigned)h;
  unsigned q = geom_div(twoh, g, 3);
  unsigned r3 = twoh - q * (unsigned)g.L[3];
  unsigned q2 = geom_div(q, g, 2);
  s.x[2] = (int)(q - q2 * (unsigned)g.L[2]);
  unsigned q1 = geom_div(q2, g, 1);
  s.x[1] = (int)(q2 - q1 * (unsigned)g.L[1]);
  s.x[0] = (int)q1;
  int b = (p + s.x[0] + s.x[1] + s.x[2]) & 1;
  s.x[3] = (int)r3 + b;
  s.lex = (int)twoh + b;
  return s;
}

// Output site of thread slot i in a launch over both parities: runs of 32 slots alternate
// parity over the same 32 half indices, p = (i / 32) mod 2, h = 32 (i / 64) + i mod 32.  Each warp
// thus reads one contiguous, aligned run of every field, and the two warps of a pair use the links
// and neighbours of one h range while they are still in cache.  Slots with h >= Vh are idle.
__host__ __device__ __forceinline__ void both_parities_site(int i, int* p, int* h) {
  *p = (i >> 5) & 1;
  *h = ((i >> 6) << 5) | (i & 31);
}

// Half index of the neighbour x + mu (fwd) or x - mu (bwd); *crossed = 1 if the hop wraps
// around the time boundary (for antiperiodic boundary conditions).
template <int MU, bool FWD>
__device__ __forceinline__ int neighbour_h(const Geom& g, const Site& s, bool* crossed) {
  int lex;
  if (FWD) {
    bool wrap = s.x[MU] == g.L[MU] - 1;
    lex = wrap ? s.lex - (g.L[MU] - 1) * g.stride[MU] : s.lex + g.stride[MU];
    *crossed = wrap && MU == 0;
  } else {
    bool wrap = s.x[MU] == 0;
    lex = wrap ? s.lex + (g.L[MU] - 1) * g.stride[MU] : s.lex - g.stride[MU];
    *crossed = wrap && MU == 0;
  }
  return lex >> 1;
}

}  // namespace nd
