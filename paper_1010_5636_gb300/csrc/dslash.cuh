// The Wilson-Dirac stencil Q = gamma5 D_W on the device (Sec. 2.1), one thread per output site.
//
//   D_W phi(x) = (4+m) phi(x) - 1/2 sum_{mu=+-0..+-3} U_mu(x) (1 - gamma_mu) phi(x+mu),
//   U_{-mu}(x) = U_mu(x-mu)^dagger, gamma_{-mu} = -gamma_mu.
//
// Chiral basis: gamma_mu = [[0, B_mu], [B_mu^dagger, 0]] with B_0 = -1, B_k = -i sigma_k, so
// (1 -+ gamma_mu) has rank 2: with h = psi_up -+ B_mu psi_dn (2 spins x 3 colours),
// (1 -+ gamma_mu) psi = [h ; -+ B_mu^dagger h].  Each hop therefore projects to a half spinor,
// multiplies two colour vectors by the link (or its dagger) and rebuilds the lower spins.
#pragma once
#include "fields.cuh"
#include "geometry.cuh"

namespace nd {

// Half spinor h = psi_up + S B psi_dn for S = -1 (forward hop, 1 - gamma) or +1 (backward, 1 + gamma).
template <int MU, bool FWD, typename T>
__device__ __forceinline__ void spin_project(const Spinor<T>& s, cx<T> (&h)[2][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if constexpr (MU == 0) {  // B = -1
      h[0][i] = FWD ? s.s[0][i] + s.s[2][i] : s.s[0][i] - s.s[2][i];
      h[1][i] = FWD ? s.s[1][i] + s.s[3][i] : s.s[1][i] - s.s[3][i];
    } else if constexpr (MU == 1) {  // B = -i sigma1: B psi_dn = (-i psi3, -i psi2)
      h[0][i] = FWD ? s.s[0][i] + itimes(s.s[3][i]) : s.s[0][i] - itimes(s.s[3][i]);
      h[1][i] = FWD ? s.s[1][i] + itimes(s.s[2][i]) : s.s[1][i] - itimes(s.s[2][i]);
    } else if constexpr (MU == 2) {  // B = -i sigma2 = [[0,-1],[1,0]]: B psi_dn = (-psi3, psi2)
      h[0][i] = FWD ? s.s[0][i] + s.s[3][i] : s.s[0][i] - s.s[3][i];
      h[1][i] = FWD ? s.s[1][i] - s.s[2][i] : s.s[1][i] + s.s[2][i];
    } else {  // B = -i sigma3 = diag(-i, i): B psi_dn = (-i psi2, i psi3)
      h[0][i] = FWD ? s.s[0][i] + itimes(s.s[2][i]) : s.s[0][i] - itimes(s.s[2][i]);
      h[1][i] = FWD ? s.s[1][i] - itimes(s.s[3][i]) : s.s[1][i] + itimes(s.s[3][i]);
    }
  }
}

// acc += [c ; S B^dagger c] with c the colour-multiplied half spinor.
template <int MU, bool FWD, typename T>
__device__ __forceinline__ void spin_accumulate(Spinor<T>& acc, const cx<T> (&c)[2][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    acc.s[0][i] = acc.s[0][i] + c[0][i];
    acc.s[1][i] = acc.s[1][i] + c[1][i];
    if constexpr (MU == 0) {  // S B^dagger = -S: fwd (+c0, +c1), bwd (-c0, -c1)
      acc.s[2][i] = FWD ? acc.s[2][i] + c[0][i] : acc.s[2][i] - c[0][i];
      acc.s[3][i] = FWD ? acc.s[3][i] + c[1][i] : acc.s[3][i] - c[1][i];
    } else if constexpr (MU == 1) {  // B^dagger = i sigma1: B^dagger c = (i c1, i c0)
      acc.s[2][i] = FWD ? acc.s[2][i] - itimes(c[1][i]) : acc.s[2][i] + itimes(c[1][i]);
      acc.s[3][i] = FWD ? acc.s[3][i] - itimes(c[0][i]) : acc.s[3][i] + itimes(c[0][i]);
    } else if constexpr (MU == 2) {  // B^dagger = i sigma2 = [[0,1],[-1,0]]: B^dagger c = (c1, -c0)
      acc.s[2][i] = FWD ? acc.s[2][i] - c[1][i] : acc.s[2][i] + c[1][i];
      acc.s[3][i] = FWD ? acc.s[3][i] + c[0][i] : acc.s[3][i] - c[0][i];
    } else {  // B^dagger = i sigma3 = diag(i, -i): B^dagger c = (i c0, -i c1)
      acc.s[2][i] = FWD ? acc.s[2][i] - itimes(c[0][i]) : acc.s[2][i] + itimes(c[0][i]);
      acc.s[3][i] = FWD ? acc.s[3][i] + itimes(c[1][i]) : acc.s[3][i] - itimes(c[1][i]);
    }
  }
}

// c = U h (forward) or U^dagger h (backward), for both spin rows of the half spinor.
template <bool DAG, typename T>
__device__ __forceinline__ void colour_mul(const Su3<T>& U, const cx<T> (&h)[2][3], cx<T> (&c)[2][3]) {
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      cx<T> v = mk((T)0, (T)0);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        if (DAG)
          cfmac(v, U.e[j][i], h[k][j]);
        else
          cfma(v, U.e[i][j], h[k][j]);
      }
      c[k][i] = v;
    }
}

// One hop (direction MU, forward or backward) from the neighbour of parity 1-p into acc.
template <int P, int R, int MU, bool FWD>
__device__ __forceinline__ void hop(Spinor<typename Traits<P>::real>& acc, const Geom& g, const Site& s, int p,
                                    int h, const char* links, const void* in) {
  using T = typename Traits<P>::real;
  bool crossed;
  const int hn = neighbour_h<MU, FWD>(g, s, &crossed);
  Spinor<T> nb;
  SpinorIO<P>::load(nb, in, g.Vh, 1 - p, hn);
  LinkRaw<P, R> raw;
  if (FWD)
    load_raw<P, R>(raw, links, g.Vh, p, MU, h);
  else
    load_raw<P, R>(raw, links, g.Vh, 1 - p, MU, hn);
  cx<T> hs[2][3], c[2][3];
  spin_project<MU, FWD>(nb, hs);
  if (g.apbc && crossed) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) hs[k][i] = -hs[k][i];
  }
  Su3<T> U;
  reconstruct<P, R>(U, raw);
  colour_mul<!FWD>(U, hs, c);
  spin_accumulate<MU, FWD>(acc, c);
}

// Sum of the eight hops: acc = sum_mu [U_mu(x)(1-gamma_mu)psi(x+mu) + U_mu(x-mu)^dag (1+gamma_mu) psi(x-mu)].
template <int P, int R>
__device__ __forceinline__ void hopping_sum(Spinor<typename Traits<P>::real>& acc, const Geom& g, const Site& s,
                                            int p, int h, const char* links, const void* in) {
  using T = typename Traits<P>::real;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) acc.s[a][i] = mk((T)0, (T)0);
  hop<P, R, 0, true>(acc, g, s, p, h, links, in);
  hop<P, R, 0, false>(acc, g, s, p, h, links, in);
  hop<P, R, 1, true>(acc, g, s, p, h, links, in);
  hop<P, R, 1, false>(acc, g, s, p, h, links, in);
  hop<P, R, 2, true>(acc, g, s, p, h, links, in);
  hop<P, R, 2, false>(acc, g, s, p, h, links, in);
  hop<P, R, 3, true>(acc, g, s, p, h, links, in);
  hop<P, R, 3, false>(acc, g, s, p, h, links, in);
}

}  // namespace nd
