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

// ------------------------------------------------------------------ packed FP32 form
// FP32 and FP16 storage run the hop on spin-row pairs (Spinor2): both rows of a half spinor meet
// the same link entries, so every SU(3) multiply-add, projection sum and accumulation acts on a
// pair (s0, s1) or (s2, s3) with one f32x2 instruction.  Per lane the operations and their order
// are those of the scalar hop above.

__device__ __forceinline__ float2 f2_swap(float2 a) { return make_float2(a.y, a.x); }
__device__ __forceinline__ float2 f2_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2_bcast(float a) { return make_float2(a, a); }

// Half spinor pairs hr[i] = (h0[i].re, h1[i].re), hi[i] = (h0[i].im, h1[i].im) of spin_project.
template <int MU, bool FWD>
__device__ __forceinline__ void spin_project2(const Spinor2& s, float2 (&hr)[3], float2 (&hi)[3]) {
  const float2 pm = make_float2(1.f, -1.f), mp = make_float2(-1.f, 1.f);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if constexpr (MU == 0) {  // h0 = s0 -+ (-s2), h1 = s1 -+ (-s3)
      hr[i] = FWD ? f2_add(s.ur[i], s.dr[i]) : f2_add(s.ur[i], f2_neg(s.dr[i]));
      hi[i] = FWD ? f2_add(s.ui[i], s.di[i]) : f2_add(s.ui[i], f2_neg(s.di[i]));
    } else if constexpr (MU == 1) {  // h0 = s0 +- i s3, h1 = s1 +- i s2
      hr[i] = FWD ? f2_add(s.ur[i], f2_neg(f2_swap(s.di[i]))) : f2_add(s.ur[i], f2_swap(s.di[i]));
      hi[i] = FWD ? f2_add(s.ui[i], f2_swap(s.dr[i])) : f2_add(s.ui[i], f2_neg(f2_swap(s.dr[i])));
    } else if constexpr (MU == 2) {  // h0 = s0 +- s3, h1 = s1 -+ s2
      hr[i] = f2_fma(f2_swap(s.dr[i]), FWD ? pm : mp, s.ur[i]);
      hi[i] = f2_fma(f2_swap(s.di[i]), FWD ? pm : mp, s.ui[i]);
    } else {  // h0 = s0 +- i s2, h1 = s1 -+ i s3
      hr[i] = f2_fma(s.di[i], FWD ? mp : pm, s.ur[i]);
      hi[i] = f2_fma(s.dr[i], FWD ? pm : mp, s.ui[i]);
    }
  }
}

// c = U h (forward) or U^dagger h (backward) on the pairs: c_re += u_re h_re - u_im h_im,
// c_im += u_re h_im + u_im h_re (conj(u) for the dagger), in the order of cfma / cfmac.
template <bool DAG>
__device__ __forceinline__ void colour_mul2(const Su3<float>& U, const float2 (&hr)[3], const float2 (&hi)[3],
                                            float2 (&cr)[3], float2 (&ci)[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float2 vr = make_float2(0.f, 0.f), vi = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const cx<float> u = DAG ? U.e[j][i] : U.e[i][j];
      const float2 ur = f2_bcast(u.re), ui = f2_bcast(u.im), un = f2_bcast(-u.im);
      vr = f2_fma(ur, hr[j], vr);
      vr = f2_fma(DAG ? ui : un, hi[j], vr);
      vi = f2_fma(ur, hi[j], vi);
      vi = f2_fma(DAG ? un : ui, hr[j], vi);
    }
    cr[i] = vr;
    ci[i] = vi;
  }
}

// acc += [c ; S B^dagger c] (spin_accumulate on the pairs).
template <int MU, bool FWD>
__device__ __forceinline__ void spin_accumulate2(Spinor2& acc, const float2 (&cr)[3], const float2 (&ci)[3]) {
  const float2 pm = make_float2(1.f, -1.f), mp = make_float2(-1.f, 1.f);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    acc.ur[i] = f2_add(acc.ur[i], cr[i]);
    acc.ui[i] = f2_add(acc.ui[i], ci[i]);
    if constexpr (MU == 0) {  // fwd (+c0, +c1), bwd (-c0, -c1)
      acc.dr[i] = FWD ? f2_add(acc.dr[i], cr[i]) : f2_add(acc.dr[i], f2_neg(cr[i]));
      acc.di[i] = FWD ? f2_add(acc.di[i], ci[i]) : f2_add(acc.di[i], f2_neg(ci[i]));
    } else if constexpr (MU == 1) {  // fwd (-i c1, -i c0), bwd (+i c1, +i c0)
      acc.dr[i] = FWD ? f2_add(acc.dr[i], f2_swap(ci[i])) : f2_add(acc.dr[i], f2_neg(f2_swap(ci[i])));
      acc.di[i] = FWD ? f2_add(acc.di[i], f2_neg(f2_swap(cr[i]))) : f2_add(acc.di[i], f2_swap(cr[i]));
    } else if constexpr (MU == 2) {  // fwd (-c1, +c0), bwd (+c1, -c0)
      acc.dr[i] = f2_fma(f2_swap(cr[i]), FWD ? mp : pm, acc.dr[i]);
      acc.di[i] = f2_fma(f2_swap(ci[i]), FWD ? mp : pm, acc.di[i]);
    } else {  // fwd (-i c0, +i c1), bwd (+i c0, -i c1)
      acc.dr[i] = f2_fma(ci[i], FWD ? pm : mp, acc.dr[i]);
      acc.di[i] = f2_fma(cr[i], FWD ? mp : pm, acc.di[i]);
    }
  }
}

__device__ __forceinline__ void zero2(Spinor2& a) {
#pragma unroll
  for (int i = 0; i < 3; ++i) a.ur[i] = a.ui[i] = a.dr[i] = a.di[i] = make_float2(0.f, 0.f);
}

// The operands of one packed hop of the FP32 / FP16 operator, loaded ahead of its arithmetic.
template <int P, int R>
struct HopOperands {
  Spinor2 nb;
  LinkRaw<P, R> raw;
  bool crossed;
};

template <int P, int R, int MU, bool FWD>
__device__ __forceinline__ void hop2_load(HopOperands<P, R>& d, const Geom& g, const Site& s, int p, int h,
                                          const char* links, const void* in) {
  const int hn = neighbour_h<MU, FWD>(g, s, &d.crossed);
  SpinorIO<P>::load2(d.nb, in, g.Vh, 1 - p, hn);
  if (FWD)
    load_raw<P, R>(d.raw, links, g.Vh, p, MU, h);
  else
    load_raw<P, R>(d.raw, links, g.Vh, 1 - p, MU, hn);
}

template <int P, int R, int MU, bool FWD>
__device__ __forceinline__ void hop2_compute(Spinor2& acc, const HopOperands<P, R>& d, const Geom& g) {
  float2 hr[3], hi[3], cr[3], ci[3];
  spin_project2<MU, FWD>(d.nb, hr, hi);
  if (g.apbc && d.crossed) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      hr[i] = f2_neg(hr[i]);
      hi[i] = f2_neg(hi[i]);
    }
  }
  Su3<float> U;
  reconstruct<P, R>(U, d.raw);
  colour_mul2<!FWD>(U, hr, hi, cr, ci);
  spin_accumulate2<MU, FWD>(acc, cr, ci);
}

// The eight packed hops with the operands of the hops two and three ahead requested before the
// current hop's arithmetic (three operand sets rotating), in the order of hopping_sum.  The same
// arithmetic as loading and computing each hop in turn, bit for bit; written this way the
// scheduler keeps the loads of later hops in flight while a hop computes.  Measured on 64x32^3 back
// to back, one-parity hop: 96.5 us with every hop loaded just before its arithmetic, 96.0 us with one
// hop ahead, 94.5 us with two (full Q 157.8 / 156.7 / 155.3 us), all at 128 registers.
template <int P, int R>
__device__ __forceinline__ void hopping_sum2(Spinor2& acc, const Geom& g, const Site& s, int p, int h,
                                             const char* L, const void* in) {
  zero2(acc);
  if constexpr (R == 8 || P == P16) {
    // one hop ahead: the 8-real rebuild needs the registers (three sets spilled ~200 bytes), and
    // FP16, bound by instruction issue, measured 5 % slower with three sets (64x32^3, flushed:
    // 12-real hop 84.6 against 80.5 us)
    HopOperands<P, R> a, b;
    hop2_load<P, R, 0, true>(a, g, s, p, h, L, in);
    hop2_load<P, R, 0, false>(b, g, s, p, h, L, in);
    hop2_compute<P, R, 0, true>(acc, a, g);
    hop2_load<P, R, 1, true>(a, g, s, p, h, L, in);
    hop2_compute<P, R, 0, false>(acc, b, g);
    hop2_load<P, R, 1, false>(b, g, s, p, h, L, in);
    hop2_compute<P, R, 1, true>(acc, a, g);
    hop2_load<P, R, 2, true>(a, g, s, p, h, L, in);
    hop2_compute<P, R, 1, false>(acc, b, g);
    hop2_load<P, R, 2, false>(b, g, s, p, h, L, in);
    hop2_compute<P, R, 2, true>(acc, a, g);
    hop2_load<P, R, 3, true>(a, g, s, p, h, L, in);
    hop2_compute<P, R, 2, false>(acc, b, g);
    hop2_load<P, R, 3, false>(b, g, s, p, h, L, in);
    hop2_compute<P, R, 3, true>(acc, a, g);
    hop2_compute<P, R, 3, false>(acc, b, g);
    return;
  }
  HopOperands<P, R> a, b, c;
  hop2_load<P, R, 0, true>(a, g, s, p, h, L, in);
  hop2_load<P, R, 0, false>(b, g, s, p, h, L, in);
  hop2_load<P, R, 1, true>(c, g, s, p, h, L, in);
  hop2_compute<P, R, 0, true>(acc, a, g);
  hop2_load<P, R, 1, false>(a, g, s, p, h, L, in);
  hop2_compute<P, R, 0, false>(acc, b, g);
  hop2_load<P, R, 2, true>(b, g, s, p, h, L, in);
  hop2_compute<P, R, 1, true>(acc, c, g);
  hop2_load<P, R, 2, false>(c, g, s, p, h, L, in);
  hop2_compute<P, R, 1, false>(acc, a, g);
  hop2_load<P, R, 3, true>(a, g, s, p, h, L, in);
  hop2_compute<P, R, 2, true>(acc, b, g);
  hop2_load<P, R, 3, false>(b, g, s, p, h, L, in);
  hop2_compute<P, R, 2, false>(acc, c, g);
  hop2_compute<P, R, 3, true>(acc, a, g);
  hop2_compute<P, R, 3, false>(acc, b, g);
}

// Sum of the eight hops: acc = sum_mu [U_mu(x)(1-gamma_mu)psi(x+mu) + U_mu(x-mu)^dag (1+gamma_mu) psi(x-mu)].
template <int P, int R>
__device__ __forceinline__ void hopping_sum(Spinor<typename Traits<P>::real>& acc, const Geom& g, const Site& s,
                                            int p, int h, const char* links, const void* in) {
  using T = typename Traits<P>::real;
  if constexpr (P == P64) {
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
  } else {
    Spinor2 a2;
    hopping_sum2<P, R>(a2, g, s, p, h, links, in);
    unpair(acc, a2);
  }
}

}  // namespace nd
