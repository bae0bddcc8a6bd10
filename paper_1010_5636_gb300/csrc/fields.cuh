// Device-side field types of libnd: complex arithmetic, precision traits, the even-odd
// structure-of-arrays spinor and link layouts, and in-register SU(3) reconstruction.
//
// Internal spinor layout (one full lattice, even-odd ordered, parity blocks contiguous):
//   site i = p*Vh + h  (p = parity, h = floor(lex/2));  24 reals per site in canonical order
//   (spin-major, colour, re/im) split into 16-byte chunks:
//     FP64: 12 chunks of double2;  FP32: 6 chunks of float4;  FP16: 3 chunks of 8 halves.
//   chunk c of site (p, h) lives at index (p*NC + c)*Vh + h, so consecutive threads (consecutive h)
//   read consecutive 16-byte words: every load is a coalesced 128-bit access.
//   FP64 chunks hold the 12 complex components in canonical order.  FP32 and FP16 hold them in
//   spin-row pairs, the operands of packed FP32 (f32x2) arithmetic: for colour i the pairs
//   (s0.re, s1.re), (s0.im, s1.im) of the upper spins and (s2.re, s3.re), (s2.im, s3.im) of the
//   lower spins.  FP32 chunk i < 3 = [(s0.re, s1.re), (s0.im, s1.im)] of colour i, chunk 3 + i the
//   lower spins of colour i; FP16 stores the same 12 pairs in that order, four per chunk.
//   FP16 fields carry one FP32 scale per site after the chunks (index p*Vh + h); the stored
//   halves are value/scale with scale = max |component| of the site.
// Internal link layout, for parity p and direction mu (U_mu(x) for x of parity p):
//   region A: (p*4 + mu)*NA + k chunks of 16 bytes (k < NA), stride Vh;
//   region B: one 8-byte word per link (p*4 + mu)*Vh + h, if the form needs it;
//   region C: one 4-byte word per link, if the form needs it.
//   18 reals: row-major U (a1 b1 c1 / a2 b2 c2 / a3 b3 c3 with columns a, b, c);
//   12 reals: a1 a2 a3 b1 b2 b3 (columns a, b; c = (a x b)^* rebuilt, Sec. 2.1);
//    8 reals: a2 a3 b1 (complex), arg a1, arg c1 (FP16 stores the angles divided by pi).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace nd {

template <typename T>
struct cx {
  T re, im;
};

template <typename T>
__device__ __forceinline__ cx<T> mk(T r, T i) {
  cx<T> z;
  z.re = r;
  z.im = i;
  return z;
}
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a) { return mk(-a.re, -a.im); }
template <typename T>
__device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
__device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return mk(s * a.re, s * a.im); }
template <typename T>
__device__ __forceinline__ cx<T> conj(cx<T> a) { return mk(a.re, -a.im); }
// i * a
template <typename T>
__device__ __forceinline__ cx<T> itimes(cx<T> a) { return mk(-a.im, a.re); }
// conj(a) * b
template <typename T>
__device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {
  return mk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
// acc += a * b
template <typename T>
__device__ __forceinline__ void cfma(cx<T>& acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename T>
__device__ __forceinline__ void cfmac(cx<T>& acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}
template <typename T>
__device__ __forceinline__ T norm2(cx<T> a) { return a.re * a.re + a.im * a.im; }

// ------------------------------------------------------------------ precision traits
enum Prec { P64 = 0, P32 = 1, P16 = 2 };

template <int P>
struct Traits;
template <>
struct Traits<P64> {
  using real = double;
  static constexpr int SP_CHUNKS = 12;
  static constexpr int SITE_BYTES = 192;
};
template <>
struct Traits<P32> {
  using real = float;
  static constexpr int SP_CHUNKS = 6;
  static constexpr int SITE_BYTES = 96;
};
template <>
struct Traits<P16> {
  using real = float;
  static constexpr int SP_CHUNKS = 3;
  static constexpr int SITE_BYTES = 52;  // 48 bytes of halves + 4-byte scale
};

// A spinor in registers: 4 spins x 3 colours.
template <typename T>
struct Spinor {
  cx<T> s[4][3];
};

// The same spinor as spin-row pairs for packed FP32 arithmetic: ur[i] = (s0[i].re, s1[i].re),
// ui[i] = (s0[i].im, s1[i].im), dr[i] = (s2[i].re, s3[i].re), di[i] = (s2[i].im, s3[i].im).
struct Spinor2 {
  float2 ur[3], ui[3], dr[3], di[3];
};

__device__ __forceinline__ void unpair(Spinor<float>& v, const Spinor2& w) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    v.s[0][i] = mk(w.ur[i].x, w.ui[i].x);
    v.s[1][i] = mk(w.ur[i].y, w.ui[i].y);
    v.s[2][i] = mk(w.dr[i].x, w.di[i].x);
    v.s[3][i] = mk(w.dr[i].y, w.di[i].y);
  }
}
__device__ __forceinline__ void pair(Spinor2& w, const Spinor<float>& v) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    w.ur[i] = make_float2(v.s[0][i].re, v.s[1][i].re);
    w.ui[i] = make_float2(v.s[0][i].im, v.s[1][i].im);
    w.dr[i] = make_float2(v.s[2][i].re, v.s[3][i].re);
    w.di[i] = make_float2(v.s[2][i].im, v.s[3][i].im);
  }
}

// ------------------------------------------------------------------ spinor access
template <int P>
struct SpinorIO;

template <>
struct SpinorIO<P64> {
  using T = double;
  __device__ __forceinline__ static void load(Spinor<T>& v, const void* base, int64_t Vh, int p, int64_t h) {
    const double2* b = reinterpret_cast<const double2*>(base) + (int64_t)p * 12 * Vh + h;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      double2 w = __ldg(b + c * Vh);
      v.s[c / 3][c % 3] = mk(w.x, w.y);
    }
  }
  __device__ __forceinline__ static void store(const Spinor<T>& v, void* base, int64_t Vh, int p, int64_t h,
                                               int part = 0, int nparts = 1) {
    double2* b = reinterpret_cast<double2*>(base) + (int64_t)p * 12 * Vh + h;
#pragma unroll
    for (int c = 0; c < 12; ++c)
      if (c % nparts == part) b[c * Vh] = make_double2(v.s[c / 3][c % 3].re, v.s[c / 3][c % 3].im);
  }
  // components (spin, colour) stored by chunk-part `part` of `nparts`
  __device__ __forceinline__ static bool owns(int a, int c, int part, int nparts) {
    return (3 * a + c) % nparts == part;
  }
};

template <>
struct SpinorIO<P32> {
  using T = float;
  __device__ __forceinline__ static void load2(Spinor2& v, const void* base, int64_t Vh, int p, int64_t h) {
    const float4* b = reinterpret_cast<const float4*>(base) + (int64_t)p * 6 * Vh + h;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float4 u = __ldg(b + i * Vh), d = __ldg(b + (3 + i) * Vh);
      v.ur[i] = make_float2(u.x, u.y);
      v.ui[i] = make_float2(u.z, u.w);
      v.dr[i] = make_float2(d.x, d.y);
      v.di[i] = make_float2(d.z, d.w);
    }
  }
  __device__ __forceinline__ static void load(Spinor<T>& v, const void* base, int64_t Vh, int p, int64_t h) {
    Spinor2 w;
    load2(w, base, Vh, p, h);
    unpair(v, w);
  }
  // chunks c with c % nparts == part
  __device__ __forceinline__ static void store2(const Spinor2& v, void* base, int64_t Vh, int p, int64_t h,
                                                int part = 0, int nparts = 1) {
    float4* b = reinterpret_cast<float4*>(base) + (int64_t)p * 6 * Vh + h;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (i % nparts == part) b[i * Vh] = make_float4(v.ur[i].x, v.ur[i].y, v.ui[i].x, v.ui[i].y);
      if ((3 + i) % nparts == part) b[(3 + i) * Vh] = make_float4(v.dr[i].x, v.dr[i].y, v.di[i].x, v.di[i].y);
    }
  }
  __device__ __forceinline__ static void store(const Spinor<T>& v, void* base, int64_t Vh, int p, int64_t h,
                                               int part = 0, int nparts = 1) {
    Spinor2 w;
    pair(w, v);
    store2(w, base, Vh, p, h, part, nparts);
  }
  __device__ __forceinline__ static bool owns(int a, int c, int part, int nparts) {
    return (a < 2 ? c : 3 + c) % nparts == part;
  }
};

template <>
struct SpinorIO<P16> {
  using T = float;
  // the 12 spin-row pairs in storage order: ur0 ui0 ur1 ui1 | ur2 ui2 dr0 di0 | dr1 di1 dr2 di2
  __device__ __forceinline__ static float2& slot(Spinor2& v, int k) {
    const int i = k >> 1;
    return i < 3 ? ((k & 1) ? v.ui[i] : v.ur[i]) : ((k & 1) ? v.di[i - 3] : v.dr[i - 3]);
  }
  __device__ __forceinline__ static const float2& slot(const Spinor2& v, int k) {
    const int i = k >> 1;
    return i < 3 ? ((k & 1) ? v.ui[i] : v.ur[i]) : ((k & 1) ? v.di[i - 3] : v.dr[i - 3]);
  }
  __device__ __forceinline__ static void load2(Spinor2& v, const void* base, int64_t Vh, int p, int64_t h) {
    const uint4* b = reinterpret_cast<const uint4*>(base) + (int64_t)p * 3 * Vh + h;
    const float* sc = reinterpret_cast<const float*>(reinterpret_cast<const uint4*>(base) + 6 * Vh);
    const float s = __ldg(sc + (int64_t)p * Vh + h);
    const float2 ss = make_float2(s, s);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const uint4 w = __ldg(b + c * Vh);
      const unsigned u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        __half2 hh = *reinterpret_cast<const __half2*>(&u[j]);
        slot(v, 4 * c + j) = __fmul2_rn(__half22float2(hh), ss);
      }
    }
  }
  __device__ __forceinline__ static void load(Spinor<T>& v, const void* base, int64_t Vh, int p, int64_t h) {
    Spinor2 w;
    load2(w, base, Vh, p, h);
    unpair(v, w);
  }
  __device__ __forceinline__ static void store2(const Spinor2& v, void* base, int64_t Vh, int p, int64_t h,
                                                int part = 0, int nparts = 1) {
    uint4* b = reinterpret_cast<uint4*>(base) + (int64_t)p * 3 * Vh + h;
    float* sc = reinterpret_cast<float*>(reinterpret_cast<uint4*>(base) + 6 * Vh);
    float mx = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const float2 f = slot(v, k);
      mx = fmaxf(mx, fmaxf(fabsf(f.x), fabsf(f.y)));
    }
    const float inv = mx > 0.f ? 1.0f / mx : 0.f;
    const float2 ii = make_float2(inv, inv);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (c % nparts != part) continue;
      unsigned u[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 f = __fmul2_rn(slot(v, 4 * c + j), ii);
        __half2 hh = __floats2half2_rn(f.x, f.y);
        u[j] = *reinterpret_cast<unsigned*>(&hh);
      }
      b[c * Vh] = make_uint4(u[0], u[1], u[2], u[3]);
    }
    if (part == 0) sc[(int64_t)p * Vh + h] = mx;
  }
  __device__ __forceinline__ static void store(const Spinor<T>& v, void* base, int64_t Vh, int p, int64_t h,
                                               int part = 0, int nparts = 1) {
    Spinor2 w;
    pair(w, v);
    store2(w, base, Vh, p, h, part, nparts);
  }
  // pair k of component (a, c): spins 0, 1 -> 2c (re) and 2c + 1 (im); spins 2, 3 -> 6 + 2c ...
  __device__ __forceinline__ static bool owns(int a, int c, int part, int nparts) {
    return (((a < 2 ? 0 : 6) + 2 * c) / 4) % nparts == part;
  }
};

// ------------------------------------------------------------------ links
template <typename T>
struct Su3 {
  cx<T> e[3][3];  // e[row][col]
};

// Storage geometry of one (precision, reconstruction) link form.
template <int P, int R>
struct LinkForm;
// FP64
template <>
struct LinkForm<P64, 18> { static constexpr int NA = 9, NB = 0, NC = 0; };
template <>
struct LinkForm<P64, 12> { static constexpr int NA = 6, NB = 0, NC = 0; };
template <>
struct LinkForm<P64, 8> { static constexpr int NA = 4, NB = 0, NC = 0; };
// FP32
template <>
struct LinkForm<P32, 18> { static constexpr int NA = 4, NB = 1, NC = 0; };
template <>
struct LinkForm<P32, 12> { static constexpr int NA = 3, NB = 0, NC = 0; };
template <>
struct LinkForm<P32, 8> { static constexpr int NA = 2, NB = 0, NC = 0; };
// FP16
template <>
struct LinkForm<P16, 18> { static constexpr int NA = 2, NB = 0, NC = 1; };
template <>
struct LinkForm<P16, 12> { static constexpr int NA = 1, NB = 1, NC = 0; };
template <>
struct LinkForm<P16, 8> { static constexpr int NA = 1, NB = 0, NC = 0; };

// Byte offsets of the three regions for a lattice of Vh sites per parity.
struct LinkRegions {
  int64_t offA, offB, offC, total;
};
template <int P, int R>
__host__ __device__ inline LinkRegions link_regions(int64_t Vh) {
  LinkRegions g;
  g.offA = 0;
  g.offB = g.offA + (int64_t)8 * LinkForm<P, R>::NA * Vh * 16;
  g.offC = g.offB + (int64_t)8 * LinkForm<P, R>::NB * Vh * 8;
  g.total = g.offC + (int64_t)8 * LinkForm<P, R>::NC * Vh * 4;
  return g;
}

// Raw reals of one link (R of them), read from the SoA regions.
template <int P, int R>
struct LinkRaw {
  using T = typename Traits<P>::real;
  T r[R];
};

template <int P, int R>
__device__ __forceinline__ void load_raw(LinkRaw<P, R>& L, const char* base, int64_t Vh, int p, int mu,
                                         int64_t h) {
  constexpr int NA = LinkForm<P, R>::NA, NB = LinkForm<P, R>::NB, NC = LinkForm<P, R>::NC;
  const LinkRegions g = link_regions<P, R>(Vh);
  const int64_t pm = (int64_t)(p * 4 + mu);
  if constexpr (P == P64) {
    const double2* a = reinterpret_cast<const double2*>(base + g.offA) + pm * NA * Vh + h;
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      double2 w = __ldg(a + k * Vh);
      L.r[2 * k] = w.x;
      L.r[2 * k + 1] = w.y;
    }
  } else if constexpr (P == P32) {
    const float4* a = reinterpret_cast<const float4*>(base + g.offA) + pm * NA * Vh + h;
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      float4 w = __ldg(a + k * Vh);
      L.r[4 * k] = w.x;
      L.r[4 * k + 1] = w.y;
      L.r[4 * k + 2] = w.z;
      L.r[4 * k + 3] = w.w;
    }
    if constexpr (NB) {
      float2 w = __ldg(reinterpret_cast<const float2*>(base + g.offB) + pm * Vh + h);
      L.r[4 * NA] = w.x;
      L.r[4 * NA + 1] = w.y;
    }
  } else {
    const uint4* a = reinterpret_cast<const uint4*>(base + g.offA) + pm * NA * Vh + h;
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      uint4 w = __ldg(a + k * Vh);
      unsigned u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float2 f = __half22float2(*reinterpret_cast<__half2*>(&u[j]));
        L.r[8 * k + 2 * j] = f.x;
        L.r[8 * k + 2 * j + 1] = f.y;
      }
    }
    if constexpr (NB) {
      uint2 w = __ldg(reinterpret_cast<const uint2*>(base + g.offB) + pm * Vh + h);
      unsigned u[2] = {w.x, w.y};
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        float2 f = __half22float2(*reinterpret_cast<__half2*>(&u[j]));
        L.r[8 * NA + 2 * j] = f.x;
        L.r[8 * NA + 2 * j + 1] = f.y;
      }
    }
    if constexpr (NC) {
      unsigned w = __ldg(reinterpret_cast<const unsigned*>(base + g.offC) + pm * Vh + h);
      float2 f = __half22float2(*reinterpret_cast<__half2*>(&w));
      L.r[8 * NA] = f.x;
      L.r[8 * NA + 1] = f.y;
    }
  }
}

template <typename T>
__device__ __forceinline__ T dev_sqrt(T x);
template <>
__device__ __forceinline__ double dev_sqrt<double>(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float dev_sqrt<float>(float x) { return sqrtf(x); }

template <typename T>
__device__ __forceinline__ void dev_sincos(T x, T* s, T* c);
template <>
__device__ __forceinline__ void dev_sincos<double>(double x, double* s, double* c) { sincos(x, s, c); }
template <>
__device__ __forceinline__ void dev_sincos<float>(float x, float* s, float* c) { sincosf(x, s, c); }

// Rebuild the full SU(3) matrix in registers from the stored reals.
template <int P, int R>
__device__ __forceinline__ void reconstruct(Su3<typename Traits<P>::real>& U, const LinkRaw<P, R>& L) {
  using T = typename Traits<P>::real;
  if constexpr (R == 18) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) U.e[i][j] = mk(L.r[2 * (3 * i + j)], L.r[2 * (3 * i + j) + 1]);
  } else if constexpr (R == 12) {
    cx<T> a1 = mk(L.r[0], L.r[1]), a2 = mk(L.r[2], L.r[3]), a3 = mk(L.r[4], L.r[5]);
    cx<T> b1 = mk(L.r[6], L.r[7]), b2 = mk(L.r[8], L.r[9]), b3 = mk(L.r[10], L.r[11]);
    U.e[0][0] = a1; U.e[1][0] = a2; U.e[2][0] = a3;
    U.e[0][1] = b1; U.e[1][1] = b2; U.e[2][1] = b3;
    // c = (a x b)^*
    U.e[0][2] = conj(a2 * b3 - a3 * b2);
    U.e[1][2] = conj(a3 * b1 - a1 * b3);
    U.e[2][2] = conj(a1 * b2 - a2 * b1);
  } else {
    // 8 reals: a2, a3, b1, theta_a1 = arg a1, theta_c1 = arg c1.
    // |a1|^2 = 1 - |a2|^2 - |a3|^2 (unit column a); |c1|^2 = 1 - |a1|^2 - |b1|^2 (unit row 1).
    // b2, b3 solve  a2 b3 - a3 b2 = c1^*  (first component of c = (a x b)^*) and
    //               a1^* b1 + a2^* b2 + a3^* b3 = 0  (columns a, b orthogonal):
    //   b2 = -(a3^* c1^* + a1^* a2 b1) / N,  b3 = (a2^* c1^* - a1^* a3 b1) / N,  N = |a2|^2 + |a3|^2;
    // then c2, c3 from c = (a x b)^*.
    cx<T> a2 = mk(L.r[0], L.r[1]), a3 = mk(L.r[2], L.r[3]), b1 = mk(L.r[4], L.r[5]);
    T th_a = L.r[6], th_c = L.r[7];
    if constexpr (P == P16) {
      th_a *= (T)3.14159265358979323846;
      th_c *= (T)3.14159265358979323846;
    }
    T N = norm2(a2) + norm2(a3);
    T a1m = dev_sqrt(fmax((T)0, (T)1 - N));
    T c1m = dev_sqrt(fmax((T)0, N - norm2(b1)));
    T sa, ca, sc, cc;
    dev_sincos(th_a, &sa, &ca);
    dev_sincos(th_c, &sc, &cc);
    cx<T> a1 = mk(a1m * ca, a1m * sa);
    cx<T> c1 = mk(c1m * cc, c1m * sc);
    T invN = (T)1 / N;
    cx<T> a1c_b1 = cmulc(a1, b1);  // a1^* b1
    cx<T> b2 = (-invN) * (cmulc(a3, conj(c1)) + a2 * a1c_b1);
    cx<T> b3 = invN * (cmulc(a2, conj(c1)) - a3 * a1c_b1);
    U.e[0][0] = a1; U.e[1][0] = a2; U.e[2][0] = a3;
    U.e[0][1] = b1; U.e[1][1] = b2; U.e[2][1] = b3;
    U.e[0][2] = c1;
    U.e[1][2] = conj(a3 * b1 - a1 * b3);
    U.e[2][2] = conj(a1 * b2 - a2 * b1);
  }
}

}  // namespace nd
