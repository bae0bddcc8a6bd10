// Layout conversion kernels: canonical FP64 or FP32 (lex order, AoS) <-> internal even-odd SoA of
// each precision, link compression to 18 / 12 / 8 reals (Sec. 2.1), and the export of the
// device's site tables for the bit-exact index test.
#include "fields.cuh"
#include "geometry.cuh"
#include "kernels.h"

namespace nd {

constexpr int PACK_THREADS = 256;

int64_t spinor_bytes(int prec, int64_t Vh) {
  switch (prec) {
    case P64: return 2 * Vh * 192;
    case P32: return 2 * Vh * 96;
    case P16: return 2 * Vh * 52;
  }
  return -1;
}

int64_t link_bytes(int prec, int recon, int64_t Vh) {
#define LB(P, R) \
  if (prec == P && recon == R) return link_regions<P, R>(Vh).total;
  LB(P64, 18) LB(P64, 12) LB(P64, 8) LB(P32, 18) LB(P32, 12) LB(P32, 8) LB(P16, 18) LB(P16, 12) LB(P16, 8)
#undef LB
  return -1;
}

template <int P, typename C>
__global__ void pack_spinor_kernel(const Geom g, void* internal, const C* canon) {
  using T = typename Traits<P>::real;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * g.Vh) return;
  const int p = i >= g.Vh ? 1 : 0, h = i - p * g.Vh;
  const Site s = site_of(g, p, h);
  const C* src = canon + (int64_t)s.lex * 24;
  Spinor<T> v;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) v.s[a][c] = mk((T)src[2 * (3 * a + c)], (T)src[2 * (3 * a + c) + 1]);
  SpinorIO<P>::store(v, internal, g.Vh, p, h);
}

template <int P, typename C>
__global__ void unpack_spinor_kernel(const Geom g, C* canon, const void* internal) {
  using T = typename Traits<P>::real;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * g.Vh) return;
  const int p = i >= g.Vh ? 1 : 0, h = i - p * g.Vh;
  const Site s = site_of(g, p, h);
  Spinor<T> v;
  SpinorIO<P>::load(v, internal, g.Vh, p, h);
  C* dst = canon + (int64_t)s.lex * 24;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      dst[2 * (3 * a + c)] = (C)v.s[a][c].re;
      dst[2 * (3 * a + c) + 1] = (C)v.s[a][c].im;
    }
}

// Store R reals of one link into the (P, R) regions.
template <int P, int R>
__device__ __forceinline__ void store_raw(const double (&r)[R], char* base, int64_t Vh, int p, int mu, int64_t h) {
  constexpr int NA = LinkForm<P, R>::NA, NB = LinkForm<P, R>::NB, NC = LinkForm<P, R>::NC;
  const LinkRegions g = link_regions<P, R>(Vh);
  const int64_t pm = (int64_t)(p * 4 + mu);
  if constexpr (P == P64) {
    double2* a = reinterpret_cast<double2*>(base + g.offA) + pm * NA * Vh + h;
#pragma unroll
    for (int k = 0; k < NA; ++k) a[k * Vh] = make_double2(r[2 * k], r[2 * k + 1]);
  } else if constexpr (P == P32) {
    float4* a = reinterpret_cast<float4*>(base + g.offA) + pm * NA * Vh + h;
#pragma unroll
    for (int k = 0; k < NA; ++k)
      a[k * Vh] = make_float4((float)r[4 * k], (float)r[4 * k + 1], (float)r[4 * k + 2], (float)r[4 * k + 3]);
    if constexpr (NB)
      reinterpret_cast<float2*>(base + g.offB)[pm * Vh + h] = make_float2((float)r[4 * NA], (float)r[4 * NA + 1]);
  } else {
    auto h2 = [](double x, double y) {
      __half2 v = __floats2half2_rn((float)x, (float)y);
      return *reinterpret_cast<unsigned*>(&v);
    };
    uint4* a = reinterpret_cast<uint4*>(base + g.offA) + pm * NA * Vh + h;
#pragma unroll
    for (int k = 0; k < NA; ++k)
      a[k * Vh] = make_uint4(h2(r[8 * k], r[8 * k + 1]), h2(r[8 * k + 2], r[8 * k + 3]), h2(r[8 * k + 4], r[8 * k + 5]),
                             h2(r[8 * k + 6], r[8 * k + 7]));
    if constexpr (NB)
      reinterpret_cast<uint2*>(base + g.offB)[pm * Vh + h] =
          make_uint2(h2(r[8 * NA], r[8 * NA + 1]), h2(r[8 * NA + 2], r[8 * NA + 3]));
    if constexpr (NC) reinterpret_cast<unsigned*>(base + g.offC)[pm * Vh + h] = h2(r[8 * NA], r[8 * NA + 1]);
  }
}

// Smallest N = |a2|^2 + |a3|^2 accepted by the 8-real form: below it the rebuild divides by a
// number of the size of the rounding error.
constexpr double RECON8_MIN_N = 1e-10;

template <int P, int R>
__global__ void pack_links_kernel(const Geom g, char* internal, const double* canon, int* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 8 * g.Vh) return;
  const int mu = i & 3;
  const int site = i >> 2;
  const int p = site >= g.Vh ? 1 : 0, h = site - p * g.Vh;
  const Site s = site_of(g, p, h);
  const double* U = canon + ((int64_t)mu * 2 * g.Vh + s.lex) * 18;  // U[row][col][re/im]
  double r[R];
  if constexpr (R == 18) {
#pragma unroll
    for (int k = 0; k < 18; ++k) r[k] = U[k];
  } else if constexpr (R == 12) {
    // columns a = U[.][0], b = U[.][1]
#pragma unroll
    for (int row = 0; row < 3; ++row) {
      r[2 * row] = U[2 * (3 * row + 0)];
      r[2 * row + 1] = U[2 * (3 * row + 0) + 1];
      r[6 + 2 * row] = U[2 * (3 * row + 1)];
      r[6 + 2 * row + 1] = U[2 * (3 * row + 1) + 1];
    }
  } else {
    // a2 = U[1][0], a3 = U[2][0], b1 = U[0][1], arg a1 = arg U[0][0], arg c1 = arg U[0][2]
    r[0] = U[2 * 3];
    r[1] = U[2 * 3 + 1];
    r[2] = U[2 * 6];
    r[3] = U[2 * 6 + 1];
    r[4] = U[2 * 1];
    r[5] = U[2 * 1 + 1];
    r[6] = atan2(U[1], U[0]);
    r[7] = atan2(U[2 * 2 + 1], U[2 * 2]);
    if (P == P16) {
      r[6] *= 0.31830988618379067154;  // 1/pi
      r[7] *= 0.31830988618379067154;
    }
    const double N = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3];
    if (!(N > RECON8_MIN_N)) atomicExch(bad, 1);
  }
  store_raw<P, R>(r, internal, g.Vh, p, mu, h);
}

static int blocks_for(int64_t n) { return (int)((n + PACK_THREADS - 1) / PACK_THREADS); }

template <typename C>
static cudaError_t pack_t(const Geom& g, int prec, void* internal, const C* canon, cudaStream_t st) {
  const int b = blocks_for(2 * (int64_t)g.Vh);
  switch (prec) {
    case P64: pack_spinor_kernel<P64, C><<<b, PACK_THREADS, 0, st>>>(g, internal, canon); break;
    case P32: pack_spinor_kernel<P32, C><<<b, PACK_THREADS, 0, st>>>(g, internal, canon); break;
    case P16: pack_spinor_kernel<P16, C><<<b, PACK_THREADS, 0, st>>>(g, internal, canon); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename C>
static cudaError_t unpack_t(const Geom& g, int prec, C* canon, const void* internal, cudaStream_t st) {
  const int b = blocks_for(2 * (int64_t)g.Vh);
  switch (prec) {
    case P64: unpack_spinor_kernel<P64, C><<<b, PACK_THREADS, 0, st>>>(g, canon, internal); break;
    case P32: unpack_spinor_kernel<P32, C><<<b, PACK_THREADS, 0, st>>>(g, canon, internal); break;
    case P16: unpack_spinor_kernel<P16, C><<<b, PACK_THREADS, 0, st>>>(g, canon, internal); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_pack_spinor(const Geom& g, int prec, void* internal, const double* canon, cudaStream_t st) {
  return pack_t(g, prec, internal, canon, st);
}
cudaError_t launch_unpack_spinor(const Geom& g, int prec, double* canon, const void* internal, cudaStream_t st) {
  return unpack_t(g, prec, canon, internal, st);
}
cudaError_t launch_pack_spinor_f32(const Geom& g, int prec, void* internal, const float* canon, cudaStream_t st) {
  return pack_t(g, prec, internal, canon, st);
}
cudaError_t launch_unpack_spinor_f32(const Geom& g, int prec, float* canon, const void* internal, cudaStream_t st) {
  return unpack_t(g, prec, canon, internal, st);
}

cudaError_t launch_pack_links(const Geom& g, int prec, int recon, void* internal, const double* canon, int* bad,
                              cudaStream_t st) {
  const int b = blocks_for(8 * (int64_t)g.Vh);
  char* dst = static_cast<char*>(internal);
#define PL(P, R)                                                                      \
  if (prec == P && recon == R) {                                                      \
    pack_links_kernel<P, R><<<b, PACK_THREADS, 0, st>>>(g, dst, canon, bad);          \
    return cudaGetLastError();                                                        \
  }
  PL(P64, 18) PL(P64, 12) PL(P64, 8) PL(P32, 18) PL(P32, 12) PL(P32, 8) PL(P16, 18) PL(P16, 12) PL(P16, 8)
#undef PL
  return cudaErrorInvalidValue;
}

template <int MU, bool FWD>
__device__ __forceinline__ void nbr_entry(const Geom& g, const Site& s, int p, int e, int32_t* nbr) {
  bool crossed;
  const int hn = neighbour_h<MU, FWD>(g, s, &crossed);
  nbr[(int64_t)(2 * MU + (FWD ? 0 : 1)) * 2 * g.Vh + e] = (1 - p) * g.Vh + hn;
}

__global__ void eo_tables_kernel(const Geom g, int32_t* lex2eo, int32_t* nbr) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * g.Vh) return;
  const int p = e >= g.Vh ? 1 : 0, h = e - p * g.Vh;
  const Site s = site_of(g, p, h);
  lex2eo[s.lex] = e;
  nbr_entry<0, true>(g, s, p, e, nbr);
  nbr_entry<0, false>(g, s, p, e, nbr);
  nbr_entry<1, true>(g, s, p, e, nbr);
  nbr_entry<1, false>(g, s, p, e, nbr);
  nbr_entry<2, true>(g, s, p, e, nbr);
  nbr_entry<2, false>(g, s, p, e, nbr);
  nbr_entry<3, true>(g, s, p, e, nbr);
  nbr_entry<3, false>(g, s, p, e, nbr);
}

cudaError_t launch_eo_tables(const Geom& g, int32_t* lex2eo, int32_t* nbr, cudaStream_t st) {
  eo_tables_kernel<<<blocks_for(2 * (int64_t)g.Vh), PACK_THREADS, 0, st>>>(g, lex2eo, nbr);
  return cudaGetLastError();
}

}  // namespace nd
