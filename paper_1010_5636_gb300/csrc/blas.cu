// BLAS-1 kernels on whole-lattice internal spinor fields: one thread per site, 128-bit
// coalesced loads and stores through SpinorIO, FP64 deterministic reductions (reduce.cuh).
// FP32/FP16 fields accumulate each site's 24 products in FP32 and convert the site sum to
// FP64 (one FP64 add per site keeps the FP64 pipe, which is narrow on this GPU, out of the way).
#include "fields.cuh"
#include "kernels.h"
#include "reduce.cuh"

namespace nd {

constexpr int B_THREADS = 256;

__device__ __forceinline__ void site_ph(const Geom& g, int i, int* p, int* h) {
  *p = i >= g.Vh ? 1 : 0;
  *h = i - *p * g.Vh;
}

static int nblocks(const Geom& g) { return (blas_sites(g) + B_THREADS - 1) / B_THREADS; }

template <int P, bool REDUCE>
__global__ void __launch_bounds__(B_THREADS) axpby_kernel(const Geom g, void* z, double a, const void* x, double b,
                                                           const void* y, ReduceSlot slot) {
  using T = typename Traits<P>::real;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double red[1] = {0.0};
  if (i < blas_sites(g)) {
    int p, h;
    site_ph(g, i, &p, &h);
    Spinor<T> vx, vy, vz;
    const T ca = (T)a, cb = (T)b;
    if (x) SpinorIO<P>::load(vx, x, g.Vh, p, h);
    if (y) SpinorIO<P>::load(vy, y, g.Vh, p, h);
    T s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        cx<T> v = mk((T)0, (T)0);
        if (x) v = ca * vx.s[k][c];
        if (y) v = v + cb * vy.s[k][c];
        vz.s[k][c] = v;
        s += norm2(v);
      }
    SpinorIO<P>::store(vz, z, g.Vh, p, h);
    red[0] = (double)s;
  }
  if (REDUCE) grid_sum<1>(red, slot);
}

template <int P>
__global__ void __launch_bounds__(B_THREADS) dot_kernel(const Geom g, const void* x, const void* y, ReduceSlot slot) {
  using T = typename Traits<P>::real;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double red[3] = {0.0, 0.0, 0.0};
  if (i < blas_sites(g)) {
    int p, h;
    site_ph(g, i, &p, &h);
    Spinor<T> vx, vy;
    SpinorIO<P>::load(vx, x, g.Vh, p, h);
    SpinorIO<P>::load(vy, y, g.Vh, p, h);
    T re = 0, im = 0, nx = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        cx<T> t = cmulc(vx.s[k][c], vy.s[k][c]);
        re += t.re;
        im += t.im;
        nx += norm2(vx.s[k][c]);
      }
    red[0] = (double)re;
    red[1] = (double)im;
    red[2] = (double)nx;
  }
  grid_sum<3>(red, slot);
}

template <int PO, int PI>
__global__ void __launch_bounds__(B_THREADS) convert_kernel(const Geom g, void* out, const void* in) {
  using TI = typename Traits<PI>::real;
  using TO = typename Traits<PO>::real;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= blas_sites(g)) return;
  int p, h;
  site_ph(g, i, &p, &h);
  Spinor<TI> v;
  SpinorIO<PI>::load(v, in, g.Vh, p, h);
  Spinor<TO> w;
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) w.s[k][c] = mk((TO)v.s[k][c].re, (TO)v.s[k][c].im);
  SpinorIO<PO>::store(w, out, g.Vh, p, h);
}

// out (precision PO) = in (FP64) / sqrt(*norm2); zero when *norm2 is zero
template <int PO>
__global__ void __launch_bounds__(B_THREADS) convert_normalized_kernel(const Geom g, void* out, const void* in,
                                                                        const double* norm2) {
  using TO = typename Traits<PO>::real;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= blas_sites(g)) return;
  int p, h;
  site_ph(g, i, &p, &h);
  const double n2 = *norm2;
  const double sc = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
  Spinor<double> v;
  SpinorIO<P64>::load(v, in, g.Vh, p, h);
  Spinor<TO> w;
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) w.s[k][c] = mk((TO)(sc * v.s[k][c].re), (TO)(sc * v.s[k][c].im));
  SpinorIO<PO>::store(w, out, g.Vh, p, h);
}

// x (FP64) += a e (e FP32)
__global__ void __launch_bounds__(B_THREADS) axpy_widen_kernel(const Geom g, void* x, double a, const void* e) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= blas_sites(g)) return;
  int p, h;
  site_ph(g, i, &p, &h);
  Spinor<double> vx;
  Spinor<float> ve;
  SpinorIO<P64>::load(vx, x, g.Vh, p, h);
  SpinorIO<P32>::load(ve, e, g.Vh, p, h);
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) vx.s[k][c] = vx.s[k][c] + a * mk((double)ve.s[k][c].re, (double)ve.s[k][c].im);
  SpinorIO<P64>::store(vx, x, g.Vh, p, h);
}

__global__ void __launch_bounds__(B_THREADS) g5_axpby_kernel(const Geom g, void* out, double c1, const void* x,
                                                              double c2, const void* y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= blas_sites(g)) return;
  int p, h;
  site_ph(g, i, &p, &h);
  Spinor<double> vx, vy, o;
  SpinorIO<P64>::load(vx, x, g.Vh, p, h);
  SpinorIO<P64>::load(vy, y, g.Vh, p, h);
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) o.s[k][c] = c1 * vx.s[k][c] + (k < 2 ? c2 : -c2) * vy.s[k][c];
  SpinorIO<P64>::store(o, out, g.Vh, p, h);
}

template <int P>
__global__ void __launch_bounds__(B_THREADS) g5_kernel(const Geom g, void* out, const void* in) {
  using T = typename Traits<P>::real;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= blas_sites(g)) return;
  int p, h;
  site_ph(g, i, &p, &h);
  Spinor<T> v;
  SpinorIO<P>::load(v, in, g.Vh, p, h);
#pragma unroll
  for (int k = 2; k < 4; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) v.s[k][c] = -v.s[k][c];
  SpinorIO<P>::store(v, out, g.Vh, p, h);
}

// (v_k, w) for K vectors; each thread reads w once and the K vectors' entries of its site.
template <int K>
__global__ void __launch_bounds__(B_THREADS) multidot_kernel(const Geom g, const char* base, size_t stride,
                                                              const void* w, ReduceSlot slot) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double red[2 * K];
#pragma unroll
  for (int k = 0; k < 2 * K; ++k) red[k] = 0.0;
  if (i < blas_sites(g)) {
    int p, h;
    site_ph(g, i, &p, &h);
    const double2* wb = reinterpret_cast<const double2*>(w) + (int64_t)p * 12 * g.Vh + h;
#pragma unroll 1
    for (int c = 0; c < 12; ++c) {
      const double2 wv = __ldg(wb + c * (int64_t)g.Vh);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const double2 v = __ldg(reinterpret_cast<const double2*>(base + k * stride) + (int64_t)p * 12 * g.Vh + h +
                                c * (int64_t)g.Vh);
        red[2 * k] = fma(v.x, wv.x, fma(v.y, wv.y, red[2 * k]));
        red[2 * k + 1] = fma(v.x, wv.y, fma(-v.y, wv.x, red[2 * k + 1]));
      }
    }
  }
  grid_sum<2 * K>(red, slot);
}

__global__ void __launch_bounds__(B_THREADS) lincomb_kernel(const Geom g, void* out, double beta, const void* y,
                                                             const char* base, size_t stride, int K,
                                                             const double* coef) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= blas_sites(g)) return;
  int p, h;
  site_ph(g, i, &p, &h);
  const int64_t off = (int64_t)p * 12 * g.Vh + h;
#pragma unroll 1
  for (int c = 0; c < 12; ++c) {
    double2 acc = make_double2(0.0, 0.0);
    if (y) {
      const double2 yv = __ldg(reinterpret_cast<const double2*>(y) + off + c * (int64_t)g.Vh);
      acc = make_double2(beta * yv.x, beta * yv.y);
    }
    for (int k = 0; k < K; ++k) {
      const double2 v = __ldg(reinterpret_cast<const double2*>(base + k * stride) + off + c * (int64_t)g.Vh);
      const double cr = __ldg(coef + 2 * k), ci = __ldg(coef + 2 * k + 1);
      acc.x = fma(cr, v.x, fma(-ci, v.y, acc.x));
      acc.y = fma(cr, v.y, fma(ci, v.x, acc.y));
    }
    reinterpret_cast<double2*>(out)[off + c * (int64_t)g.Vh] = acc;
  }
}

template <int P>
static cudaError_t axpby_p(const Geom& g, void* z, double a, const void* x, double b, const void* y, bool reduce,
                           ReduceSlot slot, cudaStream_t st) {
  if (reduce)
    axpby_kernel<P, true><<<nblocks(g), B_THREADS, 0, st>>>(g, z, a, x, b, y, slot);
  else
    axpby_kernel<P, false><<<nblocks(g), B_THREADS, 0, st>>>(g, z, a, x, b, y, slot);
  return cudaGetLastError();
}

cudaError_t blas_axpby(const Geom& g, int prec, void* z, double a, const void* x, double b, const void* y, bool reduce,
                       ReduceSlot slot, cudaStream_t st) {
  switch (prec) {
    case P64: return axpby_p<P64>(g, z, a, x, b, y, reduce, slot, st);
    case P32: return axpby_p<P32>(g, z, a, x, b, y, reduce, slot, st);
    case P16: return axpby_p<P16>(g, z, a, x, b, y, reduce, slot, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t blas_dot(const Geom& g, int prec, const void* x, const void* y, ReduceSlot slot, cudaStream_t st) {
  switch (prec) {
    case P64: dot_kernel<P64><<<nblocks(g), B_THREADS, 0, st>>>(g, x, y, slot); break;
    case P32: dot_kernel<P32><<<nblocks(g), B_THREADS, 0, st>>>(g, x, y, slot); break;
    case P16: dot_kernel<P16><<<nblocks(g), B_THREADS, 0, st>>>(g, x, y, slot); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t blas_convert(const Geom& g, int po, void* out, int pi, const void* in, cudaStream_t st) {
#define CV(A, B)                                                                   \
  if (po == A && pi == B) {                                                        \
    convert_kernel<A, B><<<nblocks(g), B_THREADS, 0, st>>>(g, out, in);            \
    return cudaGetLastError();                                                     \
  }
  CV(P64, P64) CV(P64, P32) CV(P64, P16) CV(P32, P64) CV(P32, P32) CV(P32, P16) CV(P16, P64) CV(P16, P32) CV(P16, P16)
#undef CV
  return cudaErrorInvalidValue;
}

cudaError_t blas_convert_normalized(const Geom& g, int po, void* out, const void* in, const double* norm2,
                                    cudaStream_t st) {
  switch (po) {
    case P32: convert_normalized_kernel<P32><<<nblocks(g), B_THREADS, 0, st>>>(g, out, in, norm2); break;
    case P16: convert_normalized_kernel<P16><<<nblocks(g), B_THREADS, 0, st>>>(g, out, in, norm2); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t blas_axpy_widen(const Geom& g, void* x64, double a, const void* e32, cudaStream_t st) {
  axpy_widen_kernel<<<nblocks(g), B_THREADS, 0, st>>>(g, x64, a, e32);
  return cudaGetLastError();
}

cudaError_t blas_g5_axpby(const Geom& g, void* out, double c1, const void* x, double c2, const void* y,
                          cudaStream_t st) {
  g5_axpby_kernel<<<nblocks(g), B_THREADS, 0, st>>>(g, out, c1, x, c2, y);
  return cudaGetLastError();
}

cudaError_t blas_g5(const Geom& g, int prec, void* out, const void* in, cudaStream_t st) {
  switch (prec) {
    case P64: g5_kernel<P64><<<nblocks(g), B_THREADS, 0, st>>>(g, out, in); break;
    case P32: g5_kernel<P32><<<nblocks(g), B_THREADS, 0, st>>>(g, out, in); break;
    case P16: g5_kernel<P16><<<nblocks(g), B_THREADS, 0, st>>>(g, out, in); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t blas_multidot(const Geom& g, const void* base, size_t stride, int K, const void* w, ReduceSlot slot,
                          cudaStream_t st) {
  // results for chunks of 4 vectors; each chunk writes 8 doubles at slot.result + 8 * chunk
  const char* b = static_cast<const char*>(base);
  for (int k0 = 0; k0 < K; k0 += 4) {
    ReduceSlot s = slot;
    s.result = slot.result + 2 * k0;
    const int kk = K - k0 < 4 ? K - k0 : 4;
    switch (kk) {
      case 4: multidot_kernel<4><<<nblocks(g), B_THREADS, 0, st>>>(g, b + k0 * stride, stride, w, s); break;
      case 3: multidot_kernel<3><<<nblocks(g), B_THREADS, 0, st>>>(g, b + k0 * stride, stride, w, s); break;
      case 2: multidot_kernel<2><<<nblocks(g), B_THREADS, 0, st>>>(g, b + k0 * stride, stride, w, s); break;
      case 1: multidot_kernel<1><<<nblocks(g), B_THREADS, 0, st>>>(g, b + k0 * stride, stride, w, s); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t blas_lincomb(const Geom& g, void* out, double beta, const void* y, const void* base, size_t stride, int K,
                         const double* coef, cudaStream_t st) {
  lincomb_kernel<<<nblocks(g), B_THREADS, 0, st>>>(g, out, beta, y, static_cast<const char*>(base), stride, K, coef);
  return cudaGetLastError();
}

}  // namespace nd

namespace nd {

// Deterministic pseudo-random FP64 field (a start vector for Lanczos): every real is
// (splitmix64(seed, index) mapped to [-1, 1)).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void random_kernel(const Geom g, void* out, uint64_t seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= blas_sites(g)) return;
  double2* o = reinterpret_cast<double2*>(out);
  const int p = i >= g.Vh ? 1 : 0, h = i - p * g.Vh;
  for (int c = 0; c < 12; ++c) {
    const int64_t idx = ((int64_t)p * 12 + c) * g.Vh + h;
    const uint64_t a = splitmix64(seed * 0x100000001B3ull + 2 * (uint64_t)idx);
    const uint64_t b = splitmix64(seed * 0x100000001B3ull + 2 * (uint64_t)idx + 1);
    o[idx] = make_double2((double)(a >> 11) * 0x1.0p-52 - 1.0, (double)(b >> 11) * 0x1.0p-52 - 1.0);
  }
}

cudaError_t blas_random(const Geom& g, void* out, uint64_t seed, cudaStream_t st) {
  random_kernel<<<nblocks(g), B_THREADS, 0, st>>>(g, out, seed);
  return cudaGetLastError();
}

}  // namespace nd
