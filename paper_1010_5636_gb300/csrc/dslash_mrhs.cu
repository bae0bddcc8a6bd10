// Q = gamma5 D_W (Sec. 2.1) on several right-hand sides with K of them per thread: each hop's link
// is read and rebuilt in registers once and applied to the K neighbour spinors, so the link load and
// the SU(3) reconstruction are shared by K right-hand sides, and each thread has K independent
// neighbour loads in flight per hop.  Blocks with consecutive indices take the same 64 sites for
// successive groups of K right-hand sides, so a tile of links also serves the other groups from L2.
// The per-RHS arithmetic is the one of q_kernel (packed spin-row pairs), term for term in the same order.
#include "dslash.cuh"
#include "kernels.h"

namespace nd {

constexpr int MR_THREADS = 64;
constexpr int MR_MIN_BLOCKS = 6;

template <int P, int R, int MU, bool FWD, int K>
__device__ __forceinline__ void hop_k(Spinor2 (&acc)[K], const Geom& g, const Site& s, int p, int h,
                                      const char* links, const char* in, int64_t stride, int kk) {
  bool crossed;
  const int hn = neighbour_h<MU, FWD>(g, s, &crossed);
  Spinor2 nb[K];
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (k < kk) SpinorIO<P>::load2(nb[k], in + k * stride, g.Vh, 1 - p, hn);
  LinkRaw<P, R> raw;
  if (FWD)
    load_raw<P, R>(raw, links, g.Vh, p, MU, h);
  else
    load_raw<P, R>(raw, links, g.Vh, 1 - p, MU, hn);
  Su3<float> U;
  reconstruct<P, R>(U, raw);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (k >= kk) continue;
    float2 hr[3], hi[3], cr[3], ci[3];
    spin_project2<MU, FWD>(nb[k], hr, hi);
    if (g.apbc && crossed) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        hr[i] = f2_neg(hr[i]);
        hi[i] = f2_neg(hi[i]);
      }
    }
    colour_mul2<!FWD>(U, hr, hi, cr, ci);
    spin_accumulate2<MU, FWD>(acc[k], cr, ci);
  }
}

// out_r = gamma5 (diag in_r - 1/2 hop(in_r)) for r < nrhs (fields at + r * stride bytes), output sites
// of both parities (nsites = 2 Vh, parity alternating by warp as in q_kernel) or of parity0 only (nsites = Vh).
template <int P, int R, int K>
__global__ void __launch_bounds__(MR_THREADS, MR_MIN_BLOCKS)
    q_mrhs_kernel(const Geom g, const char* links, const char* in, char* out, int64_t stride, int nrhs, int nsites,
                  int parity0, double diag) {
  using T = typename Traits<P>::real;
  const int groups = (nrhs + K - 1) / K;
  const int grp = blockIdx.x % groups, blk = blockIdx.x / groups;
  const int r0 = grp * K;
  const int kk = min(K, nrhs - r0);
  const int i = blk * MR_THREADS + threadIdx.x;
  int p = parity0, h = i;
  if (nsites == 2 * g.Vh)
    both_parities_site(i, &p, &h);
  if (h >= g.Vh) return;
  const Site s = site_of(g, p, h);
  const char* in0 = in + r0 * stride;
  char* out0 = out + r0 * stride;
  Spinor2 acc2[K];
#pragma unroll
  for (int k = 0; k < K; ++k) zero2(acc2[k]);
  hop_k<P, R, 0, true, K>(acc2, g, s, p, h, links, in0, stride, kk);
  hop_k<P, R, 0, false, K>(acc2, g, s, p, h, links, in0, stride, kk);
  hop_k<P, R, 1, true, K>(acc2, g, s, p, h, links, in0, stride, kk);
  hop_k<P, R, 1, false, K>(acc2, g, s, p, h, links, in0, stride, kk);
  hop_k<P, R, 2, true, K>(acc2, g, s, p, h, links, in0, stride, kk);
  hop_k<P, R, 2, false, K>(acc2, g, s, p, h, links, in0, stride, kk);
  hop_k<P, R, 3, true, K>(acc2, g, s, p, h, links, in0, stride, kk);
  hop_k<P, R, 3, false, K>(acc2, g, s, p, h, links, in0, stride, kk);
  const T dg = (T)diag;
  const bool read_diag = diag != 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (k >= kk) continue;
    Spinor<T> d, res, acck;
    unpair(acck, acc2[k]);
    if (read_diag) SpinorIO<P>::load(d, in0 + k * stride, g.Vh, p, h);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        cx<T> v = (T)(-0.5) * acck.s[a][c];
        if (read_diag) v = v + dg * d.s[a][c];
        res.s[a][c] = a < 2 ? v : -v;
      }
    SpinorIO<P>::store(res, out0 + k * stride, g.Vh, p, h);
  }
}

template <int P, int R>
static cudaError_t launch_mr2(const Geom& g, const QLaunch& L, cudaStream_t st) {
  const int blocks = (L.nsites + MR_THREADS - 1) / MR_THREADS;
  const char* lk = static_cast<const char*>(L.links);
  const char* in = static_cast<const char*>(L.in);
  char* out = static_cast<char*>(L.out);
  switch (L.krhs) {
    case 2:
      q_mrhs_kernel<P, R, 2><<<blocks * ((L.nrhs + 1) / 2), MR_THREADS, 0, st>>>(g, lk, in, out, L.rhs_stride, L.nrhs,
                                                                            L.nsites, L.parity0, L.diag);
      break;
    case 3:
      q_mrhs_kernel<P, R, 3><<<blocks * ((L.nrhs + 2) / 3), MR_THREADS, 0, st>>>(g, lk, in, out, L.rhs_stride, L.nrhs,
                                                                            L.nsites, L.parity0, L.diag);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int P>
static cudaError_t launch_mr1(const Geom& g, const QLaunch& L, cudaStream_t st) {
  switch (L.recon) {
    case 18: return launch_mr2<P, 18>(g, L, st);
    case 12: return launch_mr2<P, 12>(g, L, st);
    case 8: return launch_mr2<P, 8>(g, L, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_q_mrhs_k(const Geom& g, const QLaunch& L, cudaStream_t st) {
  if (L.mode != Q_MRHS || L.reduce || L.y || L.a != 1.0 || L.no_g5 || L.din) return cudaErrorInvalidValue;
  switch (L.prec) {
    case P32: return launch_mr1<P32>(g, L, st);
    case P16: return launch_mr1<P16>(g, L, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nd
