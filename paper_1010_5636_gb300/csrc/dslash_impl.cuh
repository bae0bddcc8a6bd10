// Kernels applying Q = gamma5 D_W (Sec. 2.1) on the even-odd ordered lattice.
//
// Work split: each output site is handled by SPLIT warps-parts (SPLIT = 1, 2 or 4); part k
// computes the hops of directions mu with mu % SPLIT == k (forward and backward) for 32
// consecutive sites.  Parts are whole warps, so no branch diverges inside a warp; the partial
// accumulators are summed through shared memory in a fixed order, so every part holds the
// identical full sum.  Part k then stores the output chunks it owns (chunk c with
// c % SPLIT == k).  Splitting lowers registers per thread and multiplies the number of
// independent loads in flight per SM, which is what a bandwidth-bound stencil needs.
// Epilogue: gamma5 and the diagonal (4+m) fused; optional y-term, fused FP64 norms, and the
// fused CG residual update of the multi-shift solver.
#pragma once
#include <algorithm>
#include "dslash.cuh"
#include "kernels.h"
#include "reduce.cuh"

namespace nd {

constexpr int Q_THREADS = 256;

template <int P, int R, int SPLIT>
__device__ __forceinline__ void hopping_part(Spinor<typename Traits<P>::real>& acc, const Geom& g, const Site& s,
                                             int p, int h, const char* links, const void* in, int part) {
  using T = typename Traits<P>::real;
  if constexpr (SPLIT == 1) {
    hopping_sum<P, R>(acc, g, s, p, h, links, in);
    return;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) acc.s[a][i] = mk((T)0, (T)0);
  if (SPLIT == 1 || part == 0 || (SPLIT == 2 && part == 0)) {
    hop<P, R, 0, true>(acc, g, s, p, h, links, in);
    hop<P, R, 0, false>(acc, g, s, p, h, links, in);
  }
  if (SPLIT == 1 || (SPLIT == 2 && part == 1) || (SPLIT == 4 && part == 1)) {
    hop<P, R, 1, true>(acc, g, s, p, h, links, in);
    hop<P, R, 1, false>(acc, g, s, p, h, links, in);
  }
  if (SPLIT == 1 || (SPLIT == 2 && part == 0) || (SPLIT == 4 && part == 2)) {
    hop<P, R, 2, true>(acc, g, s, p, h, links, in);
    hop<P, R, 2, false>(acc, g, s, p, h, links, in);
  }
  if (SPLIT == 1 || (SPLIT == 2 && part == 1) || (SPLIT == 4 && part == 3)) {
    hop<P, R, 3, true>(acc, g, s, p, h, links, in);
    hop<P, R, 3, false>(acc, g, s, p, h, links, in);
  }
}

// Epilogue of the FP32 / FP16 operator on spin-row pairs, specialised at compile time on whether
// the diagonal term (RD) and the y term (HY) are present: the same operations as the scalar
// epilogue below, each on a pair (s0, s1) or (s2, s3) in one f32x2 instruction.  The runtime
// choice between the four forms is taken once per thread, outside the unrolled loops (branches on
// these flags inside the per-component loop measured 40 % slower).
template <int P, int BASE, bool REDUCE, bool RD, bool HY>
__device__ __forceinline__ void pairs_tail(const Geom& g, const QLaunch& A, Spinor2& v, int p, int h,
                                           double (&red)[2]) {
  const double a_d = BASE == Q_CGUPDATE ? A.cgs[CG_ASCALE] : A.a;
  const double b_d = BASE == Q_CGUPDATE ? A.cgs[CG_SIGMA0] : A.b;
  const float ca = (float)a_d;
  const float2 mh = f2_bcast(-0.5f), dg = f2_bcast((float)A.diag), cb = f2_bcast((float)b_d);
  const float2 cu = f2_bcast(ca), cl = f2_bcast(A.no_g5 ? ca : -ca);
  // the vectors are folded in one at a time, so at most two spinors are live
  float2 s1 = f2_bcast(0.f);
  {
    Spinor2 d;
    if (RD) SpinorIO<P>::load2(d, A.din ? A.din : A.in, g.Vh, p, h);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v.ur[c] = __fmul2_rn(mh, v.ur[c]);
      v.ui[c] = __fmul2_rn(mh, v.ui[c]);
      v.dr[c] = __fmul2_rn(mh, v.dr[c]);
      v.di[c] = __fmul2_rn(mh, v.di[c]);
      if (RD) {
        v.ur[c] = f2_fma(dg, d.ur[c], v.ur[c]);
        v.ui[c] = f2_fma(dg, d.ui[c], v.ui[c]);
        v.dr[c] = f2_fma(dg, d.dr[c], v.dr[c]);
        v.di[c] = f2_fma(dg, d.di[c], v.di[c]);
        if (REDUCE && BASE != Q_CGUPDATE) {  // the CG update's second result is not used
          s1 = f2_fma(d.ur[c], d.ur[c], s1);
          s1 = f2_fma(d.ui[c], d.ui[c], s1);
          s1 = f2_fma(d.dr[c], d.dr[c], s1);
          s1 = f2_fma(d.di[c], d.di[c], s1);
        }
      }
      v.ur[c] = __fmul2_rn(cu, v.ur[c]);
      v.ui[c] = __fmul2_rn(cu, v.ui[c]);
      v.dr[c] = __fmul2_rn(cl, v.dr[c]);
      v.di[c] = __fmul2_rn(cl, v.di[c]);
    }
  }
  // v += coef * x for one more input field x
  auto fold = [&](const void* src, float2 coef) {
    Spinor2 x;
    SpinorIO<P>::load2(x, src, g.Vh, p, h);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v.ur[c] = f2_fma(coef, x.ur[c], v.ur[c]);
      v.ui[c] = f2_fma(coef, x.ui[c], v.ui[c]);
      v.dr[c] = f2_fma(coef, x.dr[c], v.dr[c]);
      v.di[c] = f2_fma(coef, x.di[c], v.di[c]);
    }
  };
  if (HY) fold(A.y, cb);
  if (BASE == Q_XPAY2 || BASE == Q_XPAY3) fold(A.z, f2_bcast((float)A.c));
  if (BASE == Q_XPAY3) fold(A.w, f2_bcast((float)A.d));
  if (BASE == Q_CGUPDATE) {
    // out = out - alpha (v + b y), in place
    const float2 nal = f2_bcast(-(float)(A.cgs[CG_RR] / (a_d * A.cgs[CG_TT] + b_d * A.cgs[CG_PP])));
    Spinor2 z;
    SpinorIO<P>::load2(z, A.out, g.Vh, p, h);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v.ur[c] = f2_fma(nal, v.ur[c], z.ur[c]);
      v.ui[c] = f2_fma(nal, v.ui[c], z.ui[c]);
      v.dr[c] = f2_fma(nal, v.dr[c], z.dr[c]);
      v.di[c] = f2_fma(nal, v.di[c], z.di[c]);
    }
  }
  SpinorIO<P>::store2(v, A.out, g.Vh, p, h);
  if (REDUCE) {
    float2 s0 = f2_bcast(0.f);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      s0 = f2_fma(v.ur[c], v.ur[c], s0);
      s0 = f2_fma(v.ui[c], v.ui[c], s0);
      s0 = f2_fma(v.dr[c], v.dr[c], s0);
      s0 = f2_fma(v.di[c], v.di[c], s0);
    }
    red[0] = (double)s0.x + (double)s0.y;
    red[1] = (double)s1.x + (double)s1.y;
  }
}

// The FP32 / FP16 operator of one thread on spin-row pairs (one warp per site, SPLIT == 1).
template <int P, int R, int MODE, bool REDUCE>
__device__ __forceinline__ void q_site_pairs(const Geom& g, const QLaunch& A, const ReduceSlot& slot, int blk,
                                             int nblk, bool act, int p, int h) {
  constexpr int BASE = (MODE == Q_MRHS || MODE == Q_BPLAIN) ? Q_PLAIN : (MODE == Q_BCG ? Q_CGUPDATE : MODE);
  if (!REDUCE && !act) return;
  double red[2] = {0.0, 0.0};
  if (act) {
    const Site s = site_of(g, p, h);
    Spinor2 acc;
    hopping_sum2<P, R>(acc, g, s, p, h, static_cast<const char*>(A.links), A.in);
    const bool rd = REDUCE || A.diag != 0.0;
    if constexpr (BASE != Q_PLAIN) {
      if (rd)
        pairs_tail<P, BASE, REDUCE, true, true>(g, A, acc, p, h, red);
      else
        pairs_tail<P, BASE, REDUCE, false, true>(g, A, acc, p, h, red);
    } else if constexpr (REDUCE) {
      if (A.y)
        pairs_tail<P, BASE, REDUCE, true, true>(g, A, acc, p, h, red);
      else
        pairs_tail<P, BASE, REDUCE, true, false>(g, A, acc, p, h, red);
    } else {
      if (A.y) {
        if (rd)
          pairs_tail<P, BASE, REDUCE, true, true>(g, A, acc, p, h, red);
        else
          pairs_tail<P, BASE, REDUCE, false, true>(g, A, acc, p, h, red);
      } else {
        if (rd)
          pairs_tail<P, BASE, REDUCE, true, false>(g, A, acc, p, h, red);
        else
          pairs_tail<P, BASE, REDUCE, false, false>(g, A, acc, p, h, red);
      }
    }
  }
  if (REDUCE) grid_sum<2>(red, slot, nblk, blk);
}

// One block's share of a launch: the SITES output sites of block index blk of nblk (for the
// multi-RHS and batched modes, blk runs over RHS fastest, then site blocks).
template <int P, int R, int MODE, bool REDUCE, int SPLIT, int THREADS>
__device__ __forceinline__ void q_block(const Geom& g, const QLaunch& A0, int blk, int nblk) {
  using T = typename Traits<P>::real;
  // batched modes run one independent system per RHS; BASE is the per-system operation
  constexpr bool BATCH = MODE == Q_BPLAIN || MODE == Q_BCG;
  constexpr int BASE = (MODE == Q_MRHS || MODE == Q_BPLAIN) ? Q_PLAIN : (MODE == Q_BCG ? Q_CGUPDATE : MODE);
  constexpr int SITES = THREADS / SPLIT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int part = SPLIT == 1 ? 0 : warp % SPLIT;
  const int jloc = (warp / SPLIT) * 32 + lane;
  QLaunch A = A0;
  ReduceSlot slot = A0.slot;
  if constexpr (MODE == Q_MRHS || BATCH) {
    // several right-hand sides: consecutive blocks take the same sites for successive RHS
    const int r = blk % A.nrhs;
    blk /= A.nrhs;
    nblk /= A.nrhs;
    A.in = static_cast<const char*>(A.in) + r * A.rhs_stride;
    A.out = static_cast<char*>(A.out) + r * A.rhs_stride;
    if (A.y) A.y = static_cast<const char*>(A.y) + r * A.rhs_stride;
    if constexpr (BATCH) {
      A.cgs = A0.cgs + r * A0.cgs_stride;
      slot.result = A0.slot.result + r * A0.cgs_stride;
      slot.counter = A0.slot.counter + r;
      slot.partials = A0.slot.partials + (int64_t)r * nblk * 2;
    }
  }
  // every block of one system sees the same flags, so whole reductions are skipped together
  if (A.cgs && (A.cgs[CG_DONE] != 0.0 || A.cgs[CG_PENDING] != 0.0)) return;
  const int i = blk * SITES + jloc;
  bool act = i < A.nsites;
  int p = 0, h = 0;
  if (A.nsites == 2 * g.Vh) {
    // both parities: the warps of a pair take the even and odd sites of the same h range, so a
    // link or spinor used by both parities is read from DRAM once while it is still in L2
    both_parities_site(i, &p, &h);
    act = h < g.Vh;
  } else {
    p = A.parity0;
    h = i;
  }
  if constexpr (P != P64 && SPLIT == 1) {
    q_site_pairs<P, R, MODE, REDUCE>(g, A, slot, blk, nblk, act, p, h);
    return;
  }
  Site s;
  if (act) s = site_of(g, p, h);
  Spinor<T> acc;
  if (act) hopping_part<P, R, SPLIT>(acc, g, s, p, h, static_cast<const char*>(A.links), A.in, part);
  if constexpr (SPLIT > 1) {
    extern __shared__ __align__(16) unsigned char qsm_raw[];
    T* sm = reinterpret_cast<T*>(qsm_raw);  // [SPLIT][24][SITES]
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        sm[(part * 24 + 2 * (3 * a + c)) * SITES + jloc] = act ? acc.s[a][c].re : (T)0;
        sm[(part * 24 + 2 * (3 * a + c) + 1) * SITES + jloc] = act ? acc.s[a][c].im : (T)0;
      }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T re = 0, im = 0;
#pragma unroll
        for (int k = 0; k < SPLIT; ++k) {
          re += sm[(k * 24 + 2 * (3 * a + c)) * SITES + jloc];
          im += sm[(k * 24 + 2 * (3 * a + c) + 1) * SITES + jloc];
        }
        acc.s[a][c] = mk(re, im);
      }
  }
  double red[2] = {0.0, 0.0};
  // in the CG mode the operator scale and the base shift come from the solver state, so one
  // captured launch serves every solve
  const double a_d = BASE == Q_CGUPDATE ? A.cgs[CG_ASCALE] : A.a;
  const double b_d = BASE == Q_CGUPDATE ? A.cgs[CG_SIGMA0] : A.b;
  const T diag = (T)A.diag, ca = (T)a_d, cb = (T)b_d;
  const T ca_lo = A.no_g5 ? ca : -ca;  // factor of the lower two spins: gamma5 = diag(1, 1, -1, -1)
  const bool read_diag = REDUCE || A.diag != 0.0;
  constexpr bool IN_PLACE = BASE == Q_CGUPDATE || BASE == Q_XPAY2 || BASE == Q_XPAY3;
  Spinor<T> d, y, z, w;
  if (act) {
    if (read_diag) SpinorIO<P>::load(d, A.din ? A.din : A.in, g.Vh, p, h);
    if (BASE != Q_PLAIN || A.y) SpinorIO<P>::load(y, A.y, g.Vh, p, h);
    if (BASE == Q_CGUPDATE) SpinorIO<P>::load(z, A.out, g.Vh, p, h);
    if (BASE == Q_XPAY2 || BASE == Q_XPAY3) SpinorIO<P>::load(z, A.z, g.Vh, p, h);
    if (BASE == Q_XPAY3) SpinorIO<P>::load(w, A.w, g.Vh, p, h);
  }
  // in the in-place modes every part must have read its copy of z before any part of the
  // block stores (each site's chunks are written by different warps)
  if constexpr (SPLIT > 1 && IN_PLACE) __syncthreads();
  if (act) {
    Spinor<T> res;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        cx<T> v = (T)(-0.5) * acc.s[a][c];
        if (read_diag) v = v + diag * d.s[a][c];
        v = (a < 2 ? ca : ca_lo) * v;
        res.s[a][c] = v;
      }
    if (BASE == Q_PLAIN) {
      if (A.y) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) res.s[a][c] = res.s[a][c] + cb * y.s[a][c];
      }
    } else if (BASE == Q_XPAY2) {
      const T cc = (T)A.c;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) res.s[a][c] = res.s[a][c] + cb * y.s[a][c] + cc * z.s[a][c];
    } else if (BASE == Q_XPAY3) {
      const T cc = (T)A.c, cd = (T)A.d;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          res.s[a][c] = res.s[a][c] + cb * y.s[a][c] + cc * z.s[a][c] + cd * w.s[a][c];
    } else {
      const double alpha = A.cgs[CG_RR] / (a_d * A.cgs[CG_TT] + b_d * A.cgs[CG_PP]);
      const T al = (T)alpha;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) res.s[a][c] = z.s[a][c] - al * (res.s[a][c] + cb * y.s[a][c]);
    }
    SpinorIO<P>::store(res, A.out, g.Vh, p, h, part, SPLIT);
    if (REDUCE) {
      T s0 = 0, s1 = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (SpinorIO<P>::owns(a, c, part, SPLIT)) {
            s0 += norm2(res.s[a][c]);
            s1 += norm2(d.s[a][c]);
          }
      red[0] = (double)s0;
      red[1] = (double)s1;
    }
  }
  if (REDUCE) grid_sum<2>(red, slot, nblk, blk);
}

template <int P, int R, int MODE, bool REDUCE, int SPLIT, int THREADS = Q_THREADS, int MINB = 1>
__global__ void __launch_bounds__(THREADS, MINB) q_kernel(const Geom g, const QLaunch A0) {
  if constexpr (MODE == Q_BPLAIN || MODE == Q_BCG) {
    // batched systems: a grid of resident blocks strides over the (running system, site block)
    // items, running systems fastest.  Each block first lists the systems that have not stopped
    // (their flags do not change during the launch), so a stopped system costs neither a block
    // launch nor a flag read per item.
    constexpr int SITES = THREADS / SPLIT;
    __shared__ short running[ND_BATCH_MAX_SYSTEMS];
    __shared__ int nrun;
    if (threadIdx.x < 32) {
      int base = 0;
      for (int c = 0; c < A0.nrhs; c += 32) {
        const int sys = c + (int)threadIdx.x;
        bool go = false;
        if (sys < A0.nrhs) {
          const double* st = A0.cgs + (int64_t)sys * A0.cgs_stride;
          go = st[CG_DONE] == 0.0 && st[CG_PENDING] == 0.0;
        }
        const unsigned m = __ballot_sync(0xffffffffu, go);
        if (go) running[base + __popc(m & ((1u << threadIdx.x) - 1u))] = (short)sys;
        base += __popc(m);
      }
      if (threadIdx.x == 0) nrun = base;
    }
    __syncthreads();
    const int nr = nrun, bps = (A0.nsites + SITES - 1) / SITES;
    for (int item = blockIdx.x; item < nr * bps; item += gridDim.x) {
      const int sys = running[item % nr], blk = item / nr;
      q_block<P, R, MODE, REDUCE, SPLIT, THREADS>(g, A0, blk * A0.nrhs + sys, bps * A0.nrhs);
    }
  } else if constexpr (P != P64 && SPLIT == 1 && MODE != Q_MRHS) {
    // one system, one warp per site: straight from the launch parameters to the packed path
    if (A0.cgs && (A0.cgs[CG_DONE] != 0.0 || A0.cgs[CG_PENDING] != 0.0)) return;
    const int i = blockIdx.x * THREADS + threadIdx.x;
    int p = A0.parity0, h = i;
    bool act = i < A0.nsites;
    if (A0.nsites == 2 * g.Vh) {
      both_parities_site(i, &p, &h);
      act = h < g.Vh;
    }
    q_site_pairs<P, R, MODE, REDUCE>(g, A0, A0.slot, blockIdx.x, gridDim.x, act, p, h);
  } else {
    q_block<P, R, MODE, REDUCE, SPLIT, THREADS>(g, A0, blockIdx.x, gridDim.x);
  }
}

template <int P, int R, int MODE, bool REDUCE, int SPLIT, int THREADS, int MINB>
static cudaError_t launch_q5(const Geom& g, const QLaunch& L, cudaStream_t st) {
  constexpr int SITES = THREADS / SPLIT;
  int blocks = (L.nsites + SITES - 1) / SITES * (L.nrhs > 1 ? L.nrhs : 1);
  const size_t smem = SPLIT > 1 ? (size_t)SPLIT * 24 * SITES * sizeof(typename Traits<P>::real) : 0;
  static bool attr = false;
  if (smem > 48 * 1024 && !attr) {
    cudaFuncSetAttribute(q_kernel<P, R, MODE, REDUCE, SPLIT, THREADS, MINB>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  if constexpr (MODE == Q_BPLAIN || MODE == Q_BCG) {
    // one wave of resident blocks (per device, looked up once)
    static int resident[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && resident[dev] == 0) {
      int per_sm = 0, sms = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, q_kernel<P, R, MODE, REDUCE, SPLIT, THREADS, MINB>,
                                                    THREADS, smem);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      resident[dev] = std::max(1, per_sm) * std::max(1, sms);
    }
    if (dev < 64) blocks = std::min(blocks, resident[dev]);
  }
  q_kernel<P, R, MODE, REDUCE, SPLIT, THREADS, MINB><<<blocks, THREADS, smem, st>>>(g, L);
  return cudaGetLastError();
}

// Block shapes.  One warp per site: FP32 and FP16 run 64-thread blocks; on 64x32^3 these beat
// 256-thread blocks by 20-30 % (more independent blocks in flight per SM, smaller tail).  The
// register cap is 128 (8 blocks per SM) except for FP32 18-real links, where 6 blocks per SM
// (170 registers) is 7 % faster (sweep of 8/6/5/4 blocks per SM: FP32-12 6002/5783/5782/5780 GB/s,
// FP32-18 6329/6752/6753/5967 GB/s).  FP64 is FP64-ALU bound and keeps 256 threads.  Split
// kernels combine warps through shared memory and use 256-thread blocks.
template <int P, int R>
constexpr int q_min_blocks() {
  return (P == P32 && R == 18) ? 6 : 8;
}

// One warp per site in 64-thread blocks.
template <int P, int R, int MODE, bool REDUCE>
static cudaError_t launch_q64(const Geom& g, const QLaunch& L, cudaStream_t st) {
  return launch_q5<P, R, MODE, REDUCE, 1, 64, q_min_blocks<P, R>()>(g, L, st);
}

template <int P, int R, int MODE, bool REDUCE>
static cudaError_t launch_q4(const Geom& g, const QLaunch& L, cudaStream_t st) {
  switch (L.split) {
    case 1:
      if (P == P64 || L.threads == 256) return launch_q5<P, R, MODE, REDUCE, 1, 256, 1>(g, L, st);
      return launch_q64<P, R, MODE, REDUCE>(g, L, st);
    case 2: return launch_q5<P, R, MODE, REDUCE, 2, 256, 1>(g, L, st);
    case 4: return launch_q5<P, R, MODE, REDUCE, 4, 256, 1>(g, L, st);
  }
  return cudaErrorInvalidValue;
}

template <int P, int R>
static cudaError_t launch_q2(const Geom& g, const QLaunch& L, cudaStream_t st) {
  switch (L.mode) {
    case Q_PLAIN:
      return L.reduce ? launch_q4<P, R, Q_PLAIN, true>(g, L, st) : launch_q4<P, R, Q_PLAIN, false>(g, L, st);
    case Q_XPAY2:
      return L.reduce ? launch_q4<P, R, Q_XPAY2, true>(g, L, st) : launch_q4<P, R, Q_XPAY2, false>(g, L, st);
    case Q_CGUPDATE:
      return L.reduce ? launch_q4<P, R, Q_CGUPDATE, true>(g, L, st) : launch_q4<P, R, Q_CGUPDATE, false>(g, L, st);
    case Q_XPAY3:
      if (L.reduce || L.split != 1) return cudaErrorInvalidValue;
      if (P == P64 || L.threads == 256) return launch_q5<P, R, Q_XPAY3, false, 1, 256, 1>(g, L, st);
      return launch_q5<P, R, Q_XPAY3, false, 1, 64, 8>(g, L, st);
    case Q_MRHS:
      if (L.reduce || L.split != 1) return cudaErrorInvalidValue;
      if (P == P64 || L.threads == 256) return launch_q5<P, R, Q_MRHS, false, 1, 256, 1>(g, L, st);
      return launch_q64<P, R, Q_MRHS, false>(g, L, st);
    case Q_BPLAIN:
      if (!L.reduce || L.split != 1) return cudaErrorInvalidValue;
      if (P == P64) return launch_q5<P, R, Q_BPLAIN, true, 1, 256, 1>(g, L, st);
      return launch_q5<P, R, Q_BPLAIN, true, 1, 256, 2>(g, L, st);
    case Q_BCG:
      if (!L.reduce || L.split != 1) return cudaErrorInvalidValue;
      if (P == P64) return launch_q5<P, R, Q_BCG, true, 1, 256, 1>(g, L, st);
      return launch_q5<P, R, Q_BCG, true, 1, 256, 2>(g, L, st);
  }
  return cudaErrorInvalidValue;
}

template <int P>
static cudaError_t launch_q1(const Geom& g, const QLaunch& L, cudaStream_t st) {
  switch (L.recon) {
    case 18: return launch_q2<P, 18>(g, L, st);
    case 12: return launch_q2<P, 12>(g, L, st);
    case 8: return launch_q2<P, 8>(g, L, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nd
