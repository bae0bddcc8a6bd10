// Host-side declarations of the kernel launchers of libnd (no torch types, no C++ exceptions).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "geometry.cuh"
#include "reduce.cuh"

namespace nd {

// Device scalar block of the multi-shift CG: CG_NSCALAR scalars followed by per-shift arrays
// of CG_NMAX entries (index CG_NSCALAR + array * CG_NMAX + shift).  Two-value reductions
// write pairs (TT, PP) and (RRNEW, JUNK).
enum CgScalar {
  CG_RR = 0,          // (r, r) of the current residual
  CG_TT = 1,          // ||Q p0||^2, fused into the first Q of the iteration
  CG_PP = 2,          // ||p0||^2
  CG_DONE = 3,        // nonzero: stop now (error); every kernel of the iteration skips
  CG_RRNEW = 4,       // (r, r) after the residual update
  CG_JUNK = 5,
  CG_PENDING = 6,     // nonzero: stop after the current iteration's solution update
  CG_STATUS = 7,      // nd_status of the run
  CG_ITER = 8,        // iterations completed
  CG_ALPHA_PREV = 9,
  CG_BETA_PREV = 10,
  CG_BNORM2 = 11,     // ||b||^2
  CG_ASCALE = 12,     // A = ascale * Q^2
  CG_SIGMA0 = 13,     // base shift
  CG_LIVE_SUM = 14,   // sum over iterations of the shifts whose direction p_l was updated
  CG_ACTIVE_SUM = 15, // sum over iterations of the shifts whose solution (x_l or its y term) was updated
  CG_NSCALAR = 16
};
enum CgArray {
  SH_SIGMA = 0, SH_ZETA, SH_ZETAP, SH_COEFX, SH_COEFR, SH_COEFP, SH_ACTIVE, SH_UPD, SH_LIVE, SH_RES, SH_TOL,
  SH_W, SH_NARRAY
};
constexpr int CG_NMAX = 32;
// Largest number of systems of one batched CG (the batched Q and update kernels list them in
// shared memory).
constexpr int ND_BATCH_MAX_SYSTEMS = 1024;
constexpr int CG_STATE_DOUBLES = CG_NSCALAR + SH_NARRAY * CG_NMAX;
__host__ __device__ inline int sh(int array, int l) { return CG_NSCALAR + array * CG_NMAX + l; }

// Q_MRHS: Q_PLAIN over nrhs fields.  Q_BPLAIN / Q_BCG: Q_PLAIN / Q_CGUPDATE with a reduction,
// over nrhs independent systems (the batched CG): field r at + r * rhs_stride, its scalar block
// at cgs + r * cgs_stride, its reduction partials / counter / result offset likewise.
enum QMode { Q_PLAIN = 0, Q_CGUPDATE = 1, Q_XPAY2 = 2, Q_MRHS = 3, Q_BPLAIN = 4, Q_BCG = 5, Q_XPAY3 = 6 };

// out = a * gamma5 (diag * in - 1/2 hop(in)) + b * y      (Q_PLAIN; y may be null)
// out = a * gamma5 (diag * in - 1/2 hop(in)) + b * y + c * z   (Q_XPAY2; z may alias out)
// out = a * gamma5 (diag * in - 1/2 hop(in)) + b * y + c * z + d * w
//                                             (Q_XPAY3, one Clenshaw step; z may alias out)
// out = out - alpha * (a * gamma5(diag * in - 1/2 hop(in)) + b * y),
//       alpha = cgs[CG_RR] / (a * cgs[CG_TT] + b * cgs[CG_PP]),
//       a = cgs[CG_ASCALE], b = cgs[CG_SIGMA0]                       (Q_CGUPDATE)
// Output sites: parity `parity0` only (nsites = Vh) or both parities (nsites = 2 Vh).
// reduce: slot.result[0] = sum ||out||^2, slot.result[1] = sum ||in||^2 over the output sites.
struct QLaunch {
  int prec;  // 0 FP64, 1 FP32, 2 FP16
  int recon; // 18, 12, 8
  int mode;
  bool reduce;
  const void* links;
  const void* in;
  void* out;
  const void* y;
  const void* z;  // Q_XPAY2 and Q_XPAY3
  const void* w;    // Q_XPAY3 only
  const void* din;  // field the diagonal term reads (null: in)
  int no_g5;        // 1: leave gamma5 out (out = a (diag * din - 1/2 hop(in)) + ...), i.e. D_W blocks
  double diag, a, b, c, d;
  int parity0, nsites;
  ReduceSlot slot;
  const double* cgs;  // multi-shift CG scalars, or null; kernels skip when cgs[CG_DONE] or cgs[CG_PENDING] != 0
  int split;          // warps per site: 1, 2 or 4 (0 = default for the precision)
  int threads;        // 0: default block shape; 256: 256-thread blocks (callers that size
                      // per-block scratch for 256 sites per block)
  int nrhs;           // right-hand sides in one launch (0 or 1: one)
  int64_t rhs_stride; // bytes between consecutive RHS fields
  int64_t cgs_stride; // doubles between consecutive systems' scalar blocks (batched modes)
  int krhs;           // Q_MRHS, FP32/FP16: right-hand sides per thread sharing each link (0 or 1: one,
                      // q_kernel; 2 or 3: dslash_mrhs.cu)
};
int default_split(int prec, int recon, bool half);

cudaError_t launch_q(const Geom& g, const QLaunch& L, cudaStream_t st);
// The same operator on nrhs fields at in + r * stride (out, y likewise), one launch: the RHS
// index is the fastest-varying block index, so the blocks that read one tile of links for all
// RHS run back to back and the links come from DRAM once (Q_PLAIN, no reduction, one warp per
// site).
cudaError_t launch_q_mrhs(const Geom& g, const QLaunch& L, int nrhs, size_t stride, cudaStream_t st);
// Q_MRHS with L.krhs (2 or 3) right-hand sides per thread (FP32 / FP16; dslash_mrhs.cu).
cudaError_t launch_q_mrhs_k(const Geom& g, const QLaunch& L, cudaStream_t st);

// Several lattices in one persistent launch (dslash_batched.cu): lattice k applies Q to nrhs
// fields at in + r * stride; its tiles (64 sites of one RHS) start at tile_begin in the list.
constexpr int ND_MAX_BATCH = 32;
struct LatticeWork {
  Geom g;
  const char* links;
  const void* in;
  void* out;
  int64_t stride;
  int nrhs;
  int tile_begin;
  double diag;
};
int batched_tiles(int64_t V);
cudaError_t launch_q_batched(int prec, int recon, const LatticeWork* work_dev, int nlat, int total, int grid,
                             cudaStream_t st);

// Launch-shape autotuner (tune.cu): on the first launch of a (precision, links, lattice, kind)
// the candidates are timed on the caller's stream and the fastest is kept (in memory and, with
// ND_AUTOTUNE_CACHE=<file>, on disk).  Applies only to launches that may be repeated (out does
// not alias in); skipped while the stream is being captured or when ND_AUTOTUNE=0.
cudaError_t autotune_launch(const Geom& g, QLaunch& L, cudaStream_t st);

// Pack / unpack between canonical FP64 ([lex][4][3][2]) and internal precision `prec`.
cudaError_t launch_pack_spinor(const Geom& g, int prec, void* internal, const double* canon, cudaStream_t st);
cudaError_t launch_unpack_spinor(const Geom& g, int prec, double* canon, const void* internal, cudaStream_t st);
cudaError_t launch_pack_spinor_f32(const Geom& g, int prec, void* internal, const float* canon, cudaStream_t st);
cudaError_t launch_unpack_spinor_f32(const Geom& g, int prec, float* canon, const void* internal, cudaStream_t st);
// Compress canonical FP64 links ([4][lex][3][3][2]) into the internal (prec, recon) form.
// For recon 8, *bad (device int) is set to 1 if any link is within the singular set.
cudaError_t launch_pack_links(const Geom& g, int prec, int recon, void* internal, const double* canon, int* bad,
                              cudaStream_t st);
int64_t link_bytes(int prec, int recon, int64_t Vh);
int64_t spinor_bytes(int prec, int64_t Vh);
cudaError_t launch_eo_tables(const Geom& g, int32_t* lex2eo, int32_t* nbr, cudaStream_t st);

// ---------------------------------------------------------------- BLAS-1 (blas.cu)
// Fields are whole-lattice internal spinors of precision `prec`.  Reductions are FP64 and
// deterministic (reduce.cuh); `slot` receives the results.
// z = a x + b y (x, y, z may alias); reduce: result[0] = ||z||^2
cudaError_t blas_axpby(const Geom& g, int prec, void* z, double a, const void* x, double b, const void* y, bool reduce,
                       ReduceSlot slot, cudaStream_t st);
// result[0..1] = (x, y) = sum conj(x) y (complex); result[2] = ||x||^2
cudaError_t blas_dot(const Geom& g, int prec, const void* x, const void* y, ReduceSlot slot, cudaStream_t st);
// out (prec_out) = in (prec_in); out may not alias in unless the precisions match
cudaError_t blas_convert(const Geom& g, int prec_out, void* out, int prec_in, const void* in, cudaStream_t st);
// out (FP32 or FP16) = in (FP64) / sqrt(*norm2_dev) (device scalar; zero field when it is zero)
cudaError_t blas_convert_normalized(const Geom& g, int prec_out, void* out, const void* in, const double* norm2_dev,
                                    cudaStream_t st);
// x64 (FP64) += a e32 (FP32)
cudaError_t blas_axpy_widen(const Geom& g, void* x64, double a, const void* e32, cudaStream_t st);
// out = gamma5 in (any precision; out may alias in)
cudaError_t blas_g5(const Geom& g, int prec, void* out, const void* in, cudaStream_t st);
// out = c1 x + c2 gamma5 y  (FP64 fields)
cudaError_t blas_g5_axpby(const Geom& g, void* out, double c1, const void* x, double c2, const void* y,
                          cudaStream_t st);
// FP64 only: result[2k..2k+1] = (v_k, w) for k < K (v_k = base + k * stride bytes), K <= 64
cudaError_t blas_multidot(const Geom& g, const void* base, size_t stride, int K, const void* w, ReduceSlot slot,
                          cudaStream_t st);
// FP64 only: out = beta * y + sum_k coef[k] v_k with complex coef (device array of 2K doubles)
cudaError_t blas_lincomb(const Geom& g, void* out, double beta, const void* y, const void* base, size_t stride, int K,
                         const double* coef, cudaStream_t st);

// FP64 field of deterministic pseudo-random reals in [-1, 1)
cudaError_t blas_random(const Geom& g, void* out, uint64_t seed, cudaStream_t st);

// ---------------------------------------------------------------- batched CG (mscg.cu)
// nsys independent shifted CG systems, each with a full scalar block (CG_STATE_DOUBLES, one
// shift) at states + s * CG_STATE_DOUBLES; fields at + s * field bytes.
cudaError_t bcg_init(double* states, int nsys, cudaStream_t st);
cudaError_t bcg_scalar(double* states, int nsys, int maxit, const cudaGraphConditionalHandle* h, cudaStream_t st);
cudaError_t bcg_update(const Geom& g, int ps, const void* r, void* p, void* x, size_t fstride, const double* states,
                       int nsys, cudaStream_t st);
// Partials needed by one batched reducing Q launch over nsys systems (doubles).
int64_t bcg_partials(const Geom& g, int prec, int nsys);

// ---------------------------------------------------------------- multi-shift CG (mscg.cu)
cudaError_t mscg_init(double* state, int n, cudaStream_t st);
cudaError_t mscg_scalar(double* state, int n, int maxit, cudaStream_t st);
// The same step inside a CUDA graph whose while-loop runs the iterations: when the run stops
// the kernel sets the loop's condition to zero.
cudaError_t mscg_scalar_graph(double* state, int n, int maxit, cudaGraphConditionalHandle h, cudaStream_t st);
// For every live shift l (x_l / p_l at base + l * stride): x_l += coefx_l p_l (or y += w_l coefx_l p_l
// when ymode), p_l = coefr_l r + coefp_l p_l.
cudaError_t mscg_update(const Geom& g, int prec_s, int prec_x, bool ymode, const void* r, void* p_all, size_t pstride,
                        void* x_all, size_t xstride, void* y, const double* state, int n, cudaStream_t st);

}  // namespace nd
