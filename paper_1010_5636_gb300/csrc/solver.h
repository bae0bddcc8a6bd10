// Host-side building blocks shared by the solver, low-mode and overlap entry points.
#pragma once
#include <string>
#include <vector>

#include "ctx.h"

namespace nd {

// out = a * Q in + b * y + cz * z + cw * w (internal fields of precision prec; z may alias out).  With result != null
// the launch also reduces ||out||^2 and ||in||^2 into result[0..1] (not with w).
nd_status q_apply(nd_ctx* c, int prec, void* out, const void* in, double a = 1.0, double b = 0.0,
                  const void* y = nullptr, double* result = nullptr, const double* cgs = nullptr,
                  const void* z = nullptr, double cz = 0.0, const void* w = nullptr, double cw = 0.0);

// Device buffer for one internal field of `prec`, cached under `name`.
void* field(nd_ctx* c, const char* name, int prec, int count = 1);

// Read n doubles from device memory (synchronises the context's stream, or st).
nd_status read_back(nd_ctx* c, const double* dev, double* host, int n);
nd_status read_back_on(nd_ctx* c, cudaStream_t st, const double* dev, double* host, int n);

// A batched CG in flight (solver.cu, bcg_start / bcg_finish).
struct BcgJob {
  int nsys = 0;
  double* states = nullptr;
  cudaStream_t stream = nullptr;
};

struct MsResult {
  int iters = 0;
  int status = ND_OK;
  std::vector<double> res;  // per-shift recurrence residual (relative to ||b||)
  double ms = 0.0;          // device time of the iterations (CUDA events on the context's stream)
  double live = 0.0;        // sum over iterations of the shifts whose p_l was updated
  double active = 0.0;      // sum over iterations of the shifts whose x_l (or y term) was updated
};

// Multi-shift CG on A = ascale * Q^2 with shifts sigma[0..n) (ascending, sigma[0] the base).
// b: field of precision ps.  ymode: y (precision px) += sum_l w_l x_l only; otherwise x_l
// (precision px, at x_all + l * field bytes) are the solutions.  x / y start from zero.
nd_status mscg_run(nd_ctx* c, int ps, int px, bool ymode, const void* b, void* x_or_y, const std::vector<double>& sigma,
                   const std::vector<double>& tol, const std::vector<double>& w, double ascale, int maxit,
                   MsResult* out);

// r = b - (ascale Q^2 + sigma) x in FP64, ||r||^2 reduced into norm2_dev (device), no host sync.
nd_status residual64_dev(nd_ctx* c, void* r, const void* b, const void* x, double sigma, double ascale,
                         double* norm2_dev);
// r = b - (ascale Q^2 + sigma) x in FP64; returns ||r|| / ||b|| through *rel (bnorm2 given).
nd_status residual64(nd_ctx* c, void* r, const void* b, const void* x, double sigma, double ascale, double bnorm2,
                     double* rel);

// Solve (ascale Q^2 + sigma_l) x_l = b for all l in mixed precision: sloppy multi-shift CG in
// precision ps, then FP64 defect correction of every shift down to tol[l].  b64: FP64 field.
// Calls `sink(l, x64)` with each refined FP64 solution (the buffer is reused after the call).
struct MixedStats {
  int iters = 0, sloppy_iters = 0, outer = 0;
  double max_resid = 0.0;
  double krylov_ms = 0.0, live = 0.0, active = 0.0;  // the sloppy multi-shift pass (MsResult)
  int residuals64 = 0;                                // FP64 residuals of the refinement
  int correction_iters = 0;                           // correction-solve iterations summed over systems
  double refine_ms = 0.0;                             // wall time of the refinement
};
template <typename Sink>
nd_status mixed_solve(nd_ctx* c, int ps, const void* b64, double bnorm2, const std::vector<double>& sigma,
                      const std::vector<double>& tol, double ascale, int maxit, MixedStats* st, Sink sink);

nd_status mixed_solve_impl(nd_ctx* c, int ps, const void* b64, double bnorm2, const std::vector<double>& sigma,
                           const std::vector<double>& tol, double ascale, int maxit, MixedStats* st,
                           nd_status (*sink)(void*, int, void*), void* sink_ctx);

template <typename Sink>
nd_status mixed_solve(nd_ctx* c, int ps, const void* b64, double bnorm2, const std::vector<double>& sigma,
                      const std::vector<double>& tol, double ascale, int maxit, MixedStats* st, Sink sink) {
  return mixed_solve_impl(
      c, ps, b64, bnorm2, sigma, tol, ascale, maxit, st,
      [](void* ctx, int l, void* x) -> nd_status { return (*static_cast<Sink*>(ctx))(l, x); }, &sink);
}

// sign(Q) in64 (internal FP64 layout) with the deflated approximation of p; *sign64 points to a
// context workspace holding the result (internal FP64) until the next sign application.
nd_status sign_internal(nd_ctx* c, const void* in64, const nd_dn_params* p, nd_dn_info* info, void** sign64);

// Hermitian eigenproblem (cyclic Jacobi): A (n x n, row-major complex as re/im pairs) is
// overwritten; evals ascending, evecs column k = eigenvector k (row-major, re/im pairs).
void hermitian_eig(int n, std::vector<double>& A, std::vector<double>& evals, std::vector<double>& evecs);

}  // namespace nd
