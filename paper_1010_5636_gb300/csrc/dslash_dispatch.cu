// Dispatch of Q launches to the per-precision translation units.
#include <cstdlib>

#include "kernels.h"

namespace nd {
cudaError_t launch_q_fp64(const Geom& g, const QLaunch& L, cudaStream_t st);
cudaError_t launch_q_fp32(const Geom& g, const QLaunch& L, cudaStream_t st);
cudaError_t launch_q_fp16(const Geom& g, const QLaunch& L, cudaStream_t st);

// Warps per site for a (precision, link form).  ND_Q_SPLIT=1|2|4 in the environment overrides
// the choice (used by the tuning sweep).
int default_split(int prec, int recon, bool half) {
  (void)recon;
  static int env = -1;
  if (env < 0) {
    const char* e = std::getenv("ND_Q_SPLIT");
    env = e ? std::atoi(e) : 0;
    if (env != 1 && env != 2 && env != 4) env = 0;
  }
  if (env) return env;
  // measured on 64x32^3 with the 64-thread block shape: one warp per site is fastest for every
  // precision and link form
  (void)prec;
  (void)half;
  return 1;
}

cudaError_t launch_q_mrhs(const Geom& g, const QLaunch& L0, int nrhs, size_t stride, cudaStream_t st) {
  if (L0.mode != Q_PLAIN || L0.reduce) return cudaErrorInvalidValue;
  QLaunch L = L0;
  L.mode = Q_MRHS;
  L.nrhs = nrhs;
  L.rhs_stride = (int64_t)stride;
  L.split = 1;
  L.threads = 0;
  return launch_q(g, L, st);
}

// Right-hand sides per thread for multi-RHS launches the autotuner has not set; ND_Q_KRHS=1|2|3
// in the environment overrides it (comparison measurements).
static int default_krhs() {
  static int v = -1;
  if (v < 0) {
    const char* e = std::getenv("ND_Q_KRHS");
    v = e ? std::atoi(e) : 1;
    if (v < 1 || v > 3) v = 1;
  }
  return v;
}

cudaError_t launch_q(const Geom& g, const QLaunch& L0, cudaStream_t st) {
  if (L0.nsites <= 0) return cudaSuccess;
  QLaunch L = L0;
  if (L.mode == Q_MRHS && L.krhs == 0) L.krhs = default_krhs();
  if (L.mode == Q_MRHS && L.krhs > 1 && L.prec != 0 && L.nrhs > 1) return launch_q_mrhs_k(g, L, st);
  if (L.mode == Q_MRHS && (L.nrhs < 1 || L.reduce)) return cudaErrorInvalidValue;
  if ((L.mode == Q_BPLAIN || L.mode == Q_BCG) && (L.nrhs < 1 || !L.reduce)) return cudaErrorInvalidValue;
  if (L.split == 0) L.split = default_split(L.prec, L.recon, L.nsites != 2 * g.Vh);
  if (L.mode == Q_MRHS || L.mode == Q_BPLAIN || L.mode == Q_BCG || L.mode == Q_XPAY3) L.split = 1;
  if (L.split != 1 && L.split != 2 && L.split != 4) return cudaErrorInvalidValue;
  switch (L.prec) {
    case 0: return launch_q_fp64(g, L, st);
    case 1: return launch_q_fp32(g, L, st);
    case 2: return launch_q_fp16(g, L, st);
  }
  return cudaErrorInvalidValue;
}
}  // namespace nd

namespace nd {
int64_t bcg_partials(const Geom& g, int prec, int nsys) {
  const int sites_per_block = prec == 0 ? 256 : 64;
  const int64_t nblk = (2 * (int64_t)g.Vh + sites_per_block - 1) / sites_per_block;
  return nblk * 2 * nsys;
}
}  // namespace nd
