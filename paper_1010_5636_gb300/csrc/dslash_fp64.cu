// Instantiations of the Q kernels for storage precision FP64 (see dslash_impl.cuh).
#include "dslash_impl.cuh"

namespace nd {
cudaError_t launch_q_fp64(const Geom& g, const QLaunch& L, cudaStream_t st) { return launch_q1<P64>(g, L, st); }
}  // namespace nd
