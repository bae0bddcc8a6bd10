// Instantiations of the Q kernels for storage precision FP16 (see dslash_impl.cuh).
#include "dslash_impl.cuh"

namespace nd {
cudaError_t launch_q_fp16(const Geom& g, const QLaunch& L, cudaStream_t st) { return launch_q1<P16>(g, L, st); }
}  // namespace nd
