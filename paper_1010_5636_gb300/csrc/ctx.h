// Host-side context of libnd and shared host helpers (error reporting, workspaces).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/nd.h"
#include "kernels.h"

constexpr int ND_PINNED_DOUBLES = 4096;

// One multi-shift CG solve captured as a CUDA graph: a device-side while loop whose body is one
// iteration (four kernels); reused while every buffer pointer and size in the key matches.
struct nd_ms_graph {
  int kind = 0;  // 0: multi-shift CG, 1: batched CG
  int ps = 0, px = 0, ymode = 0, n = 0, maxit = 0;
  const void *r = nullptr, *t = nullptr, *p = nullptr, *x = nullptr, *state = nullptr, *links = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

struct nd_ctx {
  nd::Geom g;
  int dims[4];
  int64_t V = 0, Vh = 0;
  double m = 0, s = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};  // device timing of solver passes (reported in info structs)
  // links per precision (index nd_prec); recon 0 = absent
  void* links[3] = {nullptr, nullptr, nullptr};
  int recon[3] = {0, 0, 0};
  bool poisoned = false;
  std::string err;
  // reduction scratch: partials for up to max_blocks * 8 doubles, one counter, result scratch
  double* red_partials = nullptr;
  unsigned* red_counter = nullptr;
  double* red_scratch = nullptr;  // 64 doubles of general-purpose device results
  double* host_pinned = nullptr;  // ND_PINNED_DOUBLES doubles of pinned host memory for result read-back
  int max_blocks = 0;
  // named device workspaces (grown on demand, freed in nd_destroy)
  std::map<std::string, std::pair<void*, size_t>> ws;
  // low modes: FP64 internal fields [l], nu, rho
  int nlow = 0;
  void* evecs = nullptr;
  size_t evecs_cap = 0;
  std::vector<double> nu, rho;
  double lam_next = 0.0, lam_max = 0.0;
  // captured multi-shift iterations (graphs_ok = false after a capture failure, or with ND_GRAPHS=0 in
  // the environment: chunked launches from the host)
  cudaStream_t cap_stream = nullptr;
  // second stream of the mixed-precision refinement (the slowest shifts' first correction runs on it
  // while the other shifts are refined on `stream`), with its fork and join events
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  std::vector<nd_ms_graph> ms_graphs;
  bool graphs_ok = true;
};

namespace nd {

// A named range on the NVTX timeline around a solver phase: visible to profilers (ncu --nvtx),
// a no-op when none is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};


nd_status fail(nd_ctx* c, nd_status st, const std::string& msg);
nd_status fail_cuda(nd_ctx* c, cudaError_t e, const char* what);
// Device workspace of at least `bytes`, cached under `name`.
void* workspace(nd_ctx* c, const std::string& name, size_t bytes);
ReduceSlot slot(nd_ctx* c, double* result);
inline int prec_index(nd_prec p) { return (int)p; }

}  // namespace nd

#define ND_TRY_CUDA(ctx, call)                                   \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return nd::fail_cuda((ctx), e_, #call); \
  } while (0)

#define ND_TRY(call)                 \
  do {                               \
    nd_status s_ = (call);           \
    if (s_ != ND_OK) return s_;      \
  } while (0)
