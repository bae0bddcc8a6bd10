// Q with fused norms for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they apply the operator: code that
// runs under a fixed memory budget handed out by another allocator, or a solver loop that has
// promised its host application no allocation after set-up.  nd_apply_Q_norms_static serves
// them: it applies Q and returns ||Q in||^2 and ||in||^2 like the fused-norm launch of the
// multi-shift solver, but the reduction scratch (block partials, the finishing counter and
// the two results) lives in the file-scope array below instead of context workspaces.
//
// The array is NORMS_SCRATCH_DOUBLES doubles (256 KiB + 64 bytes) on every GPU that loads
// the library, held until the process exits.  It bounds the lattice to
// NORMS_STATIC_MAX_SITES sites (one block of 256 sites per partial pair).
// In host code the name `norms_scratch` is only a host-side stand-in: the device address is
// obtained once per device with cudaGetSymbolAddress, on the first call made with that device
// current; make that first call before any stream capture.
// Every call shares the array and leaves its last contents there; calls that overlap on the
// GPU (different streams, or different host threads on the same device) race on it.
#include <mutex>

#include "ctx.h"
#include "solver.h"

namespace nd {

constexpr int NORMS_STATIC_MAX_BLOCKS = 16384;
constexpr int64_t NORMS_STATIC_MAX_SITES = (int64_t)NORMS_STATIC_MAX_BLOCKS * 256;
// [0, 2): results, [2, 8): counter word + padding, [8, 8 + 2 * MAX_BLOCKS): block partials
constexpr int NORMS_SCRATCH_DOUBLES = 8 + 2 * NORMS_STATIC_MAX_BLOCKS;

static __device__ __align__(256) double norms_scratch[NORMS_SCRATCH_DOUBLES];

namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
double* g_scratch_dev[MAX_DEVICES] = {nullptr};
}  // namespace

// Device address of the scratch array for the current device (set up on first use).
static cudaError_t scratch_address(int device, double** out) {
  if (device < 0 || device >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_dev[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, norms_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[device] = static_cast<double*>(p);
  }
  *out = g_scratch_dev[device];
  return cudaSuccess;
}

}  // namespace nd

using namespace nd;

extern "C" nd_status nd_apply_Q_norms_static(nd_ctx* c, void* out, const void* in, nd_prec prec, double* norms) {
  if (!c) return ND_ERR_INVALID_ARG;
  if (c->poisoned) return fail(c, ND_ERR_STATE, "context unusable after an earlier CUDA error: " + c->err);
  if (!out || !in || !norms || prec < ND_FP64 || prec > ND_FP16 || out == in)
    return fail(c, ND_ERR_INVALID_ARG, "nd_apply_Q_norms_static: bad argument");
  if (c->V > NORMS_STATIC_MAX_SITES)
    return fail(c, ND_ERR_INVALID_ARG,
                "nd_apply_Q_norms_static: lattice larger than the static scratch allows (4194304 sites)");
  if (!c->links[prec]) return fail(c, ND_ERR_STATE, "nd_apply_Q_norms_static: no links set in this precision");
  int dev = 0;
  ND_TRY_CUDA(c, cudaGetDevice(&dev));
  double* s = nullptr;
  ND_TRY_CUDA(c, scratch_address(dev, &s));
  // the finishing counter must start at zero (the kernel leaves it at zero, but an earlier
  // call that failed part-way would not)
  ND_TRY_CUDA(c, cudaMemsetAsync(s + 2, 0, sizeof(double), c->stream));
  QLaunch L{};
  L.prec = (int)prec;
  L.recon = c->recon[prec];
  L.mode = Q_PLAIN;
  L.reduce = true;
  L.links = c->links[prec];
  L.in = in;
  L.out = out;
  L.diag = 4.0 + c->m;
  L.a = 1.0;
  L.nsites = (int)c->V;
  L.split = 1;
  L.threads = 256;  // 256 sites per block: the partials fit the static array
  L.slot.result = s;
  L.slot.counter = reinterpret_cast<unsigned*>(s + 2);
  L.slot.partials = s + 8;
  ND_TRY_CUDA(c, launch_q(c->g, L, c->stream));
  ND_TRY_CUDA(c, cudaMemcpyAsync(norms, s, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  ND_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
  return ND_OK;
}
