// C-ABI entry points of libnd: context lifecycle, field packing, site tables and Q.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ctx.h"

namespace nd {

nd_status fail(nd_ctx* c, nd_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

nd_status fail_cuda(nd_ctx* c, cudaError_t e, const char* what) {
  if (c) {
    c->err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    c->poisoned = true;
  }
  return ND_ERR_CUDA;
}

void* workspace(nd_ctx* c, const std::string& name, size_t bytes) {
  auto it = c->ws.find(name);
  if (it != c->ws.end() && it->second.second >= bytes) return it->second.first;
  if (it != c->ws.end()) {
    cudaFree(it->second.first);
    c->ws.erase(it);
  }
  void* p = nullptr;
  if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  c->ws[name] = {p, bytes};
  return p;
}

ReduceSlot slot(nd_ctx* c, double* result) {
  ReduceSlot s;
  s.partials = c->red_partials;
  s.counter = c->red_counter;
  s.result = result;
  return s;
}

}  // namespace nd

using namespace nd;

static nd_status check_ctx(nd_ctx* c) {
  if (!c) return ND_ERR_INVALID_ARG;
  if (c->poisoned) return fail(c, ND_ERR_STATE, "context unusable after an earlier CUDA error: " + c->err);
  return ND_OK;
}

extern "C" {

const char* nd_status_string(nd_status st) {
  switch (st) {
    case ND_OK: return "ok";
    case ND_ERR_INVALID_ARG: return "invalid argument";
    case ND_ERR_CUDA: return "CUDA error";
    case ND_ERR_OOM: return "out of device memory";
    case ND_ERR_NOT_CONVERGED: return "not converged";
    case ND_ERR_BREAKDOWN: return "Krylov breakdown";
    case ND_ERR_NAN: return "NaN or Inf encountered";
    case ND_ERR_STATE: return "invalid state";
  }
  return "unknown status";
}

const char* nd_last_error(const nd_ctx* c) { return c ? c->err.c_str() : "null context"; }

int64_t nd_volume(const nd_ctx* c) { return c ? c->V : 0; }

size_t nd_spinor_bytes(const nd_ctx* c, nd_prec prec) {
  if (!c || prec < ND_FP64 || prec > ND_FP16) return 0;
  return (size_t)spinor_bytes((int)prec, c->Vh);
}

nd_status nd_create(nd_ctx** out, const int dims[4], int antiperiodic_t, double m, double s, void* stream) {
  if (!out || !dims) return ND_ERR_INVALID_ARG;
  *out = nullptr;
  int64_t V = 1;
  for (int k = 0; k < 4; ++k) {
    if (dims[k] <= 0 || dims[k] % 2) return ND_ERR_INVALID_ARG;
    V *= dims[k];
  }
  if (V > (int64_t(1) << 30) || !(s > -1.0 && s < 1.0)) return ND_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return ND_ERR_CUDA;
  }
  nd_ctx* c = new nd_ctx();
  for (int k = 0; k < 4; ++k) c->dims[k] = dims[k];
  c->V = V;
  c->Vh = V / 2;
  c->m = m;
  c->s = s;
  c->stream = static_cast<cudaStream_t>(stream);
  cudaGetDevice(&c->device);
  Geom& g = c->g;
  for (int k = 0; k < 4; ++k) g.L[k] = dims[k];
  g.stride[3] = 1;
  g.stride[2] = dims[3];
  g.stride[1] = dims[3] * dims[2];
  g.stride[0] = dims[3] * dims[2] * dims[1];
  g.Vh = (int)c->Vh;
  g.apbc = antiperiodic_t ? 1 : 0;
  g.even_only = 0;
  geom_set_divisors(g);
  // ND_GRAPHS=0: run the Krylov iterations as host-issued launches instead of captured graphs (a
  // profiler cannot see the kernel nodes of a graph with a conditional while-loop)
  if (const char* e = std::getenv("ND_GRAPHS")) c->graphs_ok = std::atoi(e) != 0;
  c->max_blocks = (int)((V + 15) / 16) + 1024;  // >= blocks of any reducing launch (64 sites per block at least)
  bool ok = cudaMalloc(&c->red_partials, sizeof(double) * 8 * c->max_blocks) == cudaSuccess &&
            cudaMalloc(&c->red_counter, sizeof(unsigned) * 16) == cudaSuccess &&
            cudaMalloc(&c->red_scratch, sizeof(double) * 64) == cudaSuccess &&
            cudaMallocHost(&c->host_pinned, sizeof(double) * ND_PINNED_DOUBLES) == cudaSuccess &&
            cudaMemset(c->red_counter, 0, sizeof(unsigned) * 16) == cudaSuccess &&
            cudaMemset(c->red_scratch, 0, sizeof(double) * 64) == cudaSuccess &&
            cudaEventCreate(&c->ev[0]) == cudaSuccess && cudaEventCreate(&c->ev[1]) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    nd_destroy(c);
    return ND_ERR_OOM;
  }
  *out = c;
  return ND_OK;
}

void nd_destroy(nd_ctx* c) {
  if (!c) return;
  if (c->stream || true) cudaStreamSynchronize(c->stream);
  for (int k = 0; k < 3; ++k)
    if (c->links[k]) cudaFree(c->links[k]);
  for (auto& gr : c->ms_graphs) {
    if (gr.exec) cudaGraphExecDestroy(gr.exec);
    if (gr.graph) cudaGraphDestroy(gr.graph);
  }
  if (c->aux_stream) {
    cudaStreamSynchronize(c->aux_stream);
    cudaStreamDestroy(c->aux_stream);
  }
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->join_ev) cudaEventDestroy(c->join_ev);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (auto& kv : c->ws) cudaFree(kv.second.first);
  if (c->evecs) cudaFree(c->evecs);
  if (c->red_partials) cudaFree(c->red_partials);
  if (c->red_counter) cudaFree(c->red_counter);
  if (c->red_scratch) cudaFree(c->red_scratch);
  if (c->host_pinned) cudaFreeHost(c->host_pinned);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  cudaGetLastError();
  delete c;
}

nd_status nd_set_stream(nd_ctx* c, void* stream) {
  ND_TRY(check_ctx(c));
  c->stream = static_cast<cudaStream_t>(stream);
  return ND_OK;
}

nd_status nd_set_links(nd_ctx* c, const double* U, const int recon[3]) {
  ND_TRY(check_ctx(c));
  if (!U || !recon) return fail(c, ND_ERR_INVALID_ARG, "nd_set_links: null pointer");
  for (int p = 0; p < 3; ++p)
    if (recon[p] != 0 && recon[p] != 8 && recon[p] != 12 && recon[p] != 18)
      return fail(c, ND_ERR_INVALID_ARG, "nd_set_links: recon must be 0, 8, 12 or 18");
  int* bad = reinterpret_cast<int*>(workspace(c, "recon8_flag", sizeof(int)));
  if (!bad) return fail(c, ND_ERR_OOM, "nd_set_links: workspace");
  for (int p = 0; p < 3; ++p) {
    if (c->links[p]) {
      ND_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
      cudaFree(c->links[p]);
      c->links[p] = nullptr;
      c->recon[p] = 0;
    }
    if (!recon[p]) continue;
    const int64_t bytes = link_bytes(p, recon[p], c->Vh);
    if (cudaMalloc(&c->links[p], bytes) != cudaSuccess) {
      cudaGetLastError();
      c->links[p] = nullptr;
      return fail(c, ND_ERR_OOM, "nd_set_links: cudaMalloc of the link field");
    }
    ND_TRY_CUDA(c, cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
    ND_TRY_CUDA(c, launch_pack_links(c->g, p, recon[p], c->links[p], U, bad, c->stream));
    if (recon[p] == 8) {
      int h = 0;
      ND_TRY_CUDA(c, cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
      ND_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
      if (h) {
        cudaFree(c->links[p]);
        c->links[p] = nullptr;
        return fail(c, ND_ERR_INVALID_ARG,
                    "nd_set_links: a link lies in the singular set of the 8-real form (|a1| = 1); use 12 or 18");
      }
    }
    c->recon[p] = recon[p];
  }
  return ND_OK;
}

nd_status nd_pack_spinor(nd_ctx* c, void* internal, const double* canon, nd_prec prec, int nrhs) {
  ND_TRY(check_ctx(c));
  if (!internal || !canon || nrhs < 1 || prec < ND_FP64 || prec > ND_FP16)
    return fail(c, ND_ERR_INVALID_ARG, "nd_pack_spinor: bad argument");
  const size_t sb = nd_spinor_bytes(c, prec);
  for (int k = 0; k < nrhs; ++k)
    ND_TRY_CUDA(c, launch_pack_spinor(c->g, (int)prec, static_cast<char*>(internal) + k * sb, canon + k * c->V * 24,
                                      c->stream));
  return ND_OK;
}

nd_status nd_unpack_spinor(nd_ctx* c, double* canon, const void* internal, nd_prec prec, int nrhs) {
  ND_TRY(check_ctx(c));
  if (!internal || !canon || nrhs < 1 || prec < ND_FP64 || prec > ND_FP16)
    return fail(c, ND_ERR_INVALID_ARG, "nd_unpack_spinor: bad argument");
  const size_t sb = nd_spinor_bytes(c, prec);
  for (int k = 0; k < nrhs; ++k)
    ND_TRY_CUDA(c, launch_unpack_spinor(c->g, (int)prec, canon + k * c->V * 24,
                                        static_cast<const char*>(internal) + k * sb, c->stream));
  return ND_OK;
}

nd_status nd_pack_spinor_f32(nd_ctx* c, void* internal, const float* canon, nd_prec prec, int nrhs) {
  ND_TRY(check_ctx(c));
  if (!internal || !canon || nrhs < 1 || prec < ND_FP64 || prec > ND_FP16)
    return fail(c, ND_ERR_INVALID_ARG, "nd_pack_spinor_f32: bad argument");
  const size_t sb = nd_spinor_bytes(c, prec);
  for (int k = 0; k < nrhs; ++k)
    ND_TRY_CUDA(c, launch_pack_spinor_f32(c->g, (int)prec, static_cast<char*>(internal) + k * sb,
                                          canon + k * c->V * 24, c->stream));
  return ND_OK;
}

nd_status nd_unpack_spinor_f32(nd_ctx* c, float* canon, const void* internal, nd_prec prec, int nrhs) {
  ND_TRY(check_ctx(c));
  if (!internal || !canon || nrhs < 1 || prec < ND_FP64 || prec > ND_FP16)
    return fail(c, ND_ERR_INVALID_ARG, "nd_unpack_spinor_f32: bad argument");
  const size_t sb = nd_spinor_bytes(c, prec);
  for (int k = 0; k < nrhs; ++k)
    ND_TRY_CUDA(c, launch_unpack_spinor_f32(c->g, (int)prec, canon + k * c->V * 24,
                                            static_cast<const char*>(internal) + k * sb, c->stream));
  return ND_OK;
}

nd_status nd_eo_tables(nd_ctx* c, int32_t* lex2eo, int32_t* nbr) {
  ND_TRY(check_ctx(c));
  if (!lex2eo || !nbr) return fail(c, ND_ERR_INVALID_ARG, "nd_eo_tables: null pointer");
  ND_TRY_CUDA(c, launch_eo_tables(c->g, lex2eo, nbr, c->stream));
  return ND_OK;
}

nd_status nd_apply_Q(nd_ctx* c, void* out, const void* in, nd_prec prec, int nrhs) {
  ND_TRY(check_ctx(c));
  if (!out || !in || nrhs < 1 || prec < ND_FP64 || prec > ND_FP16)
    return fail(c, ND_ERR_INVALID_ARG, "nd_apply_Q: bad argument");
  if (out == in) return fail(c, ND_ERR_INVALID_ARG, "nd_apply_Q: out and in must not overlap");
  if (!c->links[prec]) return fail(c, ND_ERR_STATE, "nd_apply_Q: no links set in this precision");
  const size_t sb = nd_spinor_bytes(c, prec);
  const char* ib = static_cast<const char*>(in);
  const char* ob = static_cast<const char*>(out);
  if (ib < ob + nrhs * sb && ob < ib + nrhs * sb)
    return fail(c, ND_ERR_INVALID_ARG, "nd_apply_Q: out and in must not overlap");
  QLaunch L{};
  L.prec = (int)prec;
  L.recon = c->recon[prec];
  L.mode = Q_PLAIN;
  L.reduce = false;
  L.links = c->links[prec];
  L.in = in;
  L.out = out;
  L.y = nullptr;
  L.diag = 4.0 + c->m;
  L.a = 1.0;
  L.b = 0.0;
  L.parity0 = 0;
  L.nsites = (int)c->V;
  if (nrhs > 1) {  // one launch for all RHS, links read once
    L.mode = Q_MRHS;
    L.nrhs = nrhs;
    L.rhs_stride = (int64_t)sb;
    L.split = 1;
  }
  ND_TRY_CUDA(c, autotune_launch(c->g, L, c->stream));
  ND_TRY_CUDA(c, launch_q(c->g, L, c->stream));
  return ND_OK;
}

nd_status nd_apply_Q_parity(nd_ctx* c, void* out, const void* in, nd_prec prec, int parity, double diag_coef) {
  ND_TRY(check_ctx(c));
  if (!out || !in || (parity != 0 && parity != 1) || prec < ND_FP64 || prec > ND_FP16)
    return fail(c, ND_ERR_INVALID_ARG, "nd_apply_Q_parity: bad argument");
  if (out == in) return fail(c, ND_ERR_INVALID_ARG, "nd_apply_Q_parity: out and in must not overlap");
  if (!c->links[prec]) return fail(c, ND_ERR_STATE, "nd_apply_Q_parity: no links set in this precision");
  QLaunch L{};
  L.prec = (int)prec;
  L.recon = c->recon[prec];
  L.mode = Q_PLAIN;
  L.links = c->links[prec];
  L.in = in;
  L.out = out;
  L.diag = diag_coef;
  L.a = 1.0;
  L.parity0 = parity;
  L.nsites = (int)c->Vh;
  ND_TRY_CUDA(c, autotune_launch(c->g, L, c->stream));
  ND_TRY_CUDA(c, launch_q(c->g, L, c->stream));
  return ND_OK;
}

nd_status nd_apply_Q_batched(nd_ctx* const* ctxs, int nlat, void* const* out, const void* const* in, const int* nrhs,
                             nd_prec prec, void* stream) {
  if (!ctxs || nlat < 1 || nlat > ND_MAX_BATCH || !out || !in || !nrhs || prec < ND_FP64 || prec > ND_FP16)
    return ND_ERR_INVALID_ARG;
  nd_ctx* c0 = ctxs[0];
  ND_TRY(check_ctx(c0));
  std::vector<LatticeWork> w(nlat);
  int total = 0;
  for (int k = 0; k < nlat; ++k) {
    nd_ctx* c = ctxs[k];
    ND_TRY(check_ctx(c));
    if (!out[k] || !in[k] || nrhs[k] < 1) return fail(c0, ND_ERR_INVALID_ARG, "nd_apply_Q_batched: bad field");
    if (!c->links[prec] || c->recon[prec] != c0->recon[prec])
      return fail(c0, ND_ERR_STATE, "nd_apply_Q_batched: every lattice needs links in prec with the same form");
    const size_t sb = nd_spinor_bytes(c, prec);
    const char* ib = static_cast<const char*>(in[k]);
    const char* ob = static_cast<const char*>(out[k]);
    if (ib < ob + nrhs[k] * sb && ob < ib + nrhs[k] * sb)
      return fail(c0, ND_ERR_INVALID_ARG, "nd_apply_Q_batched: out and in must not overlap");
    w[k].g = c->g;
    w[k].links = static_cast<const char*>(c->links[prec]);
    w[k].in = in[k];
    w[k].out = out[k];
    w[k].stride = (int64_t)sb;
    w[k].nrhs = nrhs[k];
    w[k].tile_begin = total;
    w[k].diag = 4.0 + c->m;
    const int64_t tiles = (int64_t)batched_tiles(c->V) * nrhs[k];
    if (total + tiles > (int64_t)1 << 30) return fail(c0, ND_ERR_INVALID_ARG, "nd_apply_Q_batched: too much work");
    total += (int)tiles;
  }
  LatticeWork* wd = static_cast<LatticeWork*>(workspace(c0, "batched_work", sizeof(LatticeWork) * nlat));
  if (!wd) return fail(c0, ND_ERR_OOM, "nd_apply_Q_batched: workspace");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ND_TRY_CUDA(c0, cudaMemcpyAsync(wd, w.data(), sizeof(LatticeWork) * nlat, cudaMemcpyHostToDevice, st));
  int sms = 0;
  ND_TRY_CUDA(c0, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c0->device));
  const int grid = std::min(total, sms * 8);
  ND_TRY_CUDA(c0, launch_q_batched((int)prec, c0->recon[prec], wd, nlat, total, grid, st));
  return ND_OK;
}

nd_status nd_apply_Q_canonical(nd_ctx* c, double* out, const double* in) {
  ND_TRY(check_ctx(c));
  if (!out || !in) return fail(c, ND_ERR_INVALID_ARG, "nd_apply_Q_canonical: null pointer");
  const size_t sb = nd_spinor_bytes(c, ND_FP64);
  void* a = workspace(c, "canon_a", sb);
  void* b = workspace(c, "canon_b", sb);
  if (!a || !b) return fail(c, ND_ERR_OOM, "nd_apply_Q_canonical: workspace");
  ND_TRY(nd_pack_spinor(c, a, in, ND_FP64, 1));
  ND_TRY(nd_apply_Q(c, b, a, ND_FP64, 1));
  ND_TRY(nd_unpack_spinor(c, out, b, ND_FP64, 1));
  return ND_OK;
}

}  // extern "C"
