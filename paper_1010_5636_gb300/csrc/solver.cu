// Host control of the Krylov solvers: the multi-shift CG driver (device-resident scalars, a
// status read-back every few iterations), FP64 residuals, the mixed-precision defect
// correction, a Hermitian Jacobi eigensolver for the small projected problems, and nd_solve.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>

#include "solver.h"

namespace nd {

nd_status q_apply(nd_ctx* c, int prec, void* out, const void* in, double a, double b, const void* y, double* result,
                  const double* cgs, const void* z, double cz, const void* w, double cw) {
  if (!c->links[prec]) return fail(c, ND_ERR_STATE, "links are not set in the precision this call needs");
  if (w && (!z || result)) return fail(c, ND_ERR_INVALID_ARG, "q_apply: w needs z and no reduction");
  QLaunch L{};
  L.prec = prec;
  L.recon = c->recon[prec];
  L.mode = w ? Q_XPAY3 : (z ? Q_XPAY2 : Q_PLAIN);
  L.w = w;
  L.d = cw;
  L.reduce = result != nullptr;
  L.links = c->links[prec];
  L.in = in;
  L.out = out;
  L.y = y;
  L.z = z;
  L.c = cz;
  L.diag = 4.0 + c->m;
  L.a = a;
  L.b = b;
  L.parity0 = 0;
  L.nsites = (int)c->V;
  if (result) L.slot = slot(c, result);
  L.cgs = cgs;
  ND_TRY_CUDA(c, launch_q(c->g, L, c->stream));
  return ND_OK;
}

void* field(nd_ctx* c, const char* name, int prec, int count) {
  return workspace(c, name, (size_t)spinor_bytes(prec, c->Vh) * (size_t)count);
}

nd_status read_back_on(nd_ctx* c, cudaStream_t st, const double* dev, double* host, int n) {
  for (int k0 = 0; k0 < n; k0 += ND_PINNED_DOUBLES) {
    const int k = std::min(ND_PINNED_DOUBLES, n - k0);
    ND_TRY_CUDA(c, cudaMemcpyAsync(c->host_pinned, dev + k0, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    ND_TRY_CUDA(c, cudaStreamSynchronize(st));
    std::copy(c->host_pinned, c->host_pinned + k, host + k0);
  }
  return ND_OK;
}

nd_status read_back(nd_ctx* c, const double* dev, double* host, int n) { return read_back_on(c, c->stream, dev, host, n); }

// One multi-shift CG iteration (K1..K4, see mscg.cu) launched on stream st; with graph != null
// the scalar kernel also drives the graph's while-loop condition.
static cudaError_t ms_iteration(nd_ctx* c, cudaStream_t st, int ps, int px, bool ymode, void* r, void* t, char* p_all,
                                size_t fs, void* x_or_y, size_t fx, double* state, int n, int maxit,
                                const cudaGraphConditionalHandle* graph) {
  QLaunch L1{};
  L1.prec = ps;
  L1.recon = c->recon[ps];
  L1.mode = Q_PLAIN;
  L1.reduce = true;
  L1.links = c->links[ps];
  L1.in = p_all;
  L1.out = t;
  L1.diag = 4.0 + c->m;
  L1.a = 1.0;
  L1.nsites = (int)c->V;
  L1.slot = slot(c, state + CG_TT);
  L1.cgs = state;
  cudaError_t e = launch_q(c->g, L1, st);
  if (e != cudaSuccess) return e;
  QLaunch L2 = L1;
  L2.mode = Q_CGUPDATE;
  L2.in = t;
  L2.out = r;
  L2.y = p_all;
  L2.slot = slot(c, state + CG_RRNEW);
  e = launch_q(c->g, L2, st);
  if (e != cudaSuccess) return e;
  e = graph ? mscg_scalar_graph(state, n, maxit, *graph, st) : mscg_scalar(state, n, maxit, st);
  if (e != cudaSuccess) return e;
  return mscg_update(c->g, ps, px, ymode, r, p_all, fs, ymode ? nullptr : x_or_y, fx, ymode ? x_or_y : nullptr,
                     state, n, st);
}

// Find or capture the graph of a solve with these buffers; null if graphs are unavailable.
static nd_ms_graph* ms_graph(nd_ctx* c, int ps, int px, bool ymode, void* r, void* t, char* p_all, size_t fs,
                             void* x_or_y, size_t fx, double* state, int n, int maxit) {
  if (!c->graphs_ok) return nullptr;
  for (auto& gr : c->ms_graphs)
    if (gr.kind == 0 && gr.ps == ps && gr.px == px && gr.ymode == (int)ymode && gr.n == n && gr.maxit == maxit &&
        gr.r == r && gr.t == t && gr.p == p_all && gr.x == x_or_y && gr.state == state && gr.links == c->links[ps])
      return &gr;
  nd_ms_graph G;
  G.ps = ps, G.px = px, G.ymode = ymode, G.n = n, G.maxit = maxit;
  G.r = r, G.t = t, G.p = p_all, G.x = x_or_y, G.state = state, G.links = c->links[ps];
  bool ok = true;
  cudaGraphConditionalHandle h{};
  cudaGraphNode_t node;
  // cudaGraphNodeParams has no default constructor (a union of parameter blocks): zeroed storage
  alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
  memset(cp_raw, 0, sizeof(cp_raw));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
  ok = ok && cudaGraphCreate(&G.graph, 0) == cudaSuccess;
  ok = ok && cudaGraphConditionalHandleCreate(&h, G.graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  if (ok) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    ok = cudaGraphAddNode(&node, G.graph, nullptr, nullptr, 0, &cp) == cudaSuccess;
  }
  if (ok && !c->cap_stream) ok = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
  if (ok) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    ok = cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
         cudaSuccess;
    if (ok) {
      const cudaError_t e1 = ms_iteration(c, c->cap_stream, ps, px, ymode, r, t, p_all, fs, x_or_y, fx, state, n,
                                          maxit, &h);
      const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &body);
      ok = e1 == cudaSuccess && e2 == cudaSuccess;
    }
  }
  ok = ok && cudaGraphInstantiate(&G.exec, G.graph, 0) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
    c->graphs_ok = false;  // fall back to launches from the host from now on
    return nullptr;
  }
  if (c->ms_graphs.size() >= 32) {
    cudaGraphExecDestroy(c->ms_graphs.front().exec);
    cudaGraphDestroy(c->ms_graphs.front().graph);
    c->ms_graphs.erase(c->ms_graphs.begin());
  }
  c->ms_graphs.push_back(G);
  return &c->ms_graphs.back();
}

nd_status mscg_run(nd_ctx* c, int ps, int px, bool ymode, const void* b, void* x_or_y, const std::vector<double>& sigma,
                   const std::vector<double>& tol, const std::vector<double>& w, double ascale, int maxit,
                   MsResult* out) {
  NvtxRange range("nd.multishift_cg");
  const int n = (int)sigma.size();
  if (n < 1 || n > CG_NMAX) return fail(c, ND_ERR_INVALID_ARG, "multi-shift CG: 1..32 shifts");
  const size_t fs = (size_t)spinor_bytes(ps, c->Vh);
  const size_t fx = (size_t)spinor_bytes(px, c->Vh);
  void* r = field(c, "ms_r", ps);
  void* t = field(c, "ms_t", ps);
  char* p_all = static_cast<char*>(field(c, "ms_p", ps, n));
  double* state = static_cast<double*>(workspace(c, "ms_state", sizeof(double) * CG_STATE_DOUBLES));
  if (!r || !t || !p_all || !state) return fail(c, ND_ERR_OOM, "multi-shift CG: workspace");
  // state: shifts, tolerances, weights, ascale
  std::vector<double> h(CG_STATE_DOUBLES, 0.0);
  for (int l = 0; l < n; ++l) {
    h[sh(SH_SIGMA, l)] = sigma[l];
    h[sh(SH_TOL, l)] = tol[l];
    h[sh(SH_W, l)] = w.empty() ? 0.0 : w[l];
  }
  h[CG_ASCALE] = ascale;
  ND_TRY_CUDA(c, cudaMemcpyAsync(state, h.data(), sizeof(double) * CG_STATE_DOUBLES, cudaMemcpyHostToDevice, c->stream));
  // r = b, p_l = b, x = 0 (or y = 0), RR = ||b||^2
  ND_TRY_CUDA(c, blas_axpby(c->g, ps, r, 1.0, b, 0.0, nullptr, true, slot(c, state + CG_RR), c->stream));
  for (int l = 0; l < n; ++l) ND_TRY_CUDA(c, cudaMemcpyAsync(p_all + l * fs, b, fs, cudaMemcpyDeviceToDevice, c->stream));
  ND_TRY_CUDA(c, cudaMemsetAsync(x_or_y, 0, ymode ? fx : fx * n, c->stream));
  ND_TRY_CUDA(c, mscg_init(state, n, c->stream));
  double hs[CG_NSCALAR];
  if (!c->links[ps]) return fail(c, ND_ERR_STATE, "multi-shift CG: links not set in the Krylov precision");
  nd_ms_graph* G = ms_graph(c, ps, px, ymode, r, t, p_all, fs, x_or_y, fx, state, n, maxit);
  ND_TRY_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
  if (G) {
    // the whole solve is one graph launch: the iterations loop on the device until the scalar
    // kernel ends the while-loop
    ND_TRY_CUDA(c, cudaGraphLaunch(G->exec, c->stream));
    ND_TRY_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
    ND_TRY(read_back(c, state, hs, CG_NSCALAR));
  } else {
    int chunk = 8;
    for (;;) {
      for (int k = 0; k < chunk; ++k)
        ND_TRY_CUDA(c, ms_iteration(c, c->stream, ps, px, ymode, r, t, p_all, fs, x_or_y, fx, state, n, maxit,
                                    nullptr));
      ND_TRY(read_back(c, state, hs, CG_NSCALAR));
      if (hs[CG_DONE] != 0.0 || hs[CG_PENDING] != 0.0) break;
      chunk = std::min(chunk * 2, 64);
    }
    ND_TRY_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
  }
  std::vector<double> res(n);
  ND_TRY(read_back(c, state + sh(SH_RES, 0), res.data(), n));
  if (out) {
    out->iters = (int)hs[CG_ITER];
    out->status = (int)hs[CG_STATUS];
    out->res = res;
    float ms = 0.f;
    ND_TRY_CUDA(c, cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
    out->ms = ms;
    out->live = hs[CG_LIVE_SUM];
    out->active = hs[CG_ACTIVE_SUM];
  }
  const int stt = (int)hs[CG_STATUS];
  if (stt != ND_OK) {
    const char* what = stt == ND_ERR_NOT_CONVERGED ? "multi-shift CG: iteration limit reached"
                       : stt == ND_ERR_BREAKDOWN   ? "multi-shift CG: breakdown, (p, A p) <= 0"
                                                   : "multi-shift CG: NaN or Inf";
    return fail(c, (nd_status)stt, what);
  }
  return ND_OK;
}

// ------------------------------------------------------------------ batched CG
// One iteration of nsys independent shifted CG systems (fields at + s * fs) on stream st.
static cudaError_t bcg_iteration(nd_ctx* c, cudaStream_t st, int ps, char* r, char* t, char* p, char* x, size_t fs,
                                 double* states, double* partials, unsigned* counters, int nsys, int maxit,
                                 const cudaGraphConditionalHandle* h) {
  QLaunch L1{};
  L1.prec = ps;
  L1.recon = c->recon[ps];
  L1.mode = Q_BPLAIN;
  L1.reduce = true;
  L1.links = c->links[ps];
  L1.in = p;
  L1.out = t;
  L1.diag = 4.0 + c->m;
  L1.a = 1.0;
  L1.nsites = (int)c->V;
  L1.nrhs = nsys;
  L1.rhs_stride = (int64_t)fs;
  L1.cgs = states;
  L1.cgs_stride = CG_STATE_DOUBLES;
  L1.slot.partials = partials;
  L1.slot.counter = counters;
  L1.slot.result = states + CG_TT;
  cudaError_t e = launch_q(c->g, L1, st);
  if (e != cudaSuccess) return e;
  QLaunch L2 = L1;
  L2.mode = Q_BCG;
  L2.in = t;
  L2.out = r;
  L2.y = p;
  L2.slot.result = states + CG_RRNEW;
  e = launch_q(c->g, L2, st);
  if (e != cudaSuccess) return e;
  e = bcg_scalar(states, nsys, maxit, h, st);
  if (e != cudaSuccess) return e;
  return bcg_update(c->g, ps, r, p, x, fs, states, nsys, st);
}

// Solve (ascale Q^2 + sigma_s) x_s = b_s for s < nsys (independent systems run in lockstep: one
// multi-RHS Q launch per step for all of them).  b, x: nsys consecutive fields of precision ps.
// bcg_start issues the solve on `stream` with workspaces named after `tag` (two solves with
// different tags may run at the same time on different streams: they share no buffer, counter or
// reduction scratch); with graphs the iterations run on the device and bcg_finish reads the result
// back, without graphs the host loop runs inside bcg_start.
nd_status bcg_start(nd_ctx* c, int ps, const void* b, void* x, const std::vector<double>& sigma,
                    const std::vector<double>& tol, double ascale, int maxit, const std::string& tag,
                    cudaStream_t stream, BcgJob* job) {
  NvtxRange range("nd.batched_cg");
  const int nsys = (int)sigma.size();
  if (nsys < 1 || nsys > ND_BATCH_MAX_SYSTEMS) return fail(c, ND_ERR_INVALID_ARG, "batched CG: 1..1024 systems");
  if (!c->links[ps]) return fail(c, ND_ERR_STATE, "batched CG: links not set in the Krylov precision");
  const size_t fs = (size_t)spinor_bytes(ps, c->Vh);
  char* r = static_cast<char*>(field(c, (tag + "_r").c_str(), ps, nsys));
  char* t = static_cast<char*>(field(c, (tag + "_t").c_str(), ps, nsys));
  char* p = static_cast<char*>(field(c, (tag + "_p").c_str(), ps, nsys));
  double* states = static_cast<double*>(workspace(c, tag + "_state", sizeof(double) * CG_STATE_DOUBLES * nsys));
  double* partials =
      static_cast<double*>(workspace(c, tag + "_partials", sizeof(double) * bcg_partials(c->g, ps, nsys)));
  // one counter per system for the batched launches, one more for the set-up reductions
  unsigned* counters = static_cast<unsigned*>(workspace(c, tag + "_counters", sizeof(unsigned) * (nsys + 1)));
  if (!r || !t || !p || !states || !partials || !counters) return fail(c, ND_ERR_OOM, "batched CG: workspace");
  std::vector<double> h((size_t)CG_STATE_DOUBLES * nsys, 0.0);
  for (int s = 0; s < nsys; ++s) {
    double* hs = h.data() + (size_t)s * CG_STATE_DOUBLES;
    hs[sh(SH_SIGMA, 0)] = sigma[s];
    hs[sh(SH_TOL, 0)] = tol[s];
    hs[CG_ASCALE] = ascale;
  }
  ND_TRY_CUDA(c, cudaMemcpyAsync(states, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, stream));
  ND_TRY_CUDA(c, cudaMemsetAsync(counters, 0, sizeof(unsigned) * (nsys + 1), stream));
  ND_TRY_CUDA(c, cudaMemcpyAsync(p, b, fs * nsys, cudaMemcpyDeviceToDevice, stream));
  ND_TRY_CUDA(c, cudaMemsetAsync(x, 0, fs * nsys, stream));
  for (int s = 0; s < nsys; ++s) {
    ReduceSlot rs;
    rs.partials = partials;
    rs.counter = counters + nsys;
    rs.result = states + (size_t)s * CG_STATE_DOUBLES + CG_RR;
    ND_TRY_CUDA(c, blas_axpby(c->g, ps, r + s * fs, 1.0, static_cast<const char*>(b) + s * fs, 0.0, nullptr, true, rs,
                              stream));
  }
  ND_TRY_CUDA(c, bcg_init(states, nsys, stream));
  job->nsys = nsys;
  job->states = states;
  job->stream = stream;
  // graph: a device while-loop over the iterations, reused while the buffers are the same
  nd_ms_graph* G = nullptr;
  if (c->graphs_ok) {
    for (auto& gr : c->ms_graphs)
      if (gr.kind == 1 && gr.ps == ps && gr.n == nsys && gr.maxit == maxit && gr.r == r && gr.t == t && gr.p == p &&
          gr.x == x && gr.state == states && gr.links == c->links[ps])
        G = &gr;
    if (!G) {
      nd_ms_graph NG;
      NG.kind = 1, NG.ps = ps, NG.n = nsys, NG.maxit = maxit;
      NG.r = r, NG.t = t, NG.p = p, NG.x = x, NG.state = states, NG.links = c->links[ps];
      bool ok = true;
      cudaGraphConditionalHandle hc{};
      cudaGraphNode_t node;
      alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
      memset(cp_raw, 0, sizeof(cp_raw));
      cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
      ok = ok && cudaGraphCreate(&NG.graph, 0) == cudaSuccess;
      ok = ok && cudaGraphConditionalHandleCreate(&hc, NG.graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
      if (ok) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = hc;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ok = cudaGraphAddNode(&node, NG.graph, nullptr, nullptr, 0, &cp) == cudaSuccess;
      }
      if (ok && !c->cap_stream) ok = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
      if (ok) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        ok = cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
          const cudaError_t e1 =
              bcg_iteration(c, c->cap_stream, ps, r, t, p, static_cast<char*>(x), fs, states, partials, counters,
                            nsys, maxit, &hc);
          const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &body);
          ok = e1 == cudaSuccess && e2 == cudaSuccess;
        }
      }
      ok = ok && cudaGraphInstantiate(&NG.exec, NG.graph, 0) == cudaSuccess;
      if (!ok) {
        cudaGetLastError();
        if (NG.exec) cudaGraphExecDestroy(NG.exec);
        if (NG.graph) cudaGraphDestroy(NG.graph);
        c->graphs_ok = false;
      } else {
        if (c->ms_graphs.size() >= 32) {
          cudaGraphExecDestroy(c->ms_graphs.front().exec);
          cudaGraphDestroy(c->ms_graphs.front().graph);
          c->ms_graphs.erase(c->ms_graphs.begin());
        }
        c->ms_graphs.push_back(NG);
        G = &c->ms_graphs.back();
      }
    }
  }
  if (G) {
    ND_TRY_CUDA(c, cudaGraphLaunch(G->exec, stream));
    return ND_OK;
  }
  std::vector<double> hs((size_t)CG_STATE_DOUBLES * nsys);
  int chunk = 8;
  for (;;) {
    for (int k = 0; k < chunk; ++k)
      ND_TRY_CUDA(c, bcg_iteration(c, stream, ps, r, t, p, static_cast<char*>(x), fs, states, partials, counters, nsys,
                                   maxit, nullptr));
    ND_TRY(read_back_on(c, stream, states, hs.data(), (int)hs.size()));
    bool all = true;
    for (int s = 0; s < nsys; ++s) {
      const double* q = hs.data() + (size_t)s * CG_STATE_DOUBLES;
      if (q[CG_DONE] == 0.0 && q[CG_PENDING] == 0.0) all = false;
    }
    if (all) break;
    chunk = std::min(chunk * 2, 64);
  }
  return ND_OK;
}

nd_status bcg_finish(nd_ctx* c, BcgJob* job, std::vector<int>* iters) {
  const int nsys = job->nsys;
  std::vector<double> hs((size_t)CG_STATE_DOUBLES * nsys);
  ND_TRY(read_back_on(c, job->stream, job->states, hs.data(), (int)hs.size()));
  if (iters) iters->assign(nsys, 0);
  for (int s = 0; s < nsys; ++s) {
    const double* q = hs.data() + (size_t)s * CG_STATE_DOUBLES;
    if (iters) (*iters)[s] = (int)q[CG_ITER];
    const int stt = (int)q[CG_STATUS];
    if (stt != ND_OK && stt != ND_ERR_NOT_CONVERGED)
      return fail(c, (nd_status)stt, stt == ND_ERR_BREAKDOWN ? "batched CG: breakdown" : "batched CG: NaN or Inf");
  }
  return ND_OK;
}

nd_status residual64_dev(nd_ctx* c, void* r, const void* b, const void* x, double sigma, double ascale,
                         double* norm2_dev) {
  void* t = field(c, "res_t", 0);
  if (!t) return fail(c, ND_ERR_OOM, "residual: workspace");
  ND_TRY(q_apply(c, 0, t, x));
  ND_TRY(q_apply(c, 0, r, t, -ascale, -sigma, x, norm2_dev, nullptr, b, 1.0));
  return ND_OK;
}

nd_status residual64(nd_ctx* c, void* r, const void* b, const void* x, double sigma, double ascale, double bnorm2,
                     double* rel) {
  void* t = field(c, "res_t", 0);
  if (!t) return fail(c, ND_ERR_OOM, "residual: workspace");
  double* res = c->red_scratch + 8;
  ND_TRY(q_apply(c, 0, t, x));
  // r = b - (ascale Q^2 + sigma) x in the second launch's epilogue, ||r||^2 reduced with it
  ND_TRY(q_apply(c, 0, r, t, -ascale, -sigma, x, res, nullptr, b, 1.0));
  double h;
  ND_TRY(read_back(c, res, &h, 1));
  *rel = std::sqrt(h / bnorm2);
  return ND_OK;
}

nd_status mixed_solve_impl(nd_ctx* c, int ps, const void* b64, double bnorm2, const std::vector<double>& sigma,
                           const std::vector<double>& tol, double ascale, int maxit, MixedStats* st,
                           nd_status (*sink)(void*, int, void*), void* sink_ctx) {
  NvtxRange range("nd.mixed_solve");
  const int n = (int)sigma.size();
  // Sloppy pass: the Krylov vectors in ps, the shifted solutions in FP32.
  // floor_s: where the sloppy multi-shift recurrence stops being trusted; floor_in: the smallest
  // reduction asked of one FP32 correction solve.  ND_MIXED_FLOOR_S / ND_MIXED_FLOOR_IN in the
  // environment override them (tuning).
  // defaults from a grid on 16^3x32 Haar links with 20 deflated modes (D_N to 1e-10): FP32 sloppy
  // floors 1e-5/1e-6/1e-7/3e-8 x correction floors 1e-4/1e-5/1e-6 gave 0.087-0.105 s per D_N, best
  // at (1e-7, 1e-6); FP16 sloppy floors 1e-2/1e-3/1e-4 gave 0.113-0.129 s, best at (1e-4, 1e-6)
  double floor_s = ps == 2 ? 1e-4 : 1e-7;
  double floor_in = 1e-6;
  if (const char* e = std::getenv("ND_MIXED_FLOOR_S")) floor_s = std::atof(e);
  if (const char* e = std::getenv("ND_MIXED_FLOOR_IN")) floor_in = std::atof(e);
  void* bS = field(c, "mx_bS", ps);
  char* x32 = static_cast<char*>(field(c, "mx_x32", 1, n));
  void* r64 = field(c, "mx_r64", 0);
  if (!bS || !x32 || !r64) return fail(c, ND_ERR_OOM, "mixed solve: workspace");
  // Every field handed to the sloppy precision is scaled to unit norm first (and its solution
  // scaled back in FP64): a source or residual of small norm would otherwise reach FP32 products
  // and squared norms in the subnormal range, where the Krylov scalars lose their digits.
  const double bnorm = std::sqrt(bnorm2);
  ND_TRY_CUDA(c, blas_axpby(c->g, 0, r64, 1.0 / bnorm, b64, 0.0, nullptr, false, slot(c, nullptr), c->stream));
  ND_TRY_CUDA(c, blas_convert(c->g, ps, bS, 0, r64, c->stream));
  std::vector<double> tol_s(n);
  for (int l = 0; l < n; ++l) tol_s[l] = std::max(tol[l], floor_s);
  const bool trace = std::getenv("ND_TRACE") != nullptr;
  auto now = [&]() {
    if (trace) cudaStreamSynchronize(c->stream);
    return std::chrono::steady_clock::now();
  };
  auto ms_since = [](std::chrono::steady_clock::time_point t) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t).count();
  };
  double t_res = 0.0, t_bcg = 0.0;
  auto t0 = now();
  MsResult ms;
  nd_status s = mscg_run(c, ps, 1, false, bS, x32, sigma, tol_s, {}, ascale, maxit, &ms);
  if (s != ND_OK) return s;
  if (trace) std::fprintf(stderr, "mixed solve: sloppy multi-shift %d iterations %.2f ms\n", ms.iters, ms_since(t0));
  st->iters = ms.iters;
  st->sloppy_iters = ms.iters;
  st->max_resid = 0.0;
  st->krylov_ms = ms.ms;
  st->live = ms.live;
  st->active = ms.active;
  const auto t_refine = std::chrono::steady_clock::now();
  // FP64 defect correction of every shift, the correction solves of all shifts that still miss
  // their target batched into one lockstep CG (one multi-RHS Q launch per step).  A sweep computes
  // the FP64 residuals of all open shifts back to back, each normalised into its FP32 correction
  // source on the device, and reads their norms back once.
  const size_t f32 = (size_t)spinor_bytes(1, c->Vh), f64 = (size_t)spinor_bytes(0, c->Vh);
  char* X64 = static_cast<char*>(field(c, "mx_X64", 0, n));
  char* R32 = static_cast<char*>(field(c, "mx_R32", 1, n));
  char* E32 = static_cast<char*>(field(c, "mx_E32", 1, n));
  // [2l, 2l + 1]: ||r_l||^2 and the residual launch's second norm; [2 CG_NMAX + l]: ||x_l||^2
  double* nrm = static_cast<double*>(workspace(c, "mx_norms", sizeof(double) * 3 * CG_NMAX));
  if (!X64 || !R32 || !E32 || !nrm) return fail(c, ND_ERR_OOM, "mixed solve: workspace");
  for (int l = 0; l < n; ++l) {
    ND_TRY_CUDA(c, blas_convert(c->g, 0, X64 + l * f64, 1, x32 + l * f32, c->stream));
    ND_TRY_CUDA(c, blas_axpby(c->g, 0, X64 + l * f64, bnorm, X64 + l * f64, 0.0, nullptr, false, slot(c, nullptr),
                              c->stream));
  }
  std::vector<double> rel(n, 1.0), first(n, -1.0), prev(n, 1e300);
  // per-shift reduction asked of a correction solve; raised tenfold (up to 1e-2) after a correction
  // that ran into its iteration cap: an FP32 CG resolves relative reductions down to about
  // u_32 kappa, which the lowest shifts of a deflated system only just clear
  std::vector<double> tin(n, floor_in), rnorm(n, 1.0), h(3 * CG_NMAX, 0.0), tol_p(n, 1.0);
  std::vector<int> outer(n, 0), flat(n, 0);
  std::vector<bool> done(n, false);
  // a correction asks for a modest reduction; needing many more iterations than the sloppy pass
  // means it is stuck on rounding, and the next FP64 residual decides (rounded up to a power of two:
  // the captured graph is keyed by the limit)
  int cap = 128;
  while (cap < 8 * st->iters + 100) cap *= 2;
  const int bmax = std::min(maxit, cap);
  // FP64 residuals of the open shifts in [lo, hi) on the context's stream, their norms read back
  // once; sets tol_p and *npend (the shifts that need another correction)
  auto residual_sweep = [&](int lo, int hi, int* npend) -> nd_status {
    auto tr = now();
    for (int l = lo; l < hi; ++l) {
      if (done[l]) continue;
      // r = b - (ascale Q^2 + sigma_l) x_l in FP64, ||r||^2 -> nrm[l]; R32_l = r / ||r||
      ND_TRY(residual64_dev(c, r64, b64, X64 + l * f64, sigma[l], ascale, nrm + 2 * l));
      ND_TRY_CUDA(c, blas_convert_normalized(c->g, 1, R32 + l * f32, r64, nrm + 2 * l, c->stream));
      if (flat[l] >= 1) {  // ||x_l||^2 for the rounding-floor test below (r64 is free again)
        ND_TRY_CUDA(c, blas_axpby(c->g, 0, r64, 1.0, X64 + l * f64, 0.0, nullptr, true,
                                  slot(c, nrm + 2 * CG_NMAX + l), c->stream));
      }
      ++st->residuals64;
    }
    ND_TRY(read_back(c, nrm, h.data(), 3 * CG_NMAX));
    if (trace) t_res += ms_since(tr);
    *npend = 0;
    for (int l = lo; l < hi; ++l) {
      tol_p[l] = 1.0;
      if (done[l]) continue;
      rel[l] = std::sqrt(h[2 * l] / bnorm2);
      if (first[l] < 0) first[l] = rel[l];
      // A correction that no longer halves the FP64 residual twice in a row means the target lies
      // at or below what an FP64 residual of this system resolves: |fl(b - A x) - (b - A x)| is
      // about u (||b|| + || |A| || ||x||) with ||A|| <= ascale lambda_max + sigma ~ 1 + sigma; the
      // entrywise |Q|^2 exceeds ||Q^2|| about fourfold and each stencil sums ~50 products, so a
      // shift stagnating within 256 u (1 + (1 + sigma) ||x|| / ||b||) is accepted there, with its
      // residual reported; above it the solve fails.
      flat[l] = rel[l] > 0.5 * prev[l] ? flat[l] + 1 : 0;
      prev[l] = rel[l];
      if (rel[l] <= tol[l]) {
        done[l] = true;
      } else if (flat[l] >= 2) {
        // flat[l] >= 2 means it was >= 1 before this sweep, so ||x_l||^2 was reduced above
        const double xn2 = h[2 * CG_NMAX + l];
        const double floor64 = 256.0 * 1.1102230246251565e-16 * (1.0 + (1.0 + sigma[l]) * std::sqrt(xn2 / bnorm2));
        if (rel[l] > floor64) {
          char msg[160];
          std::snprintf(msg, sizeof msg, "mixed solve: shift %d stagnates at relative residual %.3g (target %.3g)",
                        l, rel[l], tol[l]);
          return fail(c, ND_ERR_NOT_CONVERGED, msg);
        }
        done[l] = true;
      } else {
        rnorm[l] = rel[l] * bnorm;
        tol_p[l] = std::max(0.3 * tol[l] / rel[l], tin[l]);
        ++*npend;
      }
      // a shift that is done takes part in the batched solve with a zero source (it stops at once)
      if (done[l]) ND_TRY_CUDA(c, cudaMemsetAsync(R32 + l * f32, 0, f32, c->stream));
    }
    return ND_OK;
  };
  // the correction solves of [lo, hi) as one batched CG on stream stx
  auto correct_start = [&](int lo, int hi, const char* tag, cudaStream_t stx, BcgJob* job) -> nd_status {
    const std::vector<double> sg(sigma.begin() + lo, sigma.begin() + hi), tp(tol_p.begin() + lo, tol_p.begin() + hi);
    return bcg_start(c, 1, R32 + lo * f32, E32 + lo * f32, sg, tp, ascale, bmax, tag, stx, job);
  };
  // x_l += ||r_l|| e_l in FP64 for the open shifts of [lo, hi), after their correction solve
  auto correct_apply = [&](int lo, int hi, const std::vector<int>& it) -> nd_status {
    for (int l = lo; l < hi; ++l) {
      if (done[l]) continue;
      st->sloppy_iters += it[l - lo];
      st->correction_iters += it[l - lo];
      if (it[l - lo] >= bmax) tin[l] = std::min(10.0 * tin[l], 1e-2);
      ++outer[l];
      ND_TRY_CUDA(c, blas_axpy_widen(c->g, X64 + l * f64, rnorm[l], E32 + l * f32, c->stream));
    }
    return ND_OK;
  };
  // sweeps of residuals and corrections over [lo, hi) on the context's stream until every shift there
  // meets its target
  auto refine = [&](int lo, int hi, const char* tag) -> nd_status {
    for (int sweep = 0;; ++sweep) {
      int npend = 0;
      ND_TRY(residual_sweep(lo, hi, &npend));
      if (npend == 0) return ND_OK;
      if (sweep >= 60) return fail(c, ND_ERR_NOT_CONVERGED, "mixed solve: defect correction did not converge");
      auto tb = now();
      BcgJob job;
      std::vector<int> it;
      ND_TRY(correct_start(lo, hi, tag, c->stream, &job));
      ND_TRY(bcg_finish(c, &job, &it));
      if (trace) {
        const double dt = ms_since(tb);
        t_bcg += dt;
        std::fprintf(stderr, "mixed solve: shifts [%d, %d) sweep %d, %d systems, batched CG max %d iterations %.2f ms\n",
                     lo, hi, sweep, npend, *std::max_element(it.begin(), it.end()), dt);
      }
      ND_TRY(correct_apply(lo, hi, it));
    }
  };
  // The lowest shifts need the longest correction solves (the condition number of A + sigma grows as
  // sigma falls), and on a small lattice their lockstep tail leaves the GPU mostly idle.  So the lowest
  // third starts its first correction on a second stream, the other shifts are refined meanwhile on
  // the context's stream (their FP64 residuals and correction solves fill the idle time), and then the
  // lowest third is refined to the end.  Without CUDA graphs the batched CG is driven from the host
  // and nothing overlaps, so the split is skipped.
  // ND_MIXED_LOW in the environment sets the number of shifts in the low group (tuning)
  int ks = (c->graphs_ok && n >= 6) ? (n + 2) / 3 : 0;
  if (const char* e = std::getenv("ND_MIXED_LOW")) ks = (c->graphs_ok && n >= 2) ? std::max(0, std::min(n - 1, std::atoi(e))) : 0;
  if (ks > 0) {
    if (!c->aux_stream) ND_TRY_CUDA(c, cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking));
    if (!c->fork_ev) ND_TRY_CUDA(c, cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
    if (!c->join_ev) ND_TRY_CUDA(c, cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming));
    int npend = 0;
    ND_TRY(residual_sweep(0, ks, &npend));
    BcgJob job;
    if (npend > 0) {
      ND_TRY_CUDA(c, cudaEventRecord(c->fork_ev, c->stream));
      ND_TRY_CUDA(c, cudaStreamWaitEvent(c->aux_stream, c->fork_ev, 0));
      ND_TRY(correct_start(0, ks, "bc_low", c->aux_stream, &job));
    }
    ND_TRY(refine(ks, n, "bc_high"));
    if (npend > 0) {
      std::vector<int> it;
      ND_TRY(bcg_finish(c, &job, &it));
      ND_TRY_CUDA(c, cudaEventRecord(c->join_ev, c->aux_stream));
      ND_TRY_CUDA(c, cudaStreamWaitEvent(c->stream, c->join_ev, 0));
      if (trace)
        std::fprintf(stderr, "mixed solve: shifts [0, %d) first correction (second stream) max %d iterations\n", ks,
                     *std::max_element(it.begin(), it.end()));
      ND_TRY(correct_apply(0, ks, it));
    }
    ND_TRY(refine(0, ks, "bc_low"));
  } else {
    ND_TRY(refine(0, n, "bc_all"));
  }
  st->refine_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_refine).count();
  if (trace)
    std::fprintf(stderr, "mixed solve: FP64 residuals %.2f ms, batched CG %.2f ms, total %.2f ms\n", t_res, t_bcg,
                 ms_since(t0));
  for (int l = 0; l < n; ++l) {
    if (std::getenv("ND_TRACE"))
      std::fprintf(stderr, "mixed solve: shift %d sigma %.3e sloppy resid %.3e outer %d final %.3e\n", l, sigma[l],
                   first[l], outer[l], rel[l]);
    st->outer = std::max(st->outer, outer[l]);
    st->max_resid = std::max(st->max_resid, rel[l]);
    ND_TRY(sink(sink_ctx, l, X64 + l * f64));
  }
  return ND_OK;
}

// ------------------------------------------------------------------ Hermitian Jacobi
void hermitian_eig(int n, std::vector<double>& A, std::vector<double>& evals, std::vector<double>& evecs) {
  auto re = [&](int i, int j) -> double& { return A[2 * (i * n + j)]; };
  auto im = [&](int i, int j) -> double& { return A[2 * (i * n + j) + 1]; };
  std::vector<double> Vm(2 * n * n, 0.0);
  for (int i = 0; i < n; ++i) Vm[2 * (i * n + i)] = 1.0;
  double scale = 0.0;
  for (int i = 0; i < n * n; ++i) scale = std::max(scale, std::hypot(A[2 * i], A[2 * i + 1]));
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += re(p, q) * re(p, q) + im(p, q) * im(p, q);
    if (off <= 1e-34 * scale * scale * n * n || scale == 0.0) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double br = re(p, q), bi = im(p, q);
        const double bm = std::hypot(br, bi);
        if (bm <= 1e-300) continue;
        // D = diag(1, e^{-i phi}) makes the (p, q) entry real and positive; then a real rotation.
        const double cph = br / bm, sph = bi / bm;  // e^{i phi}
        const double app = re(p, p), aqq = re(q, q);
        const double zeta = (aqq - app) / (2.0 * bm);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
        // G = D R with R = [[c, s], [-s, c]]:  G = [[c, s], [-s e^{-i phi}, c e^{-i phi}]]
        // g_pp = c, g_pq = s, g_qp = -s e^{-i phi}, g_qq = c e^{-i phi}
        const double gqp_r = -sn * cph, gqp_i = sn * sph;
        const double gqq_r = cs * cph, gqq_i = -cs * sph;
        // columns: A <- A G
        for (int k = 0; k < n; ++k) {
          const double akp_r = re(k, p), akp_i = im(k, p), akq_r = re(k, q), akq_i = im(k, q);
          re(k, p) = cs * akp_r + (akq_r * gqp_r - akq_i * gqp_i);
          im(k, p) = cs * akp_i + (akq_r * gqp_i + akq_i * gqp_r);
          re(k, q) = sn * akp_r + (akq_r * gqq_r - akq_i * gqq_i);
          im(k, q) = sn * akp_i + (akq_r * gqq_i + akq_i * gqq_r);
          double* v = Vm.data();
          const double vkp_r = v[2 * (k * n + p)], vkp_i = v[2 * (k * n + p) + 1];
          const double vkq_r = v[2 * (k * n + q)], vkq_i = v[2 * (k * n + q) + 1];
          v[2 * (k * n + p)] = cs * vkp_r + (vkq_r * gqp_r - vkq_i * gqp_i);
          v[2 * (k * n + p) + 1] = cs * vkp_i + (vkq_r * gqp_i + vkq_i * gqp_r);
          v[2 * (k * n + q)] = sn * vkp_r + (vkq_r * gqq_r - vkq_i * gqq_i);
          v[2 * (k * n + q) + 1] = sn * vkp_i + (vkq_r * gqq_i + vkq_i * gqq_r);
        }
        // rows: A <- G^dagger A;  (G^dagger)_pk = conj(g_kp), rows p, q mix with conj(G) columns
        for (int k = 0; k < n; ++k) {
          const double apk_r = re(p, k), apk_i = im(p, k), aqk_r = re(q, k), aqk_i = im(q, k);
          // new_p = conj(g_pp) a_p + conj(g_qp) a_q ; new_q = conj(g_pq) a_p + conj(g_qq) a_q
          re(p, k) = cs * apk_r + (gqp_r * aqk_r + gqp_i * aqk_i);
          im(p, k) = cs * apk_i + (gqp_r * aqk_i - gqp_i * aqk_r);
          re(q, k) = sn * apk_r + (gqq_r * aqk_r + gqq_i * aqk_i);
          im(q, k) = sn * apk_i + (gqq_r * aqk_i - gqq_i * aqk_r);
        }
        re(p, q) = im(p, q) = re(q, p) = im(q, p) = 0.0;
        im(p, p) = im(q, q) = 0.0;
      }
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int a, int b) { return re(a, a) < re(b, b); });
  evals.assign(n, 0.0);
  evecs.assign(2 * n * n, 0.0);
  for (int k = 0; k < n; ++k) {
    evals[k] = re(order[k], order[k]);
    for (int i = 0; i < n; ++i) {
      evecs[2 * (i * n + k)] = Vm[2 * (i * n + order[k])];
      evecs[2 * (i * n + k) + 1] = Vm[2 * (i * n + order[k]) + 1];
    }
  }
}

}  // namespace nd

using namespace nd;

extern "C" nd_status nd_solve(nd_ctx* c, double* const* x, const double* b, const double* shifts, int n, double tol,
                              int maxit, nd_prec inner, nd_solve_info* info) {
  if (!c) return ND_ERR_INVALID_ARG;
  if (c->poisoned) return fail(c, ND_ERR_STATE, "context unusable after an earlier CUDA error: " + c->err);
  if (!x || !b || !shifts || n < 1 || n > CG_NMAX || !(tol > 0) || maxit < 1 || inner < ND_FP64 || inner > ND_FP16)
    return fail(c, ND_ERR_INVALID_ARG, "nd_solve: bad argument (1 <= n <= 32, tol > 0, maxit >= 1)");
  for (int k = 0; k < n; ++k)
    if (!x[k] || !(shifts[k] >= 0.0)) return fail(c, ND_ERR_INVALID_ARG, "nd_solve: null x or negative shift");
  if (!c->links[0] || !c->links[inner] || (inner != ND_FP64 && !c->links[1]))
    return fail(c, ND_ERR_STATE, "nd_solve: links must be set in FP64, in the inner precision and (mixed) FP32");
  auto t0 = std::chrono::steady_clock::now();
  std::vector<int> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int bb) { return shifts[a] < shifts[bb]; });
  std::vector<double> sig(n), tols(n, tol);
  for (int l = 0; l < n; ++l) sig[l] = shifts[perm[l]];
  void* b64 = field(c, "solve_b64", 0);
  if (!b64) return fail(c, ND_ERR_OOM, "nd_solve: workspace");
  ND_TRY(nd_pack_spinor(c, b64, b, ND_FP64, 1));
  double bn2;
  ND_TRY_CUDA(c, blas_axpby(c->g, 0, b64, 1.0, b64, 0.0, nullptr, true, slot(c, c->red_scratch), c->stream));
  ND_TRY(read_back(c, c->red_scratch, &bn2, 1));
  nd_solve_info inf{};
  if (bn2 == 0.0) {
    for (int k = 0; k < n; ++k) ND_TRY_CUDA(c, cudaMemsetAsync(x[k], 0, sizeof(double) * 24 * c->V, c->stream));
    if (info) *info = inf;
    return ND_OK;
  }
  if (!std::isfinite(bn2)) return fail(c, ND_ERR_NAN, "nd_solve: source has NaN or Inf");
  nd_status s = ND_OK;
  if (inner == ND_FP64) {
    char* x64 = static_cast<char*>(field(c, "solve_x64", 0, n));
    void* r64 = field(c, "solve_r64", 0);
    if (!x64 || !r64) return fail(c, ND_ERR_OOM, "nd_solve: workspace");
    MsResult ms;
    s = mscg_run(c, 0, 0, false, b64, x64, sig, tols, {}, 1.0, maxit, &ms);
    if (s != ND_OK && s != ND_ERR_NOT_CONVERGED) return s;
    inf.iters = inf.sloppy_iters = ms.iters;
    const size_t f64 = (size_t)spinor_bytes(0, c->Vh);
    for (int l = 0; l < n; ++l) {
      double rel;
      ND_TRY(residual64(c, r64, b64, x64 + l * f64, sig[l], 1.0, bn2, &rel));
      inf.max_resid = std::max(inf.max_resid, rel);
      ND_TRY(nd_unpack_spinor(c, x[perm[l]], x64 + l * f64, ND_FP64, 1));
    }
  } else {
    MixedStats ms;
    auto sink = [&](int l, void* x64) -> nd_status { return nd_unpack_spinor(c, x[perm[l]], x64, ND_FP64, 1); };
    s = mixed_solve(c, (int)inner, b64, bn2, sig, tols, 1.0, maxit, &ms, sink);
    if (s != ND_OK) return s;
    inf.iters = ms.iters;
    inf.sloppy_iters = ms.sloppy_iters;
    inf.outer = ms.outer;
    inf.max_resid = ms.max_resid;
  }
  ND_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
  inf.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  return s;
}
