// solve.cu -- the CCD driver (Sec. "Developing a CCD code": MBPT2 start, Jacobi updates of
// Eq. ccd3, mixing, stop on |dE^(n+1) - dE^(n)| < eta) and single-element V access.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "pnm_context.cuh"

__global__ void k_v_one(const char4* __restrict__ nvec, const double* __restrict__ lut, int p,
                        int q, int r, int s, double* out) {
  *out = v_minnesota_as(nvec[p], nvec[q], nvec[r], nvec[s], lut);
}

static float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

// ------------------------------------------------------------------ whole-solve graphs
// A solve that is not host-driven runs as one graph: the start (learned-start inference, control
// blocks, initial energy, FP32 copies), the first iteration loop (a WHILE node over one update),
// the spin flips of the FP64 amplitudes, the refinement gate and loop, settling and the copy of
// the control blocks to pinned host memory.  One launch and one synchronisation per solve: no
// host round trip between the phases leaves the device idle.
void pnm_drop_solve_graphs(pnm_ctx* ctx) {
  for (auto& g : ctx->solve_graphs) cudaGraphExecDestroy(g.second);
  for (auto& g : ctx->solve_graph_defs) cudaGraphDestroy(g.second);
  ctx->solve_graphs.clear();
  ctx->solve_graph_defs.clear();
}

static size_t round64(size_t b) { return (b + 63) & ~(size_t)63; }

// Pinned parameter and result block, device parameters and tolerances (once per context).
static void solve_buffers(pnm_ctx* ctx) {
  if (ctx->h_pinned) return;
  const size_t nsys = ctx->sys.size();
  const size_t o_ctl = round64(sizeof(SolveParams)), o_sc = o_ctl + round64(sizeof(LoopCtl));
  const size_t o_err = o_sc + round64(nsys * sizeof(SysCtl)), total = o_err + 64;
  void* p = nullptr;
  if (cudaHostAlloc(&p, total, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    throw PnmError{PNM_ENOMEM, "pinned host allocation failed"};
  }
  ctx->h_pinned = p;
  char* b = (char*)p;
  ctx->h_par = (SolveParams*)b;
  ctx->h_ctl = (LoopCtl*)(b + o_ctl);
  ctx->h_sc = (SysCtl*)(b + o_sc);
  ctx->h_mlp_err = (int*)(b + o_err);
  ctx->d_par = ctx_alloc<SolveParams>(ctx, 1);
  ctx->d_tol = ctx_alloc<double>(ctx, nsys);
}

// Graph under construction: stream segments captured after the current frontier `deps`, and
// WHILE nodes whose body is one update.
struct SolveGraphBuilder {
  pnm_ctx* ctx;
  cudaGraph_t g = nullptr;
  std::vector<cudaGraphNode_t> deps;
  template <typename F>
  void segment(F&& f) {
    cudaStream_t s = ctx->stream;
    CUDA_TRY(cudaStreamBeginCaptureToGraph(s, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                           cudaStreamCaptureModeThreadLocal));
    try {
      f();
    } catch (...) {
      cudaGraph_t dummy;
      cudaStreamEndCapture(s, &dummy);
      throw;
    }
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t* dp = nullptr;
    size_t nd = 0;
    CUDA_TRY(cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &dp, nullptr, &nd));
    std::vector<cudaGraphNode_t> next(dp, dp + nd);
    cudaGraph_t out;
    CUDA_TRY(cudaStreamEndCapture(s, &out));
    deps = next;
  }
  void loop(int mode, cudaGraphConditionalHandle h) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CUDA_TRY(cudaGraphAddNode(&node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CUDA_TRY(cudaStreamBeginCaptureToGraph(ctx->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
      pnm_enqueue_body(ctx, mode, 1, h);
    } catch (...) {
      cudaGraph_t dummy;
      cudaStreamEndCapture(ctx->stream, &dummy);
      throw;
    }
    cudaGraph_t captured;
    CUDA_TRY(cudaStreamEndCapture(ctx->stream, &captured));
    pnm_set_node_priorities(body);
    deps.assign(1, node);
  }
};

static cudaGraphExec_t solve_graph(pnm_ctx* ctx, bool mixed, bool refine, bool pair, int init, int terms) {
  const int key = (mixed ? 1 : 0) | (refine ? 2 : 0) | (pair ? 4 : 0) | (init << 4) | (terms << 8);
  auto f = ctx->solve_graphs.find(key);
  if (f != ctx->solve_graphs.end()) return f->second;
  const auto w0 = std::chrono::steady_clock::now();
  cudaStream_t s = ctx->stream;
  const int nsys = (int)ctx->sys.size();
  SolveGraphBuilder b{ctx};
  CUDA_TRY(cudaGraphCreate(&b.g, 0));
  try {
    cudaGraphConditionalHandle h1, h2 = 0;
    CUDA_TRY(cudaGraphConditionalHandleCreate(&h1, b.g, 1, cudaGraphCondAssignDefault));
    if (refine) CUDA_TRY(cudaGraphConditionalHandleCreate(&h2, b.g, 0, cudaGraphCondAssignDefault));
    const int mode1 = mixed ? PNM_PREC_BF16X3 : (PNM_PREC_FP64 | (terms << 4));
    b.segment([&] {
      CUDA_TRY(cudaMemcpyAsync(ctx->d_par, ctx->h_par, sizeof(SolveParams), cudaMemcpyHostToDevice, s));
      CUDA_TRY(cudaEventRecordWithFlags(ctx->ev[0], s, cudaEventRecordExternal));
      pnm_solve_begin(ctx);
      if (init == PNM_INIT_MLP) pnm_mlp_enqueue(ctx);  // t0 = learned start, kept like a given start
      pnm_start_device(ctx, init == PNM_INIT_MLP ? PNM_INIT_KEEP : init);
      if (mixed) pnm_mixed_pack_t(ctx);
      pnm_prepare_terms(ctx, terms);
      pnm_loop_begin(ctx, mode1);
    });
    b.loop(mode1, h1);
    b.segment([&] {
      if (mixed) pnm_flip_copy_device(ctx);
      CUDA_TRY(cudaEventRecordWithFlags(ctx->ev[1], s, cudaEventRecordExternal));
      if (refine) pnm_refine_gate(ctx, h2);
    });
    if (refine) b.loop(PNM_PREC_FP64 | (pair ? 1 << 8 : 0), h2);
    b.segment([&] {
      CUDA_TRY(cudaEventRecordWithFlags(ctx->ev[2], s, cudaEventRecordExternal));
      // the control blocks as the loops left them, then t0 = the latest amplitudes
      CUDA_TRY(cudaMemcpyAsync(ctx->h_ctl, ctx->ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaMemcpyAsync(ctx->h_sc, ctx->sysctl, sizeof(SysCtl) * nsys, cudaMemcpyDeviceToHost, s));
      if (init == PNM_INIT_MLP)
        CUDA_TRY(cudaMemcpyAsync(ctx->h_mlp_err, pnm_mlp_err(ctx), sizeof(int), cudaMemcpyDeviceToHost, s));
      pnm_loop_end_settle(ctx);
    });
    cudaGraphExec_t ge;
    CUDA_TRY(cudaGraphInstantiate(&ge, b.g, cudaGraphInstantiateFlagUseNodePriority));
    ctx->solve_graphs[key] = ge;
    ctx->solve_graph_defs[key] = b.g;
  } catch (...) {
    cudaGraphDestroy(b.g);
    throw;
  }
  ctx->t_graph_host += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
  return ctx->solve_graphs[key];
}

static int pnm_solve_finish(pnm_ctx* ctx, const pnm_solve_opts& o, int status, double* dE, int* iters,
                            double* resid);

int pnm_solve(pnm_ctx* ctx, const pnm_solve_opts& o, double* dE, int* iters, double* resid) {
  if (!(o.mix_alpha > 0.0 && o.mix_alpha <= 1.0)) throw PnmError{PNM_EINVAL, "mix_alpha must be in (0,1]"};
  if (o.max_iter < 1) throw PnmError{PNM_EINVAL, "max_iter must be >= 1"};
  if (o.precision != PNM_PREC_FP64 && o.precision != PNM_PREC_BF16X3)
    throw PnmError{PNM_EINVAL, "unknown precision mode"};
  if (o.init < PNM_INIT_MBPT2 || o.init > PNM_INIT_MLP) throw PnmError{PNM_EINVAL, "unknown init"};
  if (o.refine_sweeps < 0) throw PnmError{PNM_EINVAL, "refine_sweeps must be >= 0"};
  if (!(o.tol_dE > 0.0) && !(o.tol_dE_per_N > 0.0)) throw PnmError{PNM_EINVAL, "no tolerance given"};
  if (o.terms < PNM_TERMS_FULL || o.terms > PNM_TERMS_LINEAR) throw PnmError{PNM_EINVAL, "unknown terms"};
  if (o.terms != PNM_TERMS_FULL && o.precision != PNM_PREC_FP64)
    throw PnmError{PNM_EINVAL, "truncated iterations run in FP64 only"};
  if (o.refine_kernels != PNM_PREC_FP64 && o.refine_kernels != PNM_PREC_F32PAIR)
    throw PnmError{PNM_EINVAL, "refine_kernels must be PNM_PREC_FP64 or PNM_PREC_F32PAIR"};
  cudaStream_t s = ctx->stream;
  int nsys = (int)ctx->sys.size();
  // work skipping for converged systems is scoped to the solve loops
  CUDA_TRY(cudaMemsetAsync(&ctx->ctl->skip_done, 0, sizeof(int), s));
  std::vector<double> tol(nsys);
  for (int k = 0; k < nsys; k++)
    tol[k] = o.tol_dE_per_N > 0.0 ? o.tol_dE_per_N * ctx->sys[k].N : o.tol_dE;
  int cap = o.max_iter + o.refine_sweeps + 2;
  if (cap > ctx->hist_cap) {
    if (ctx->hist) {
      // the old buffer stays owned by the context until destroy
    }
    ctx->hist = ctx_alloc<double>(ctx, (size_t)cap * nsys);
    ctx->hist_cap = cap;
    // graphs capture hist pointer and capacity: rebuild them
    for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.second);
    for (auto& g : ctx->graph_defs) cudaGraphDestroy(g.second);
    ctx->graphs.clear();
    ctx->graph_defs.clear();
    pnm_drop_solve_graphs(ctx);
  }
  const auto w0 = std::chrono::steady_clock::now();
  const double g0 = ctx->t_graph_host;
  bool mixed = o.precision != PNM_PREC_FP64;
  if (mixed) {
    pnm_prepare_mixed(ctx);
    pnm_mixed_set_alpha(ctx, o.mix_alpha);  // alpha / eps, read by the tuned updates too
  }
  const bool pair_refine = mixed && o.refine_sweeps > 0 && o.refine_kernels == PNM_PREC_F32PAIR;
  if (pair_refine) pnm_prepare_f2(ctx);
  // the FP64 ladder V and schedule only where an FP64 pp ladder runs (the FP64 iteration, or
  // refinement sweeps on the FP64 pipe); FP32-pair refinement has its own schedule slot
  const bool fp64_ladder = !mixed || (o.refine_sweeps > 0 && !pair_refine);
  if (fp64_ladder) {
    pnm_need_vpp64(ctx);
    pnm_tune_schedule(ctx, PNM_PREC_FP64, o.mix_alpha);
  }
  if (pair_refine) pnm_tune_schedule(ctx, PNM_PREC_FP64 | (1 << 8), o.mix_alpha);
  if (mixed) pnm_tune_schedule(ctx, PNM_PREC_BF16X3, o.mix_alpha);
  if (!o.host_loop) {
    // one graph launch: the learned start's one-time state, the tolerances and alpha / eps
    // are prepared first (on the stream, ahead of the graph)
    solve_buffers(ctx);
    if (o.init == PNM_INIT_MLP) pnm_mlp_prepare(ctx);
    if (tol != ctx->tol_host) {
      CUDA_TRY(cudaMemcpyAsync(ctx->d_tol, tol.data(), sizeof(double) * nsys, cudaMemcpyHostToDevice, s));
      ctx->tol_host = tol;
    }
    if (mixed) pnm_mixed_set_alpha(ctx, o.mix_alpha);
    const bool refine = mixed && o.refine_sweeps > 0;
    cudaGraphExec_t ge = solve_graph(ctx, mixed, refine, pair_refine, o.init, o.terms);
    const double prep_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
    ctx->h_par->max_iter = o.max_iter;
    ctx->h_par->refine_sweeps = o.refine_sweeps;
    ctx->h_par->alpha = o.mix_alpha;
    CUDA_TRY(cudaGraphLaunch(ge, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    ctx->t_solve = elapsed(ctx->ev[0], ctx->ev[2]);
    ctx->t_mixed = mixed ? elapsed(ctx->ev[0], ctx->ev[1]) : 0.0;
    ctx->t_refine = mixed ? elapsed(ctx->ev[1], ctx->ev[2]) : 0.0;
    ctx->t_prepare = prep_ms;
    ctx->last_iters_host = ctx->h_ctl->iter;
    const int status = ctx->h_ctl->status;
    for (int k = 0; k < nsys; k++) {
      if (dE) dE[k] = ctx->h_sc[k].e_new;
      if (iters) iters[k] = ctx->h_sc[k].iters;
      if (resid) resid[k] = ctx->h_sc[k].resid;
    }
    if (o.init == PNM_INIT_MLP && *ctx->h_mlp_err) {
      CUDA_TRY(cudaMemsetAsync(pnm_mlp_err(ctx), 0, sizeof(int), s));
      pnm_set_error(PNM_ETIMEOUT, "a device-side wait of the learned start ran out of its budget");
      return PNM_ETIMEOUT;
    }
    return pnm_solve_finish(ctx, o, status, dE, iters, resid);
  }
  const double prep_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();

  cudaEvent_t e0 = ctx->ev[0], e1 = ctx->ev[1], e2 = ctx->ev[2];
  CUDA_TRY(cudaEventRecord(e0, s));
  int init = o.init;
  if (init == PNM_INIT_MLP) {
    pnm_mlp_start(ctx);  // t0 = learned start; its energy is taken below as for a kept start
    init = PNM_INIT_KEEP;
  }
  pnm_start(ctx, init, tol);
  if (mixed) pnm_mixed_pack_initial(ctx, o.mix_alpha);
  pnm_prepare_terms(ctx, o.terms);
  int it0 = 0;
  int status = pnm_run_loop(ctx, mixed ? PNM_PREC_BF16X3 : (PNM_PREC_FP64 | (o.terms << 4)), o.max_iter, 0,
                            o.host_loop, o.mix_alpha, &it0);
  if (mixed) pnm_flip_copy_current(ctx, it0);
  CUDA_TRY(cudaEventRecord(e1, s));
  if (mixed && status == 1 && o.refine_sweeps > 0) {
    // exactly refine_sweeps FP64 updates, then (if the FP64 test has not passed by then)
    // further FP64 updates until it does, within max_iter more
    pnm_reopen(ctx);
    status = pnm_run_loop(ctx, PNM_PREC_FP64 | (pair_refine ? 1 << 8 : 0), it0 + o.refine_sweeps + o.max_iter,
                          it0 + o.refine_sweeps, o.host_loop, o.mix_alpha);
  }
  CUDA_TRY(cudaEventRecord(e2, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  ctx->t_solve = elapsed(e0, e2);
  ctx->t_mixed = mixed ? elapsed(e0, e1) : 0.0;
  ctx->t_refine = mixed ? elapsed(e1, e2) : 0.0;
  ctx->t_prepare = prep_ms + (ctx->t_graph_host - g0);
  pnm_settle_amplitudes(ctx);
  std::vector<SysCtl> hs(nsys);
  CUDA_TRY(cudaMemcpyAsync(hs.data(), ctx->sysctl, sizeof(SysCtl) * nsys, cudaMemcpyDeviceToHost, s));
  int start_err = 0;
  int* d_err = o.init == PNM_INIT_MLP ? pnm_mlp_err(ctx) : nullptr;
  if (d_err) CUDA_TRY(cudaMemcpyAsync(&start_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (start_err) {
    // the learned start is incomplete (a bounded wait of the inference kernel ran out)
    CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), s));
    pnm_set_error(PNM_ETIMEOUT, "a device-side wait of the learned start ran out of its budget");
    return PNM_ETIMEOUT;
  }
  for (int k = 0; k < nsys; k++) {
    if (dE) dE[k] = hs[k].e_new;
    if (iters) iters[k] = hs[k].iters;
    if (resid) resid[k] = hs[k].resid;
  }
  return pnm_solve_finish(ctx, o, status, dE, iters, resid);
}

// The end of a solve: the MBPT2 fallback of a learned start that did not converge, and the
// status code.
static int pnm_solve_finish(pnm_ctx* ctx, const pnm_solve_opts& o, int status, double* dE, int* iters,
                            double* resid) {
  if (o.init == PNM_INIT_MLP) ctx->mlp_fallback = 0;
  if (o.init == PNM_INIT_MLP && (status == PNM_ENOTCONV || status == PNM_EDIVERGED)) {
    // the CCD iteration judges the learned start: if it does not lead to convergence,
    // solve again from the MBPT2 guess
    pnm_solve_opts o2 = o;
    o2.init = PNM_INIT_MBPT2;
    float t_first = (float)ctx->t_solve;
    double p_first = ctx->t_prepare;
    int rc = pnm_solve(ctx, o2, dE, iters, resid);
    ctx->t_solve += t_first;
    ctx->t_prepare += p_first;
    ctx->mlp_fallback = 1;
    return rc;
  }
  if (status == 1) return PNM_OK;
  if (status == PNM_ENOTCONV) pnm_set_error(status, "iteration cap reached before convergence");
  if (status == PNM_EDIVERGED)
    pnm_set_error(status, "NaN or Inf in the energy or residual, or an energy change growing geometrically");
  if (status == PNM_ETIMEOUT) pnm_set_error(status, "a device-side wait ran out of its budget");
  return status;
}

extern "C" int pnm_v_element(const pnm_ctx* ctx, int sys, int p, int q, int r, int s, double* out) {
  try {
    if (!ctx || !out || sys < 0 || sys >= (int)ctx->sys.size())
      throw PnmError{PNM_EINVAL, "bad argument"};
    const SysInfo& S = ctx->sys[sys];
    for (int x : {p, q, r, s})
      if (x < 0 || x >= S.nsp) throw PnmError{PNM_EINVAL, "state index out of range"};
    double* d = ctx->small;
    k_v_one<<<1, 1, 0, ctx->stream>>>(ctx->d.nvec + S.sp_off, ctx->d.lut + S.lut_off, p, q, r, s, d);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(out, d, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return PNM_OK;
  } catch (const PnmError& e) {
    pnm_set_error(e.code, e.msg);
    return e.code;
  }
}
