// pnm_context.cuh -- the opaque pnm_ctx behind the C ABI.
#pragma once
#include <map>
#include <vector>

#include "pnm_internal.cuh"

struct MixedState;  // mixed-precision operand arenas (mixed.cu)
struct MlpState;    // learned warm start (mlp.cu)

// Kernel ids of the per-kernel profiler.
enum {
  KID_TSTATS = 0, KID_DCHI, KID_PH64, KID_PP64, KID_UPDATE, KID_FINALIZE,
  KID_PP_TC, KID_PH32, KID_TSTATS32, KID_UPDATE_MIX, KID_PACK, KID_DCHI32, KID_PH_F2, KID_PP_F2, PNM_NKERNELS
};
extern const char* const pnm_kernel_names[PNM_NKERNELS];

struct pnm_ctx {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<SysInfo> sys;
  DevState d{};
  std::vector<void*> owned;  // device allocations released by pnm_destroy

  // sizes
  int nsp_total = 0, nch = 0, nx = 0, nrows = 0, n_hh_pairs = 0, n_pp_pairs = 0;
  long nt = 0, nvpp = 0, nvhh = 0, nxt = 0, nxc = 0;
  long ns = 0;  // elements of the ladder layout (n_hh x n_lad over the channels with V_pppp)
  int max_x_dim = 0, max_npp = 0, max_nlad = 0;
  int2* lad_rows = nullptr;  // (channel, ij) rows of the channels with V_pppp (ladder gather)
  int n_lad_rows = 0;

  // host copies of the channel metadata
  std::vector<int> h_ch_sys, h_key, h_nhh, h_npp, h_hh_off, h_pp_off, h_vpp;
  std::vector<long> h_t_off, h_x_t_off;
  std::vector<int> h_nlad;               // ladder basis size per channel (0: no V_pppp block)
  std::vector<long> h_s_off, h_vl_off;   // ladder-layout and ladder-V offsets per channel
  std::vector<int2> h_rows;
  std::vector<int> h_x_nph, h_x_nhp, h_x_ph_off, h_x_hp_off;
  std::vector<int> h_x_cls;  // spin-flip class of each cross channel (+1, 0, -1)
  std::vector<int> h_row_mode;  // per row (h_rows): 2/1 computed by the updates, 0 a flip

  // work lists
  int2* pp_items = nullptr;   // (channel, first pp column) of the FP64 pp ladder
  int n_pp_items = 0;
  int4* upd_items = nullptr;  // (channel, ij, first pp column) of the update
  int n_upd_items = 0;
  int *upd_lo_d = nullptr, *upd_hi_d = nullptr;  // per system ranges of the (row, column) items
  int4* grp_items = nullptr;  // (channel, first ij, first pp column, rows) of the update
  int n_grp_items = 0, upd_rows = 1;
  int* ph_list = nullptr;  // cross channels of the ph launches (S_z >= 0, costliest first)
  // channels of the larger size class (k_ph_big), of the middle and the small class of the CTA
  // path and of the warp path of k_ph, in that order in ph_list
  int n_ph_big = 0, n_ph_mid = 0, n_ph = 0, n_ph_warp = 0;
  size_t ph_smem64 = 0, ph_smem32 = 0;          // shared memory of a small-class k_ph CTA
  size_t ph_mid_smem64 = 0, ph_mid_smem32 = 0;  // of a middle-class k_ph CTA
  size_t ph_big_smem64 = 0, ph_big_smem32 = 0;  // and of a k_ph_big CTA
  f2* t_pair = nullptr;                          // FP32-pair copy of the current amplitudes
  int *grp_lo_d = nullptr, *grp_hi_d = nullptr;  // per system ranges of the update items
  int *ab_lo_d = nullptr, *ab_hi_d = nullptr;    // per system ranges of the column items
  int max_nhh = 1;
  int2* ab_items = nullptr;
  int n_ab_items = 0;

  // loop control
  int *row_lo_d = nullptr, *row_hi_d = nullptr, *lut_off_d = nullptr;  // per system
  LoopCtl* ctl = nullptr;     // device
  double* small = nullptr;    // device scratch for single-value queries
  double* mbpt3_buf = nullptr;
  double* expand_buf = nullptr;  // the pp ladder in the amplitude layout (operator call)  // per-row partials and per-system results of pnm_mbpt3
  SysCtl* sysctl = nullptr;   // device, one per system
  double* hist = nullptr;     // device, (hist_cap) per system
  int hist_cap = 0;
  int last_iters_host = 0;

  // graphs, one per precision mode
  std::map<int, cudaGraphExec_t> graphs;
  std::map<int, cudaGraph_t> graph_defs;
  // whole-solve graphs (start, iteration loop, refinement loop, settling, read-back), one per
  // solve configuration; their run-time parameters and results pass through pinned host memory
  std::map<int, cudaGraphExec_t> solve_graphs;
  std::map<int, cudaGraph_t> solve_graph_defs;
  void* h_pinned = nullptr;      // one block: h_par, h_ctl, h_sc[nsys], h_mlp_err
  SolveParams* h_par = nullptr;
  LoopCtl* h_ctl = nullptr;
  SysCtl* h_sc = nullptr;
  int* h_mlp_err = nullptr;
  SolveParams* d_par = nullptr;
  double* d_tol = nullptr;       // per-system tolerance of the energy test
  std::vector<double> tol_host;  // the values d_tol holds
  unsigned long long cond_handle_for_mode[4] = {0, 0, 0, 0};

  MixedState* mixed = nullptr;
  MlpState* mlp = nullptr;
  // FP32-pair copies of the ladder-basis V_pppp, V_pphh, W and <kb|v|cj> (made on first use by
  // the FP32-pair contractions)
  f2 *vpp_f2 = nullptr, *vpphh_f2 = nullptr, *xw_f2 = nullptr, *xv1_f2 = nullptr;
  // work list of the ladder-basis V (items (channel, first row), per system a run) and the
  // shared memory of its kernel; the V itself is built on first use (pnm_need_vpp64 / _f2)
  int2* vl_items = nullptr;
  std::vector<int> vl_sys;
  size_t vl_smem = 0;
  double hbar2_2m = 0.0;
  int mlp_fallback = 0;  // 1 when the last learned start was replaced by the MBPT2 start

  // side streams for the independent parts of an update (ph term, pp ladder), joined by events
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
  bool serial_sched[3] = {false, false, false};  // per mode (0 FP64, 1 mixed, 2 FP32-pair refinement): one stream only
  bool sched_tuned[3] = {false, false, false};
  int cur_mode = 0;

  // per-kernel CUDA-event profiling of host-driven solves (never active during capture)
  bool prof_on = false, prof_live = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev;
  std::vector<int> prof_pending;  // kernel id per used event pair
  double prof_ms[PNM_NKERNELS] = {};
  int prof_n[PNM_NKERNELS] = {};

  // timings (ms)
  double t_setup = 0, t_mbpt2 = 0, t_solve = 0, t_mixed = 0, t_refine = 0, t_mbpt3 = 0;
  // host wall time (ms) of the last solve's one-time preparation: pair and FP32 copies, schedule
  // tuning, and the capture and instantiation of its graphs (t_graph_host accumulates the latter)
  double t_prepare = 0, t_graph_host = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

// Autotuner cache key: device and the (N, n2max) of every system, which fix all channel
// sizes (the density only rescales values).
inline std::string pnm_shape_key(const pnm_ctx* ctx) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::string k = "dev" + std::to_string(dev);
  for (const SysInfo& S : ctx->sys) k += ";" + std::to_string(S.N) + "," + std::to_string(S.n2max);
  return k;
}

// Device memory of contexts: stream-ordered allocations from one memory pool per device, owned
// by the library, whose freed blocks stay cached for the next context (a create/solve/destroy
// loop then maps no new memory).  pnm_pool_alloc throws PNM_ENOMEM.
void* pnm_pool_alloc(cudaStream_t s, size_t bytes);
void pnm_pool_free(cudaStream_t s, void* p);
// Raise a kernel's dynamic shared-memory limit (a property of the function, shared by every
// context of the process) to at least `bytes`; never lowers it, so a context built later with
// smaller channels cannot break the launches of an earlier one.
void pnm_smem_at_least(const void* func, size_t bytes);
template <typename F>
void smem_at_least(F* func, size_t bytes) {
  pnm_smem_at_least((const void*)func, bytes);
}
// An allocation on the context stream recorded in ctx->owned (released by pnm_destroy).
void* pnm_ctx_alloc(pnm_ctx* ctx, size_t bytes);
template <typename T>
T* ctx_alloc(pnm_ctx* ctx, size_t n) {
  return (T*)pnm_ctx_alloc(ctx, (n ? n : 1) * sizeof(T));
}
void pnm_build(pnm_ctx* ctx, int nsys, const int* Ns, const int* Zs, const double* rhos,
               const int* n2maxs, const double* thetas, const pnm_minnesota& P);
void pnm_prepare_iteration(pnm_ctx* ctx);
void pnm_eref_all(pnm_ctx* ctx);
void pnm_mbpt2_all(pnm_ctx* ctx, double* out);
int pnm_solve(pnm_ctx* ctx, const pnm_solve_opts& o, double* dE, int* iters, double* resid);
void pnm_free_mixed(pnm_ctx* ctx);
void pnm_enqueue_body(pnm_ctx* ctx, int mode, int use_cond, cudaGraphConditionalHandle h);
void pnm_prepare_terms(pnm_ctx* ctx, int terms);
void pnm_mbpt3_all(pnm_ctx* ctx, double* out);
// The pp ladder from its ladder layout (planes summed) into host memory in the amplitude layout.
void pnm_lad_expand(pnm_ctx* ctx, const float* rs, int planes, long pstride, double* host_out);
void pnm_lad_expand(pnm_ctx* ctx, const double* rs, int planes, long pstride, double* host_out);
void pnm_lad_expand(pnm_ctx* ctx, const f2* rs, int planes, long pstride, double* host_out);
// alpha / eps_ij^ab of the current mixed solve (the step of the mixed and refinement updates)
const double* pnm_mixed_aw(const pnm_ctx* ctx);
void pnm_enqueue_body_mixed(pnm_ctx* ctx, int use_cond, cudaGraphConditionalHandle h);
void pnm_prepare_mixed(pnm_ctx* ctx);
void pnm_start(pnm_ctx* ctx, int init, const std::vector<double>& tol);
int pnm_run_loop(pnm_ctx* ctx, int mode, int max_iter, int min_iter, int host_loop, double alpha,
                 int* iter_out = nullptr);
void pnm_reopen(pnm_ctx* ctx);
void pnm_settle_amplitudes(pnm_ctx* ctx);
void pnm_mlp_start(pnm_ctx* ctx);
void pnm_mlp_prepare(pnm_ctx* ctx);
void pnm_ladder_v(pnm_ctx* ctx, double* out64, f2* out2);
void pnm_need_vpp64(pnm_ctx* ctx);
void pnm_need_vpp_f2(pnm_ctx* ctx);
void pnm_mlp_enqueue(pnm_ctx* ctx);
void pnm_drop_solve_graphs(pnm_ctx* ctx);
void pnm_set_node_priorities(cudaGraph_t body);
void pnm_solve_begin(pnm_ctx* ctx);
void pnm_start_device(pnm_ctx* ctx, int init);
void pnm_loop_begin(pnm_ctx* ctx, int mode);
void pnm_refine_gate(pnm_ctx* ctx, cudaGraphConditionalHandle h);
void pnm_loop_end_settle(pnm_ctx* ctx);
void pnm_flip_copy_device(pnm_ctx* ctx);
void pnm_mixed_pack_t(pnm_ctx* ctx);
void pnm_mixed_set_alpha(pnm_ctx* ctx, double alpha);
void pnm_free_mlp(pnm_ctx* ctx);
int* pnm_mlp_err(pnm_ctx* ctx);
void prof_begin(pnm_ctx* ctx, int kid);
void prof_end(pnm_ctx* ctx);
void prof_collect(pnm_ctx* ctx);
FinArgs fin_args(pnm_ctx* ctx, int use_cond, cudaGraphConditionalHandle h, bool per_row);
void pnm_enqueue_stats(pnm_ctx* ctx, bool mixed, bool pair = false);
void pnm_launch_pp64(pnm_ctx* ctx, cudaStream_t s, bool rep_only = true, const f2* vpp_f2 = nullptr);
void launch_ph_f2(pnm_ctx* ctx, const f2* tpair, const f2* xw, const f2* xv1, cudaStream_t s);
void pnm_split_f2(const double* a, f2* b, long n, cudaStream_t s);
void pnm_prepare_f2(pnm_ctx* ctx);
void pnm_split_cur(pnm_ctx* ctx, cudaStream_t s);
size_t ph_smem_bytes(int max_dim, int nm, size_t elem);
void pnm_mixed_pack_initial(pnm_ctx* ctx, double alpha);
void pnm_fork(pnm_ctx* ctx);
void pnm_join(pnm_ctx* ctx);
void pnm_launch_mbpt2_into(const pnm_ctx* ctx, double* partials, double* results);
void pnm_apply_ph(pnm_ctx* ctx, int sys, int precision, const double* t, double* r, size_t n);
void pnm_apply_pp(pnm_ctx* ctx, int sys, int precision, const double* t, double* r, size_t n);
void launch_ph64(pnm_ctx* ctx, cudaStream_t s, bool linear = false);
void pnm_flip_symmetrise(pnm_ctx* ctx, double* t, cudaStream_t s);
void pnm_flip_copy(pnm_ctx* ctx, double* t, cudaStream_t s);
void pnm_flip_copy_current(pnm_ctx* ctx, int iter);
void launch_ph_mix(pnm_ctx* ctx, const float* xt, const float* xw, const float* xv1, float* xq, cudaStream_t s);
void launch_update64(pnm_ctx* ctx, int use_cond, cudaGraphConditionalHandle h, bool pair = false);
void launch_update_mix(pnm_ctx* ctx, const float* rpp, const float* xq, const double* aw, float* xt, int use_cond,
                       cudaGraphConditionalHandle h, int nplanes, long pstride);
void pnm_alpha_inv(pnm_ctx* ctx, double alpha, double* aw);
void pnm_mixed_tuning(const pnm_ctx* ctx, int* ksplit, int* stages, float* us, int* serial_mask);
bool pnm_concurrent(const pnm_ctx* ctx);
void pnm_tune_schedule(pnm_ctx* ctx, int mode, double alpha);
void pnm_selftest_wait(pnm_ctx* ctx);
