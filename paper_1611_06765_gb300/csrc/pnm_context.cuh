// pnm_context.cuh -- the opaque pnm_ctx behind the C ABI.
#pragma once
#include <map>
#include <vector>

#include "pnm_internal.cuh"

struct MixedState;  // mixed-precision operand arenas (mixed.cu)

struct pnm_ctx {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<SysInfo> sys;
  DevState d{};
  std::vector<void*> owned;  // device allocations released by pnm_destroy

  // sizes
  int nsp_total = 0, nch = 0, nx = 0, nrows = 0, n_hh_pairs = 0, n_pp_pairs = 0;
  long nt = 0, nvpp = 0, nvhh = 0, nxt = 0, nxc = 0;
  int max_x_dim = 0, max_npp = 0;

  // host copies of the channel metadata
  std::vector<int> h_ch_sys, h_key, h_nhh, h_npp, h_hh_off, h_pp_off, h_szero;
  std::vector<long> h_t_off, h_vpp_off, h_x_t_off;
  std::vector<int2> h_rows;
  std::vector<int> h_x_nph, h_x_nhp, h_x_ph_off, h_x_hp_off;

  // work lists
  PPItem* pp_items = nullptr;
  int n_pp_items = 0;
  int2* ab_items = nullptr;
  int n_ab_items = 0;

  // loop control
  int *row_lo_d = nullptr, *row_hi_d = nullptr, *lut_off_d = nullptr;  // per system
  LoopCtl* ctl = nullptr;     // device
  double* small = nullptr;    // device scratch for single-value queries
  SysCtl* sysctl = nullptr;   // device, one per system
  double* hist = nullptr;     // device, (hist_cap) per system
  int hist_cap = 0;
  int last_iters_host = 0;

  // graphs, one per precision mode
  std::map<int, cudaGraphExec_t> graphs;
  std::map<int, cudaGraph_t> graph_defs;
  unsigned long long cond_handle_for_mode[4] = {0, 0, 0, 0};

  MixedState* mixed = nullptr;

  // timings (ms)
  double t_setup = 0, t_mbpt2 = 0, t_solve = 0, t_mixed = 0, t_refine = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

void pnm_build(pnm_ctx* ctx, int nsys, const int* Ns, const double* rhos, const int* n2maxs,
               const pnm_minnesota& P);
void pnm_prepare_iteration(pnm_ctx* ctx);
void pnm_eref_all(pnm_ctx* ctx);
void pnm_mbpt2_all(pnm_ctx* ctx, double* out);
int pnm_solve(pnm_ctx* ctx, const pnm_solve_opts& o, double* dE, int* iters, double* resid);
void pnm_free_mixed(pnm_ctx* ctx);
void pnm_enqueue_body(pnm_ctx* ctx, int mode, int use_cond, cudaGraphConditionalHandle h);
void pnm_enqueue_body_mixed(pnm_ctx* ctx, int use_cond, cudaGraphConditionalHandle h);
void pnm_prepare_mixed(pnm_ctx* ctx);
void pnm_start(pnm_ctx* ctx, int init, const std::vector<double>& tol);
int pnm_run_loop(pnm_ctx* ctx, int mode, int max_iter, int host_loop, double alpha);
void pnm_reopen(pnm_ctx* ctx);
void pnm_settle_amplitudes(pnm_ctx* ctx);
