// pnm_internal.cuh -- device data layout of a pnmcc context and shared helpers.
//
// Layout in HBM (all systems of a context concatenated; every index below is global):
//   states       char4 nvec[n_sp_total] = (n_x, n_y, n_z, s); double eps[], ekin[]
//   direct chans per channel c: sys, key, n_hh, n_pp, hh_off, pp_off, t_off, vpp_off, vhh_off
//                int2 hh_pair[], pp_pair[] (global state indices, lexicographic per channel)
//   amplitudes   t[c] is an n_hh x n_pp row-major block (hh rows, pp contiguous): element
//                (ij, ab) at t_off[c] + ij * n_pp + ab.  v_pphh has the same layout.
//   V_pppp       only for channels where <ab|v|cd> can be nonzero (not both |S_z| = 2 and
//                |T_z| = 2: identical nucleons of equal spin do not interact; for neutrons
//                that leaves S_z = 0): n_pp x n_pp, symmetric, row-major at vpp_off[c].
//   cross chans  per channel x: n_ph rows (a,i), n_hp columns (k,c); T_x/Q_x are
//                n_ph x n_hp at xt_off[x]; V1_x (<kb|v|cj>) n_hp x n_hp at xc_off[x];
//                W_x (<kl|v|ce>, n_hp x n_ph) stored transposed (n_ph x n_hp) at xw_off[x].
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pnmcc.h"
#include "fp2.cuh"

#define PNM_PI 3.14159265358979323846

struct PnmError {
  int code;
  std::string msg;
};

void pnm_set_error(int code, const std::string& msg);

#define CUDA_TRY(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      throw PnmError{PNM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

// One system (N, rho, n2max) of a context.
struct SysInfo {
  int N, n2max, r, m, M, nkeys;  // N: particles (holes) of all species
  int Z = 0;                     // protons among them
  int species = 1;               // 1 neutrons, 2 protons, 3 both
  double rho, L;
  int nsp, sp_off;        // states [sp_off, sp_off + nsp)
  int ch_begin, ch_end;   // direct channels
  int x_begin, x_end;     // cross channels
  long t_begin, t_end;    // restricted amplitudes
  int row_begin, row_end; // (channel, ij) rows
  int lut_off, lut_len;
  double eref;
  double phi[3];          // twist theta / (2 pi) per axis; all zero = periodic
};

// Static data of one row (hole pair ij) of an update item: the pair's states, their spin labels
// and eps_i + eps_j, so that an update's row setup is one load and the one-body gathers.
struct __align__(16) UpdRow {
  int ij, hx, hy, pad;
  char4 si, sj;
  double eij;
};

// Device arena pointers; all arrays are global over the systems of the context.
struct DevState {
  // states
  char4* nvec;
  double *eps, *ekin, *lut;
  int* sp_sys;           // state -> system
  int* sp_hole;          // 1 for hole states
  // direct channels
  int *ch_sys, *ch_key, *ch_nhh, *ch_npp, *ch_hh_off, *ch_pp_off, *ch_vpp;
  long *ch_t_off, *ch_vpp_off, *ch_vhh_off;
  // ladder basis of the pp ladder (channels with a V_pppp block): n_lad vectors per channel,
  // ladder-layout blocks (n_hh x n_lad) at ch_s_off; lad_map per pp pair: its vector and sign
  // as +-(index + 1); lad_mem per vector (at the channel's pp offset): its one or two pairs as
  // +-(position + 1), 0 for no second pair
  int* ch_nlad;
  long* ch_s_off;
  int* lad_map;
  int2* lad_mem;
  int2 *hh_pair, *pp_pair;
  // rows (channel, ij) for the update and energy partials
  int2* row_item;        // (channel, ij)
  // cross channels
  int *x_nph, *x_nhp;
  int* x_sys;            // cross channel -> system
  long *x_t_off, *x_c_off, *x_w_off;
  int2 *ph_pair, *hp_pair;
  int* x_ph_off;
  int* x_hp_off;
  // global spin flip F: class of each cross channel (+1: S_z > 0, formed in full; 0: S_z = 0,
  // formed on its spin-up rows; -1: S_z < 0, not formed), the flipped column of every hp
  // column, and for S_z = 0 channels the spin-up rows and columns (first half of the slots)
  int *x_cls, *x_fcol, *x_rrow, *x_rcol;
  int* fmap;             // per t element: sign * (index + 1) of its spin-flipped element
  // mixed and FP64 updates: the hole-pair rows they compute (flip representatives), per item
  // a run of this list (items hold (channel, first entry, first column, rows))
  int* upd_row;
  int* ch_uoff;          // per direct channel its run of upd_row (nch + 1 offsets)
  UpdRow* upd_rowinfo;   // per update item UPD_ROWS rows (rows past the item's last repeat it)
  // maps
  int* xmap;             // per T element: sign * (t index + 1), 0 = structurally zero
  int4* qmap;            // per t element: the four Q positions of P(ij)P(ab) Q (formed positions)
  int *occ_off, *occ_idx; // per state: pair indices (pp for particles, hh for holes)
  // blocks
  double *v_pphh, *v_pppp, *v_hhhh, *x_v1, *x_w;  // v_pppp: n_lad x n_lad per channel, ladder basis
  double *den, *inv_den;  // eps_i + eps_j - eps_a - eps_b per amplitude, and its reciprocal
  // iteration state
  double *t0, *t1;       // double buffer, parity = iteration & 1
  float *t32_0, *t32_1;  // FP32 copies of t0/t1 kept by the mixed-precision update (else null)
  // FP32 intermediates of the mixed-precision iteration (null until it is first prepared):
  // v_pphh and v_hhhh copies, chi_hh, the one-body row/column sums and the one-body terms
  float *v32, *vhh32, *chi32, *sij32, *sab32, *dchi32;
  double *rpp, *chi_hh, *dchi, *sab, *sij, *xq;  // rpp: pp ladder in the ladder layout
  double* s64;           // amplitudes in the ladder basis (input of the FP64 pp ladder)
  double *eparts, *rparts;
  // per-system loop state (converged systems are frozen: later steps skip their work)
  const struct SysCtl* sysctl;
};

// Work-list items for the grouped pp-ladder launch (FP64 path).
struct PPItem {
  int ch;      // direct channel
  int ab0;     // first pp column of the tile
  int ij0;     // first hh row of the tile
  int nij;     // rows in the tile
};

// Solve-loop control block in device memory (one per context).
struct LoopCtl {
  int iter;          // updates made in the current solve
  int blocks_done;   // blocks of the current update that have finished (last-block finalize)
  int dev_error;     // set by a kernel whose bounded wait ran out (the loop then stops)
  int max_iter;
  int status;        // 0 running, 1 converged, PNM_ENOTCONV, PNM_EDIVERGED
  int mode;          // 0 FP64 iteration, 1 mixed iteration
  int min_iter;      // no system counts as converged before this many updates
  int skip_done;     // 1 inside the solve loop: kernels skip the work of converged systems
  double alpha;
};

// Run-time parameters of a whole-solve graph, copied from pinned host memory by its first node.
struct SolveParams {
  int max_iter;       // iteration cap of the first loop; the refinement adds refine_sweeps + it
  int refine_sweeps;  // refinement updates before the FP64 test may stop the loop
  double alpha;       // mixing
};

struct SysCtl {
  double e_old, e_new, resid;
  double tol;
  int done;       // 1 once converged
  int iters;
  int frozen_at;  // index of the update after which it converged (valid while done)
  int grow;       // consecutive updates whose |dE| at least doubled (above tol): divergence
  double d_old;   // |dE| of the previous update
};

// Divergence: |dE| at least doubling, above the tolerance, over this many consecutive updates
// (a 64-fold geometric growth; NaN or Inf diverges at once).
constexpr int PNM_DIVERGE_STEPS = 6;

// True inside the solve loop once system `sys` has met its stopping rule (its amplitudes are
// frozen): the contraction kernels of later steps skip its work, and the update skips it too
// from the second step on (the first one copies the amplitudes into the other buffer, after
// which both buffers hold them).
__device__ __forceinline__ bool sys_done(const DevState& D, const LoopCtl* ctl, int sys) {
  return ctl->skip_done != 0 && D.sysctl != nullptr && D.sysctl[sys].done != 0;
}
__device__ __forceinline__ bool sys_settled(const SysCtl& S, const LoopCtl* ctl) {
  return ctl->skip_done != 0 && S.done != 0 && ctl->iter >= S.frozen_at + 2;
}

// Arguments of the end-of-update step (energy, convergence test, loop condition).
struct FinArgs {
  const double* eparts;
  const double* rparts;
  const int* lo;        // per system: first partial
  const int* hi;        // per system: one past the last partial
  int nsys;
  SysCtl* sc;
  double* hist;
  int hist_cap;
  int use_cond;
  cudaGraphConditionalHandle handle;
};

// The update kernels: at most UPD_ROWS hole pairs per CTA (the FP64 update shares one pass
// over a t column for the hh ladder among them), loads issued in batches of UPD_BATCH rows,
// at least UPD_MIN_BLOCKS CTAs of the mixed update per SM; channels may hold at most
// UPD_MAX_NHH hole pairs.  The PNM_UPD_* macros override the tuning constants at build time.
#ifndef PNM_UPD_ROWS
#define PNM_UPD_ROWS 8
#endif
#ifndef PNM_UPD_BATCH
#define PNM_UPD_BATCH 2
#endif
#ifndef PNM_UPD_MIN_BLOCKS
#define PNM_UPD_MIN_BLOCKS 6
#endif
constexpr int UPD_ROWS = PNM_UPD_ROWS, UPD_MAX_NHH = 128, UPD_BATCH = PNM_UPD_BATCH;
constexpr int UPD_MIN_BLOCKS = PNM_UPD_MIN_BLOCKS;

// Threads of a ph-term CTA (one cross channel each); channels of at most PH_WARP_DIM rows and
// columns (of their halves for S_z = 0) take one warp each.
// Channels with more than PH_SMALL_DIM rows or columns go to the larger size class, those with
// more than PH_MID_DIM to the middle one (each class with its own launch and shared-memory
// size, so that the many smaller channels keep more CTAs per SM).
constexpr int PH_THREADS = 128, PH_WARP_DIM = 16, PH_SMALL_DIM = 32, PH_MID_DIM = 24;

// pp ladder of amplitude (ij, ab) of channel c from its ladder-layout value (planes summed by
// the caller where there are several).
__device__ __forceinline__ long lad_index(const DevState& D, int c, int ij, int ab, int& sign) {
  int m = D.lad_map[D.ch_pp_off[c] + ab];
  sign = m > 0 ? 1 : -1;
  return D.ch_s_off[c] + (long)ij * D.ch_nlad[c] + ((m > 0 ? m : -m) - 1);
}

// --------------------------------------------------------------------- device helpers

__device__ __forceinline__ int dot3(int x, int y, int z) { return x * x + y * y + z * z; }

// Double-buffered amplitudes: an update reads t[iter & 1] and writes the other buffer.
__device__ __forceinline__ const double* cur_t(const DevState& D, const LoopCtl* ctl) {
  return (ctl->iter & 1) ? D.t1 : D.t0;
}
__device__ __forceinline__ double* next_t(const DevState& D, const LoopCtl* ctl) {
  return (ctl->iter & 1) ? D.t0 : D.t1;
}
__device__ __forceinline__ const float* cur_t32(const DevState& D, const LoopCtl* ctl) {
  return (ctl->iter & 1) ? D.t32_1 : D.t32_0;
}
__device__ __forceinline__ float* next_t32(const DevState& D, const LoopCtl* ctl) {
  return (ctl->iter & 1) ? D.t32_0 : D.t32_1;
}

// Antisymmetrized Minnesota element with protons present.  The charge label w = s + 4t
// (t = +1 neutron, -1 proton) carries spin and isospin.  From V = 1/2 (V_R + 1/2(1+P_s) V_T +
// 1/2(1-P_s) V_S)(1 - P_s P_t), with the product-basis structures of the ket (r, s)
//   one = d(s_p,s_r) d(s_q,s_s) d(t_p,t_r) d(t_q,t_s), ps: spins of r and s exchanged,
//   pt: isospins exchanged, pst: both,
// the direct operator weights are 4 O_R = 2(one - pst), 4 O_T = one + ps - pt - pst and
// 4 O_S = one - ps + pt - pst; the exchange term (r <-> s) carries the opposite weights, so the
// antisymmetrized element is 1/4 sum_a (4 O_a) [Vt_a(n_p - n_r) + Vt_a(n_p - n_s)].
// hlut3[3m + a] = Vt_a / 2 at |dn|^2 = m.
__device__ __forceinline__ double v_minnesota_nucleons(char4 p, char4 q, char4 r, char4 s,
                                                       const double* __restrict__ hlut3) {
  auto tz = [](int w) { return w > 0 ? 1 : -1; };
  int tp = tz(p.w), tq = tz(q.w), tr = tz(r.w), ts = tz(s.w);
  int sp = p.w - 4 * tp, sq = q.w - 4 * tq, sr = r.w - 4 * tr, ss = s.w - 4 * ts;
  int one = (sp == sr && sq == ss && tp == tr && tq == ts);
  int ps = (sp == ss && sq == sr && tp == tr && tq == ts);
  int pt = (sp == sr && sq == ss && tp == ts && tq == tr);
  int pst = (sp == ss && sq == sr && tp == ts && tq == tr);
  int cR = 2 * (one - pst), cT = one + ps - pt - pst, cS = one - ps + pt - pst;
  if (cR == 0 && cT == 0 && cS == 0) return 0.0;
  int m1 = 3 * dot3(p.x - r.x, p.y - r.y, p.z - r.z);
  int m2 = 3 * dot3(p.x - s.x, p.y - s.y, p.z - s.z);
  double v = (double)cR * (hlut3[m1] + hlut3[m2]) + (double)cT * (hlut3[m1 + 1] + hlut3[m2 + 1]) +
             (double)cS * (hlut3[m1 + 2] + hlut3[m2 + 2]);
  return 0.5 * v;
}

// Antisymmetrized Minnesota element.  For two neutrons (charge labels w = s = +-1) P_tau = 1
// and the exchange form reduces to 1/2 (V_R + V_S)(1 - P_sigma) (the V_T term cancels), whose
// antisymmetrized plane-wave element is 1/2 [Vt(n_p - n_r) + Vt(n_p - n_s)] times the spin
// factor d(s_p,s_r) d(s_q,s_s) - d(s_p,s_s) d(s_q,s_r), with momentum conservation.
// hlut[m] = Vt / 2 at |dn|^2 = m for this system, so the element is one FP64 addition and a
// sign (bit for bit 0.5 (Vt_1 + Vt_2) sf: halving is exact); the FP64 unit of a GB300 runs
// at about 1/64 of its FP32 rate, and the V blocks are generated element by element.
// Systems with protons (labels |w| >= 3) use v_minnesota_nucleons and its interleaved LUT.
__device__ __forceinline__ double v_minnesota_as(char4 p, char4 q, char4 r, char4 s,
                                                 const double* __restrict__ hlut) {
  if (p.x + q.x != r.x + s.x || p.y + q.y != r.y + s.y || p.z + q.z != r.z + s.z) return 0.0;
  if (p.w > 1 || p.w < -1) return v_minnesota_nucleons(p, q, r, s, hlut);
  int sf = (p.w == r.w && q.w == s.w) - (p.w == s.w && q.w == r.w);
  if (sf == 0) return 0.0;
  int m1 = dot3(p.x - r.x, p.y - r.y, p.z - r.z);
  int m2 = dot3(p.x - s.x, p.y - s.y, p.z - s.z);
  double v = hlut[m1] + hlut[m2];
  return sf > 0 ? v : __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ull);
}

// Element offset inside a (rows x 64) BF16 plane stored as 8-row x 16-byte core matrices
// (K-major canonical layout of the tensor-core operands, no swizzle).
__device__ __forceinline__ int tile_core_off(int r, int k) {
  return (((r >> 3) * 8 + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

// x = hi + lo with hi, lo in BF16: x is rounded to FP32 once (the only FP64 instruction),
// hi = round(x), lo = round(x - hi) with the difference exact in FP32.
__device__ __forceinline__ void split_bf16(double x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  float xf = (float)x;
  hi = __float2bfloat16_rn(xf);
  lo = __float2bfloat16_rn(xf - __bfloat162float(hi));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum for blockDim.x a multiple of 32 (<= 1024); result valid in thread 0.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh32) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh32[w] = v;
  __syncthreads();
  int nw = blockDim.x >> 5;
  v = (threadIdx.x < nw) ? sh32[threadIdx.x] : (T)0;
  if (w == 0) v = warp_sum(v);
  __syncthreads();
  return v;
}

// Two block-wide sums at once (sh32: 32 doubles); results valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b, double* sh32) {
  a = warp_sum(a);
  b = warp_sum(b);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sh32[w] = a;
    sh32[16 + w] = b;
  }
  __syncthreads();
  int nw = blockDim.x >> 5;
  a = (threadIdx.x < nw) ? sh32[threadIdx.x] : 0.0;
  b = (threadIdx.x < nw) ? sh32[16 + threadIdx.x] : 0.0;
  if (w == 0) {
    a = warp_sum(a);
    b = warp_sum(b);
  }
  __syncthreads();
}
