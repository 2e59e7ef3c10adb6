// mixed.cu -- mixed-precision CCD update.
//
// The particle-particle ladder 1/2 sum_cd <ab|v|cd> t_cd^ij (Eq. ccd3 with the
// intermediate <ab|chi|cd> = <ab|v|cd> of Sec. "Developing a CCD code") is the dense
// per-channel contraction of the method.  Here it runs on the 5th-generation tensor cores:
//
//   D(ab, ij) = sum_cd V(ab, cd) t(ij, cd)          (M = ab tile of 128, N = n_hh padded
//                                                    to 16/32/48, K = cd)
//   with V = V_hi + V_lo and t = t_hi + t_lo split into BF16 pairs, and
//   D = V_hi t_hi + V_hi t_lo + V_lo t_hi accumulated in FP32 in tensor memory (TMEM).
//
// V is written once per context into HBM already in the UMMA canonical K-major layout
// (8-row x 16-byte core matrices, no swizzle), one 32 KB chunk (hi, lo) per 128 x 64 tile,
// so each tile moves with one bulk asynchronous copy (the TMA engine) into a 3-stage
// shared-memory ring guarded by mbarriers.  Warp 0 lane 0 issues the copies, warp 1 lane 0
// issues tcgen05.mma and commits each stage back to the producer, all four warps read the
// accumulator with tcgen05.ld.  The other contractions of the mixed update run in FP32 on
// the CUDA cores; denominators, mixing, energy and residual stay in FP64.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include <cuda.h>  // CUtensorMap and its enums (the encoder is fetched through the runtime)
#include <cudaTypedefs.h>

#include "pnm_context.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int TC_M = 128;        // ab rows per tile (one TMEM lane per row)
constexpr int TC_BK = 64;        // cd elements per k-block
constexpr int TC_MAX_STAGES = 4;  // the ring depth is chosen per context by the autotuner
constexpr int TC_MAX_SPLIT = 4;   // k-range splits of one (channel, ab tile), also autotuned
constexpr uint32_t A_PLANE = TC_M * TC_BK * 2;  // bytes of one BF16 plane of a V tile
constexpr uint32_t CORE_LBO = 128;              // next core matrix along K
constexpr uint32_t CORE_SBO = (TC_BK / 8) * 128;  // next 8-row group along M/N

struct TCItem {
  int ch, mt, kb0, nkb;  // channel, ab tile, first k-block and number of k-blocks of this item
  int sys;               // system of the channel
  int npad, npp, nhh, plane;  // padded N, sizes, output plane (k-range split index)
  long voff;   // element offset of tile (mt, 0) in the V tile arena
  long boff;   // element offset of k-block 0 in the t tile arena
  long toff;   // element offset of the channel in the t layout
};

using namespace tc;

static_assert(TC_BK == 64, "tile_core_off assumes 64-element k-blocks");
__device__ __forceinline__ int core_off(int r, int k) { return tile_core_off(r, k); }

// ------------------------------------------------------------------------ kernels
// V tiles of the channels with a V_pppp block (setup): one CTA per (item, k-block).
// Read from the FP32-pair copy of V: its high part is the FP32 rounding of the FP64 element,
// the value the BF16 split starts from.
__global__ void k_pack_v(const TCItem* __restrict__ items, const f2* __restrict__ v_pppp,
                         const long* __restrict__ ch_vpp_off, __nv_bfloat16* __restrict__ vt) {
  TCItem it = items[blockIdx.x];  // an unsplit item: kb0 = 0, nkb = all k-blocks
  int kb = blockIdx.y;
  if (kb >= it.nkb) return;
  const f2* V = v_pppp + ch_vpp_off[it.ch];
  __nv_bfloat16* hi = vt + it.voff + (long)kb * 2 * (TC_M * TC_BK);
  __nv_bfloat16* lo = hi + TC_M * TC_BK;
  // V is symmetric (bit for bit: <ab|v|cd> and <cd|v|ab> are evaluated by the same
  // arithmetic), so the element (cd, ab) is read as (ab, cd): consecutive threads then read
  // consecutive doubles of one row.
  for (int e = threadIdx.x; e < TC_M * TC_BK; e += blockDim.x) {
    int r = e / TC_BK, k = e % TC_BK;
    int ab = it.mt * TC_M + r, cd = kb * TC_BK + k;
    double x = (ab < it.npp && cd < it.npp) ? (double)V[(long)ab * it.npp + cd].hi : 0.0;
    __nv_bfloat16 h, l;
    split_bf16(x, h, l);
    hi[core_off(r, k)] = h;
    lo[core_off(r, k)] = l;
  }
}

// t tiles of the channels with a V_pppp block, in the ladder basis (before every tensor-core
// ladder): one CTA per (channel, k-block of 64 basis vectors); each tile entry gathers the
// signed members of its vector from the current amplitudes (FP32 copy in the iteration, FP64
// for the operator call) and stores the BF16 hi/lo split.
template <typename T_>
__global__ void k_pack_t(const int4* __restrict__ pk, const long* __restrict__ pk_boff,
                         DevState D, const LoopCtl* __restrict__ ctl, __nv_bfloat16* __restrict__ bt) {
  int4 p = pk[blockIdx.x];  // (channel, k-block, npad, 0)
  int c = p.x, kb = p.y, npad = p.z;
  if (sys_done(D, ctl, D.ch_sys[c])) return;
  int npp = D.ch_npp[c], nh = D.ch_nhh[c], nl = D.ch_nlad[c], off = D.ch_pp_off[c];
  const T_* t;
  if constexpr (std::is_same<T_, double>::value) t = cur_t(D, ctl) + D.ch_t_off[c];
  else t = cur_t32(D, ctl) + D.ch_t_off[c];
  __nv_bfloat16* hi = bt + pk_boff[blockIdx.x];
  __nv_bfloat16* lo = hi + npad * TC_BK;
  for (int e = threadIdx.x; e < npad * TC_BK; e += blockDim.x) {
    int n = e / TC_BK, k = e % TC_BK;
    int q = kb * TC_BK + k;
    T_ x = 0;
    if (n < nh && q < nl) {
      int2 m = D.lad_mem[off + q];
      T_ a = t[(long)n * npp + (m.x > 0 ? m.x : -m.x) - 1];
      x = m.x > 0 ? a : -a;
      if (m.y != 0) {
        T_ b = t[(long)n * npp + (m.y > 0 ? m.y : -m.y) - 1];
        x += m.y > 0 ? b : -b;
      }
    }
    __nv_bfloat16 h, l;
    split_bf16((double)x, h, l);
    hi[core_off(n, k)] = h;
    lo[core_off(n, k)] = l;
  }
}

// Persistent grouped pp ladder: R^T(ij, ab) = sum_cd t(ij, cd) V(cd, ab) for every (channel,
// ab tile, k-range) item of every system in one launch.  CTA c takes items cta_off[c] ...
// cta_off[c+1] - 1 (a longest-first greedy plan of the host balances the CTAs); warp 0 streams the V and t tiles of
// its items through an mbarrier ring of bulk-async copies without a break between items,
// warp 1 issues the BF16x3 MMAs (hi*hi + hi*lo + lo*hi, FP32 accumulator in tensor memory)
// into one of two accumulator buffers, and warps 2-5 drain the other buffer (item j-1) while
// item j accumulates.  Every wait is bounded; a wait that runs out sets ctl->dev_error and
// the CTA winds down (its own copies waited for, tensor memory freed).
constexpr int PP_THREADS = 192;

__global__ void __launch_bounds__(PP_THREADS, 1) k_pp_tc(const __grid_constant__ CUtensorMap tmap_v,
                                                         const TCItem* __restrict__ items,
                                                         const int* __restrict__ cta_off,
                                                         const SysCtl* __restrict__ sc,
                                                         const __nv_bfloat16* __restrict__ vt,
                                                         const __nv_bfloat16* __restrict__ bt,
                                                         float* __restrict__ rpp32, LoopCtl* __restrict__ ctl,
                                                         uint32_t stage_bytes, int nst, long plane_stride) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + TC_MAX_STAGES;
  uint64_t* tfull = empty + TC_MAX_STAGES;
  uint64_t* tempty = tfull + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tempty + 2);
  unsigned char* stage0 = smem + 1024;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ int err;
  const int i_begin = cta_off[blockIdx.x], i_end = cta_off[blockIdx.x + 1];
  // items of converged systems are skipped by all three roles alike (the flags do not change
  // during a launch)
  const bool skip = ctl->skip_done != 0;

  if (threadIdx.x == 0) {
    err = 0;
    for (int s = 0; s < nst; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);  // one arrival per epilogue warp
    }
    mbar_fence_init();
  }
  if (warp == 0) {
    tmem_alloc(tslot, 128);
    tmem_relinquish();
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      // producer: per stage one tiled tensor copy of the V tile (hi, lo planes: 256 rows of 64
      // BF16; each read once per launch, so marked first to evict from L2) and one bulk copy of
      // the t tile
      const uint64_t vpol = policy_evict_first();
      long g = 0;
      bool ok = true;
      for (int i = i_begin; i < i_end && ok; i++) {
        const TCItem it = items[i];
        if (skip && sc[it.sys].done) continue;
        const uint32_t b_plane = (uint32_t)it.npad * TC_BK * 2;
        const __nv_bfloat16* tb = bt + it.boff + (long)it.kb0 * 2 * (it.npad * TC_BK);
        for (int kb = 0; kb < it.nkb; kb++) {
          int s = (int)(g % nst);
          long use = g / nst;
          if (use > 0 && !mbar_wait(&empty[s], (uint32_t)((use - 1) & 1))) {
            err = 1;
            ok = false;
            break;
          }
          unsigned char* st = stage0 + s * stage_bytes;
          mbar_expect_tx(&full[s], 2 * A_PLANE + 2 * b_plane);
          tma_load_2d_hint(st, &tmap_v, 0, (int)((it.voff + (long)(it.kb0 + kb) * 2 * (TC_M * TC_BK)) / TC_BK),
                           &full[s], vpol);
          bulk_g2s(st + 2 * A_PLANE, tb + (long)kb * 2 * (it.npad * TC_BK), 2 * b_plane, &full[s]);
          g++;
        }
      }
      // every copy this thread started has landed before the CTA may retire
      for (long k = (g > nst ? g - nst : 0); k < g; k++)
        if (!mbar_wait(&full[k % nst], (uint32_t)((k / nst) & 1))) err = 1;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      long g = 0;
      int j = 0;
      bool ok = true;
      for (int i = i_begin; i < i_end && ok; i++) {
        const TCItem it = items[i];
        if (skip && sc[it.sys].done) continue;
        const int buf = j & 1;
        if (j >= 2 && !mbar_wait(&tempty[buf], (uint32_t)(((j >> 1) - 1) & 1))) {
          err = 1;
          break;
        }
        fence_after();
        const uint32_t dt = tbase + (uint32_t)(buf * 64);
        const uint32_t b_plane = (uint32_t)it.npad * TC_BK * 2;
        const uint32_t idesc = idesc_bf16(TC_M, it.npad);
        for (int kb = 0; kb < it.nkb; kb++) {
          int s = (int)(g % nst);
          long use = g / nst;
          if (!mbar_wait(&full[s], (uint32_t)(use & 1))) {
            err = 1;
            ok = false;
            break;
          }
          fence_after();
          unsigned char* a_hi = stage0 + s * stage_bytes;
          unsigned char* a_lo = a_hi + A_PLANE;
          unsigned char* b_hi = a_hi + 2 * A_PLANE;
          unsigned char* b_lo = b_hi + b_plane;
#pragma unroll
          for (int ks = 0; ks < TC_BK / 16; ks++) {
            uint32_t o = ks * 2 * 128;  // two core matrices of K per MMA
            uint64_t ah = smem_desc(a_hi + o, CORE_LBO, CORE_SBO), al = smem_desc(a_lo + o, CORE_LBO, CORE_SBO);
            uint64_t bh = smem_desc(b_hi + o, CORE_LBO, CORE_SBO), bl = smem_desc(b_lo + o, CORE_LBO, CORE_SBO);
            mma_bf16(dt, ah, bh, idesc, (kb > 0 || ks > 0) ? 1u : 0u);
            mma_bf16(dt, ah, bl, idesc, 1u);
            mma_bf16(dt, al, bh, idesc, 1u);
          }
          commit(&empty[s]);
          g++;
        }
        if (ok) commit(&tfull[buf]);
        j++;
      }
    }
  } else {
    // epilogue warps 2-5: TMEM lane = ab row (quarter warp % 4), column = ij
    const int q = warp & 3;
    const int row = q * 32 + lane;
    int j = 0;
    for (int i = i_begin; i < i_end; i++) {
      const TCItem it = items[i];
      if (skip && sc[it.sys].done) continue;
      const int buf = j & 1;
      const bool ok = mbar_wait(&tfull[buf], (uint32_t)((j >> 1) & 1));
      fence_after();
      if (!ok) {
        if (lane == 0) err = 1;
        break;
      }
      const int ab = it.mt * TC_M + row;
      for (int c0 = 0; c0 < it.npad; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(tbase + (uint32_t)(buf * 64) + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, r);
        if (ab < it.npp) {
#pragma unroll
          for (int jj = 0; jj < 16; jj++) {
            int ij = c0 + jj;
            if (ij < it.nhh) rpp32[it.plane * plane_stride + it.toff + (long)ij * it.npp + ab] = __uint_as_float(r[jj]);
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
      j++;
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, 128);
  if (threadIdx.x == 0 && err) atomicExch(&ctl->dev_error, 1);
}

// T[(a,i)][(k,c)] = t_ik^ac of the current amplitudes through the signed index map (the FP32
// cross-channel copy the mixed ph term reads; later updates keep it current by scattering).
__global__ void k_remap_t32(DevState D, const LoopCtl* __restrict__ ctl, float* __restrict__ xt, long n) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  int code = D.xmap[e];
  const float* t32 = cur_t32(D, ctl);
  float g = code == 0 ? 0.0f : t32[code > 0 ? code - 1 : -code - 1];
  xt[e] = code < 0 ? -g : g;
}

// FP32 copy of the current amplitudes.
__global__ void k_to_float_cur(DevState D, const LoopCtl* __restrict__ ctl, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float* dst = (ctl->iter & 1) ? D.t32_1 : D.t32_0;
  dst[i] = (float)cur_t(D, ctl)[i];
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

template <typename T>
T* mdalloc(pnm_ctx* ctx, size_t n) {
  return ctx_alloc<T>(ctx, n);
}

}  // namespace

struct MixedState {
  __nv_bfloat16* vt = nullptr;
  __nv_bfloat16* bt = nullptr;
  float *rpp32 = nullptr, *xw32 = nullptr, *xv132 = nullptr;
  float* xt32 = nullptr;  // T of the ph term, cross-channel layout, written by the update
  float* xq32 = nullptr;  // Q of the ph term, cross-channel layout, gathered by the update
  double* aw = nullptr;   // alpha / eps_ij^ab per amplitude (the step of the mixed update)
  double aw_alpha = -1.0;  // the alpha aw was made for
  TCItem* items = nullptr;
  int nitems = 0;
  int4* pk = nullptr;
  long* pk_boff = nullptr;
  int npk = 0;
  uint32_t stage_bytes = 0;
  size_t smem = 0;
  int nst = 3, ksplit = 1;  // chosen by the autotuner
  int grid = 1;             // CTAs of the persistent ladder
  int* cta_off = nullptr;   // per CTA: first item (items grouped by CTA), then the total
  CUtensorMap tmap_v;       // the V tile arena for the tiled tensor copies
  const SysCtl* sysctl = nullptr;  // the context's per-system loop state
  float tuned_us = 0.0f;
};

// Items of the tensor-core ladder for one k-range split factor: each (channel, ab tile)
// becomes up to `split` items over consecutive k-block ranges (never empty).
// Sorted by decreasing k-block count, so that the persistent kernel's round robin over CTAs
// balances.
static std::vector<TCItem> split_items(const std::vector<TCItem>& base, int split) {
  std::vector<TCItem> out;
  for (const TCItem& b : base) {
    int parts = std::min(split, b.nkb);
    for (int p = 0; p < parts; p++) {
      TCItem t = b;
      t.kb0 = (int)((long)b.nkb * p / parts);
      t.nkb = (int)((long)b.nkb * (p + 1) / parts) - t.kb0;
      t.plane = p;
      out.push_back(t);
    }
  }
  std::stable_sort(out.begin(), out.end(), [](const TCItem& x, const TCItem& y) { return x.nkb > y.nkb; });
  return out;
}

// Grid of the persistent ladder: every CTA that fits on the GPU at this shared-memory size.
static int pp_grid(size_t smem, int nitems) {
  int dev = 0, nsm = 1, per_sm = 1;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pp_tc, PP_THREADS, smem));
  // at most 4 CTAs per SM: 4 x 128 tensor-memory columns fill the SM's 512
  return std::max(1, std::min(nitems, nsm * std::min(4, std::max(1, per_sm))));
}

// Longest-first greedy plan: items (in decreasing cost) go one by one to the least loaded CTA
// (cost = k-blocks + 1 for the epilogue); returns the items grouped by CTA and the CTA offsets.
static void plan_items(const std::vector<TCItem>& its, int grid, std::vector<TCItem>* order, std::vector<int>* off) {
  std::vector<std::vector<int>> per(grid);
  std::vector<std::pair<long, int>> heap;
  for (int c = 0; c < grid; c++) heap.push_back({0L, c});
  auto cmp = [](const std::pair<long, int>& a, const std::pair<long, int>& b) {
    return a.first != b.first ? a.first > b.first : a.second > b.second;
  };
  std::make_heap(heap.begin(), heap.end(), cmp);
  for (int i = 0; i < (int)its.size(); i++) {
    std::pop_heap(heap.begin(), heap.end(), cmp);
    auto& h = heap.back();
    per[h.second].push_back(i);
    h.first += its[i].nkb + 1;
    std::push_heap(heap.begin(), heap.end(), cmp);
  }
  order->clear();
  off->assign(grid + 1, 0);
  for (int c = 0; c < grid; c++) {
    for (int i : per[c]) order->push_back(its[i]);
    (*off)[c + 1] = (int)order->size();
  }
}

static void launch_pp_tc(const TCItem* items, const int* cta_off, int grid, const MixedState* M, size_t smem,
                         int nst, LoopCtl* ctl, long nt, cudaStream_t s) {
  if (grid > 0)
    k_pp_tc<<<grid, PP_THREADS, smem, s>>>(M->tmap_v, items, cta_off, M->sysctl, M->vt, M->bt, M->rpp32, ctl,
                                           M->stage_bytes, nst, nt);
}

// Tensor map of the V tile arena as a 2-D BF16 tensor of rows x 64 (128-byte rows); one box
// is a whole tile (hi and lo planes, 256 rows).
static CUtensorMap v_tensor_map(__nv_bfloat16* vt, long elems) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!encode) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
      CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
      if (q != cudaDriverEntryPointSuccess || !fn) throw PnmError{PNM_ECUDA, "cuTensorMapEncodeTiled not available"};
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
  }
  CUtensorMap map;
  cuuint64_t dims[2] = {(cuuint64_t)TC_BK, (cuuint64_t)(elems / TC_BK)};
  cuuint64_t strides[1] = {(cuuint64_t)TC_BK * 2};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)(2 * TC_M)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, vt, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw PnmError{PNM_ECUDA, "cuTensorMapEncodeTiled failed for the V tiles"};
  return map;
}

// Tile choices already measured in this process, per channel-size signature.
static std::mutex g_tile_mu;
static std::map<std::string, std::tuple<int, int, float>> g_tile_cache;

void pnm_prepare_mixed(pnm_ctx* ctx) {
  if (ctx->mixed) return;
  cudaStream_t s = ctx->stream;
  pnm_need_vpp_f2(ctx);  // the V tiles are split from it
  MixedState* M = new MixedState();
  M->sysctl = ctx->sysctl;
  try {
    std::vector<TCItem> items;
    std::vector<int4> pk;
    std::vector<long> pk_boff;
    long voff = 0, boff = 0;
    int max_npad = 16, max_nkb = 1;
    for (int c = 0; c < ctx->nch; c++) {
      if (!ctx->h_vpp[c]) continue;
      int npp = ctx->h_nlad[c], nh = ctx->h_nhh[c];  // the ladder basis is the GEMM's M and K
      int npad = std::max(16, (nh + 15) / 16 * 16);
      if (npad > 64) throw PnmError{PNM_EINVAL, "n_hh > 64 in one channel: tensor-core tile too small"};
      int nmt = (npp + TC_M - 1) / TC_M, nkb = (npp + TC_BK - 1) / TC_BK;
      max_npad = std::max(max_npad, npad);
      max_nkb = std::max(max_nkb, nkb);
      for (int mt = 0; mt < nmt; mt++) {
        TCItem t{};
        t.ch = c;
        t.mt = mt;
        t.kb0 = 0;
        t.plane = 0;
        t.nkb = nkb;
        t.npad = npad;
        t.npp = npp;
        t.nhh = nh;
        t.voff = voff + (long)mt * nkb * 2 * (TC_M * TC_BK);
        t.boff = boff;
        t.toff = ctx->h_s_off[c];
        t.sys = ctx->h_ch_sys[c];
        items.push_back(t);
      }
      for (int kb = 0; kb < nkb; kb++) {
        pk.push_back(make_int4(c, kb, npad, 0));
        pk_boff.push_back(boff + (long)kb * 2 * npad * TC_BK);
      }
      voff += (long)nmt * nkb * 2 * (TC_M * TC_BK);
      boff += (long)nkb * 2 * npad * TC_BK;
    }
    M->nitems = (int)items.size();
    M->npk = (int)pk.size();
    const long vt_elems = std::max<long>(voff, 2L * TC_M * TC_BK);  // at least one whole box
    M->vt = mdalloc<__nv_bfloat16>(ctx, vt_elems);
    M->tmap_v = v_tensor_map(M->vt, vt_elems);
    M->bt = mdalloc<__nv_bfloat16>(ctx, boff);
    M->items = mdalloc<TCItem>(ctx, split_items(items, TC_MAX_SPLIT).size());
    M->pk = mdalloc<int4>(ctx, pk.size());
    M->pk_boff = mdalloc<long>(ctx, pk_boff.size());
    if (!items.empty())
      CUDA_TRY(cudaMemcpyAsync(M->items, items.data(), sizeof(TCItem) * items.size(), cudaMemcpyHostToDevice, s));
    if (!pk.empty()) {
      CUDA_TRY(cudaMemcpyAsync(M->pk, pk.data(), sizeof(int4) * pk.size(), cudaMemcpyHostToDevice, s));
      CUDA_TRY(cudaMemcpyAsync(M->pk_boff, pk_boff.data(), sizeof(long) * pk_boff.size(),
                               cudaMemcpyHostToDevice, s));
    }
    // padding rows/columns of the t tiles are never written again: they stay zero
    CUDA_TRY(cudaMemsetAsync(M->bt, 0, sizeof(__nv_bfloat16) * std::max<long>(boff, 1), s));
    ctx->d.t32_0 = mdalloc<float>(ctx, ctx->nt);
    ctx->d.t32_1 = mdalloc<float>(ctx, ctx->nt);
    ctx->d.chi32 = mdalloc<float>(ctx, ctx->nvhh);
    ctx->d.v32 = mdalloc<float>(ctx, ctx->nt);
    ctx->d.vhh32 = mdalloc<float>(ctx, ctx->nvhh);
    ctx->d.sij32 = mdalloc<float>(ctx, ctx->n_hh_pairs);
    ctx->d.sab32 = mdalloc<float>(ctx, ctx->n_pp_pairs);
    ctx->d.dchi32 = mdalloc<float>(ctx, ctx->nsp_total);
    if (ctx->nt > 0)
      k_to_float<<<(unsigned)((ctx->nt + 255) / 256), 256, 0, s>>>(ctx->d.v_pphh, ctx->d.v32, ctx->nt);
    if (ctx->nvhh > 0)
      k_to_float<<<(unsigned)((ctx->nvhh + 255) / 256), 256, 0, s>>>(ctx->d.v_hhhh, ctx->d.vhh32, ctx->nvhh);
    M->rpp32 = mdalloc<float>(ctx, (size_t)TC_MAX_SPLIT * ctx->ns);
    // planes a channel with fewer k-blocks than the split never writes stay zero
    CUDA_TRY(cudaMemsetAsync(M->rpp32, 0, sizeof(float) * TC_MAX_SPLIT * std::max<long>(ctx->ns, 1), s));
    M->xw32 = mdalloc<float>(ctx, ctx->nxt);
    M->xv132 = mdalloc<float>(ctx, ctx->nxc);
    M->xt32 = mdalloc<float>(ctx, ctx->nxt);
    // entries no amplitude maps to (repeated state index) stay zero
    CUDA_TRY(cudaMemsetAsync(M->xt32, 0, sizeof(float) * std::max<long>(ctx->nxt, 1), s));
    M->xq32 = mdalloc<float>(ctx, ctx->nxt);
    M->aw = mdalloc<double>(ctx, ctx->nt);
    if (ctx->nxt > 0)
      k_to_float<<<(unsigned)((ctx->nxt + 255) / 256), 256, 0, s>>>(ctx->d.x_w, M->xw32, ctx->nxt);
    if (ctx->nxc > 0)
      k_to_float<<<(unsigned)((ctx->nxc + 255) / 256), 256, 0, s>>>(ctx->d.x_v1, M->xv132, ctx->nxc);
    if (M->nitems > 0)
      k_pack_v<<<dim3(M->nitems, max_nkb), 256, 0, s>>>(M->items, ctx->vpp_f2, ctx->d.ch_vpp_off, M->vt);
    CUDA_TRY(cudaGetLastError());
    M->stage_bytes = (2 * A_PLANE + 2 * (uint32_t)max_npad * TC_BK * 2 + 1023) / 1024 * 1024;
    auto smem_for = [&](int nst) { return 1024 + (size_t)nst * M->stage_bytes + 8192; };  // tail guard
    if (smem_for(2) > 227 * 1024) throw PnmError{PNM_EINVAL, "tensor-core stage ring exceeds shared memory"};
    int max_st = TC_MAX_STAGES;
    while (smem_for(max_st) > 227 * 1024) max_st--;
    smem_at_least(k_pp_tc, smem_for(max_st));
    CUDA_TRY(cudaStreamSynchronize(s));
    // Autotuner: time every (k-range split, ring depth) on this context's channels and keep
    // the fastest.  The ladder's cost does not depend on the amplitude values.
    CUDA_TRY(cudaMemsetAsync(&ctx->ctl->dev_error, 0, sizeof(int), s));
    float best = 1e30f;
    std::vector<TCItem> best_items = items;
    const std::string key = pnm_shape_key(ctx);
    bool cached = false;
    {
      std::lock_guard<std::mutex> lock(g_tile_mu);
      auto f = g_tile_cache.find(key);
      if (f != g_tile_cache.end()) {
        M->ksplit = std::get<0>(f->second);
        M->nst = std::min(std::get<1>(f->second), max_st);
        best = std::get<2>(f->second) * 5 / 1000.0f;
        best_items = split_items(items, M->ksplit);
        cached = true;
      }
    }
    TCItem* trial = mdalloc<TCItem>(ctx, split_items(items, TC_MAX_SPLIT).size());
    int dev = 0, nsm = 1;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int* trial_off = mdalloc<int>(ctx, 4 * (size_t)nsm + 1);
    M->cta_off = mdalloc<int>(ctx, 4 * (size_t)nsm + 1);
    std::vector<TCItem> order;
    std::vector<int> off;
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    for (int split : {1, 2, 4}) {
      if (cached) break;
      std::vector<TCItem> its = split_items(items, split);
      if (its.empty()) break;
      for (int nst = 2; nst <= max_st; nst++) {
        int grid = pp_grid(smem_for(nst), (int)its.size());
        plan_items(its, grid, &order, &off);
        CUDA_TRY(cudaMemcpyAsync(trial, order.data(), sizeof(TCItem) * order.size(), cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(trial_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, s));
        for (int w = 0; w < 2; w++)
          launch_pp_tc(trial, trial_off, grid, M, smem_for(nst), nst, ctx->ctl, ctx->ns, s);
        CUDA_TRY(cudaEventRecord(e0, s));
        for (int rep = 0; rep < 5; rep++)
          launch_pp_tc(trial, trial_off, grid, M, smem_for(nst), nst, ctx->ctl, ctx->ns, s);
        CUDA_TRY(cudaEventRecord(e1, s));
        CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0;
        CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
          best = ms;
          best_items = its;
          M->nst = nst;
          M->ksplit = split;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CUDA_TRY(cudaGetLastError());
    int dev_err = 0;
    CUDA_TRY(cudaMemcpy(&dev_err, &ctx->ctl->dev_error, sizeof(int), cudaMemcpyDeviceToHost));
    if (dev_err) throw PnmError{PNM_ETIMEOUT, "a device-side wait ran out of its budget while tuning"};
    M->tuned_us = best / 5 * 1000.0f;
    if (!cached) {
      std::lock_guard<std::mutex> lock(g_tile_mu);
      g_tile_cache[key] = std::make_tuple(M->ksplit, M->nst, M->tuned_us);
    }
    M->smem = smem_for(M->nst);
    M->nitems = (int)best_items.size();
    M->grid = pp_grid(M->smem, M->nitems);
    plan_items(best_items, M->grid, &order, &off);
    CUDA_TRY(cudaMemcpyAsync(M->items, order.data(), sizeof(TCItem) * order.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(M->cta_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemsetAsync(M->rpp32, 0, sizeof(float) * TC_MAX_SPLIT * std::max<long>(ctx->ns, 1), s));
    CUDA_TRY(cudaStreamSynchronize(s));
  } catch (...) {
    delete M;
    throw;
  }
  ctx->mixed = M;
}

void pnm_enqueue_body_mixed(pnm_ctx* ctx, int use_cond, cudaGraphConditionalHandle h) {
  MixedState* M = ctx->mixed;
  cudaStream_t s_ph = pnm_concurrent(ctx) ? ctx->side[0] : ctx->stream;
  cudaStream_t s_pp = pnm_concurrent(ctx) ? ctx->side[1] : ctx->stream;
  pnm_fork(ctx);
  if (ctx->nx > 0) {
    prof_begin(ctx, KID_PH32);
    launch_ph_mix(ctx, M->xt32, M->xw32, M->xv132, M->xq32, s_ph);
    prof_end(ctx);
  }
  if (M->nitems > 0) {
    // t tiles of the current amplitudes in the ladder basis, then the ladder (same stream)
    prof_begin(ctx, KID_PACK);
    k_pack_t<float><<<M->npk, 256, 0, s_pp>>>(M->pk, M->pk_boff, ctx->d, ctx->ctl, M->bt);
    prof_end(ctx);
    prof_begin(ctx, KID_PP_TC);
    launch_pp_tc(M->items, M->cta_off, M->grid, M, M->smem, M->nst, ctx->ctl, ctx->ns, s_pp);
    prof_end(ctx);
  }
  pnm_enqueue_stats(ctx, true);
  pnm_join(ctx);
  prof_begin(ctx, KID_UPDATE_MIX);
  launch_update_mix(ctx, M->rpp32, M->xq32, M->aw, M->xt32, use_cond, h, M->ksplit, ctx->ns);
  prof_end(ctx);
}

// Before the first mixed update of a solve: the FP32 copies of the start amplitudes (t32 and the
// ph term's T; the t tiles of the ladder are packed at the start of every mixed update), and
// alpha / eps_ij^ab if alpha changed.
// FP32 copies of the starting amplitudes, in the direct and the cross-channel layouts.
void pnm_mixed_pack_t(pnm_ctx* ctx) {
  MixedState* M = ctx->mixed;
  if (ctx->nt > 0)
    k_to_float_cur<<<(unsigned)((ctx->nt + 255) / 256), 256, 0, ctx->stream>>>(ctx->d, ctx->ctl, ctx->nt);
  if (ctx->nxt > 0)
    k_remap_t32<<<(unsigned)((ctx->nxt + 255) / 256), 256, 0, ctx->stream>>>(ctx->d, ctx->ctl, M->xt32, ctx->nxt);
  CUDA_TRY(cudaGetLastError());
}

// alpha / eps_ij^ab per amplitude for this mixing (recomputed only when alpha changes).
void pnm_mixed_set_alpha(pnm_ctx* ctx, double alpha) {
  MixedState* M = ctx->mixed;
  if (alpha != M->aw_alpha) {
    pnm_alpha_inv(ctx, alpha, M->aw);
    M->aw_alpha = alpha;
  }
  CUDA_TRY(cudaGetLastError());
}

void pnm_mixed_pack_initial(pnm_ctx* ctx, double alpha) {
  pnm_mixed_pack_t(ctx);
  pnm_mixed_set_alpha(ctx, alpha);
}

const double* pnm_mixed_aw(const pnm_ctx* ctx) {
  if (!ctx->mixed) throw PnmError{PNM_EINVAL, "the mixed-precision path has not been prepared"};
  return ctx->mixed->aw;
}

void pnm_mixed_tuning(const pnm_ctx* ctx, int* ksplit, int* stages, float* us, int* serial_mask) {
  if (serial_mask)
    *serial_mask = (ctx->sched_tuned[0] ? (ctx->serial_sched[0] ? 1 : 0) : 4) |
                   (ctx->sched_tuned[1] ? (ctx->serial_sched[1] ? 2 : 0) : 8) |
                   (ctx->sched_tuned[2] ? (ctx->serial_sched[2] ? 16 : 0) : 32);
  if (!ctx->mixed) throw PnmError{PNM_EINVAL, "the mixed-precision path has not been prepared"};
  if (ksplit) *ksplit = ctx->mixed->ksplit;
  if (stages) *stages = ctx->mixed->nst;
  if (us) *us = ctx->mixed->tuned_us;
}

void pnm_free_mixed(pnm_ctx* ctx) {
  delete ctx->mixed;  // device arenas are in ctx->owned
  ctx->mixed = nullptr;
}

// Apply only the particle-particle ladder to amplitudes t (library order, system `sys`):
// r = sum_{c<d} <ab|v|cd> t_cd^ij on channels with a V_pppp block, 0 elsewhere.  Uses the solver's
// buffers (the iteration state is reset).
void pnm_apply_pp(pnm_ctx* ctx, int sys, int precision, const double* t, double* r, size_t n) {
  const SysInfo& S = ctx->sys[sys];
  cudaStream_t s = ctx->stream;
  if (n != (size_t)(S.t_end - S.t_begin)) throw PnmError{PNM_EINVAL, "size mismatch"};
  if (precision == PNM_PREC_BF16X3) pnm_prepare_mixed(ctx);
  int zero = 0;
  CUDA_TRY(cudaMemcpyAsync(&ctx->ctl->iter, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(&ctx->ctl->dev_error, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(&ctx->ctl->skip_done, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(ctx->d.t0 + S.t_begin, t, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  std::vector<double> out(ctx->nt, 0.0);
  if (precision == PNM_PREC_BF16X3) {
    MixedState* M = ctx->mixed;
    CUDA_TRY(cudaMemsetAsync(M->rpp32, 0, sizeof(float) * TC_MAX_SPLIT * std::max<long>(ctx->ns, 1), s));
    if (M->npk > 0) k_pack_t<double><<<M->npk, 256, 0, s>>>(M->pk, M->pk_boff, ctx->d, ctx->ctl, M->bt);
    launch_pp_tc(M->items, M->cta_off, M->grid, M, M->smem, M->nst, ctx->ctl, ctx->ns, s);
    pnm_lad_expand(ctx, M->rpp32, M->ksplit, ctx->ns, out.data());
  } else {
    if (precision == PNM_PREC_F32PAIR) {
      pnm_prepare_f2(ctx);
      pnm_split_cur(ctx, s);
    }
    if (precision == PNM_PREC_FP64) pnm_need_vpp64(ctx);
    CUDA_TRY(cudaMemsetAsync(ctx->d.rpp, 0, sizeof(double) * std::max<long>(ctx->ns, 1), s));
    // every row: the operator acts on any amplitudes
    pnm_launch_pp64(ctx, s, false, precision == PNM_PREC_F32PAIR ? ctx->vpp_f2 : nullptr);
    if (precision == PNM_PREC_F32PAIR)
      pnm_lad_expand(ctx, reinterpret_cast<const f2*>(ctx->d.rpp), 1, ctx->ns, out.data());
    else
      pnm_lad_expand(ctx, ctx->d.rpp, 1, ctx->ns, out.data());
  }
  int err = 0;
  CUDA_TRY(cudaMemcpy(&err, &ctx->ctl->dev_error, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) throw PnmError{PNM_ETIMEOUT, "a device-side wait ran out of its budget"};
  for (int c = S.ch_begin; c < S.ch_end; c++) {
    long o = ctx->h_t_off[c], len = (long)ctx->h_nhh[c] * ctx->h_npp[c];
    for (long z = 0; z < len; z++) r[o - S.t_begin + z] = ctx->h_vpp[c] ? out[o + z] : 0.0;
  }
}

// out[z] = Q_ij^ab - Q_ji^ab - Q_ij^ba + Q_ji^ba of amplitude z from the cross-channel Q (FP32,
// FP64, or FP32 pairs summed as pairs).
template <typename T>
__global__ void k_ph_assemble(DevState D, const T* __restrict__ xq, long nt, double* __restrict__ out) {
  using A = Arith<T>;
  long z = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= nt) return;
  int4 q = D.qmap[z];
  T a0 = q.x >= 0 ? xq[q.x] : A::zero(), a1 = q.y >= 0 ? xq[q.y] : A::zero();
  T a2 = q.z >= 0 ? xq[q.z] : A::zero(), a3 = q.w >= 0 ? xq[q.w] : A::zero();
  if constexpr (std::is_same<T, f2>::value)
    out[z] = A::to_double(A::sub(A::sub(a0, a1), A::sub(a2, a3)));
  else
    out[z] = ((double)a0 - (double)a1) - ((double)a2 - (double)a3);
}

// The ph term P(ij)P(ab) sum_kc t_ik^ac chi_kb^cj as an operator on the amplitudes of one
// system (FP64 kernels, or the mixed-precision ones: FP32 T copy, tensor-core or CUDA-core
// contractions by channel size).
void pnm_apply_ph(pnm_ctx* ctx, int sys, int precision, const double* t, double* r, size_t n) {
  const SysInfo& S = ctx->sys[sys];
  cudaStream_t s = ctx->stream;
  if (n != (size_t)(S.t_end - S.t_begin)) throw PnmError{PNM_EINVAL, "size mismatch"};
  if (precision == PNM_PREC_BF16X3) pnm_prepare_mixed(ctx);
  int zero = 0;
  CUDA_TRY(cudaMemcpyAsync(&ctx->ctl->iter, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(&ctx->ctl->dev_error, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(&ctx->ctl->skip_done, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(ctx->d.t0 + S.t_begin, t, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  pnm_flip_symmetrise(ctx, ctx->d.t0, s);  // the term of the flip-symmetric part of t
  unsigned nb = (unsigned)((ctx->nt + 255) / 256);
  if (!ctx->expand_buf) ctx->expand_buf = ctx_alloc<double>(ctx, ctx->nt);  // the assembled term
  if (precision == PNM_PREC_BF16X3) {
    MixedState* M = ctx->mixed;
    k_to_float_cur<<<nb, 256, 0, s>>>(ctx->d, ctx->ctl, ctx->nt);
    if (ctx->nxt > 0)
      k_remap_t32<<<(unsigned)((ctx->nxt + 255) / 256), 256, 0, s>>>(ctx->d, ctx->ctl, M->xt32, ctx->nxt);
    if (ctx->nx > 0) launch_ph_mix(ctx, M->xt32, M->xw32, M->xv132, M->xq32, s);
    k_ph_assemble<float><<<nb, 256, 0, s>>>(ctx->d, M->xq32, ctx->nt, ctx->expand_buf);
  } else {
    if (precision == PNM_PREC_F32PAIR) {
      pnm_prepare_f2(ctx);
      pnm_split_cur(ctx, s);
      if (ctx->nx > 0) launch_ph_f2(ctx, ctx->t_pair, ctx->xw_f2, ctx->xv1_f2, s);
      k_ph_assemble<f2><<<nb, 256, 0, s>>>(ctx->d, reinterpret_cast<const f2*>(ctx->d.xq), ctx->nt, ctx->expand_buf);
    } else {
      if (ctx->nx > 0) launch_ph64(ctx, s);
      k_ph_assemble<double><<<nb, 256, 0, s>>>(ctx->d, ctx->d.xq, ctx->nt, ctx->expand_buf);
    }
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(r, ctx->expand_buf + S.t_begin, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  int err = 0;
  CUDA_TRY(cudaMemcpy(&err, &ctx->ctl->dev_error, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) throw PnmError{PNM_ETIMEOUT, "a device-side wait ran out of its budget"};
}

// Failure-path self test: one thread waits, with the bounded wait of the tensor-core
// kernels, on an mbarrier that nothing ever arrives on.  The wait gives up, the kernel
// records the failure in the context's device flag and returns; nothing traps or hangs.
__global__ void k_wait_selftest(LoopCtl* __restrict__ ctl) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0)) atomicExch(&ctl->dev_error, 1);
}

void pnm_selftest_wait(pnm_ctx* ctx) {
  int zero = 0, err = 0;
  CUDA_TRY(cudaMemcpyAsync(&ctx->ctl->dev_error, &zero, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  k_wait_selftest<<<1, 32, 0, ctx->stream>>>(ctx->ctl);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(&err, &ctx->ctl->dev_error, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  CUDA_TRY(cudaMemcpyAsync(&ctx->ctl->dev_error, &zero, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (err) throw PnmError{PNM_ETIMEOUT, "device-side wait ran out of its budget (self test)"};
}
