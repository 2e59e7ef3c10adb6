// api.cu -- the extern "C" entry points declared in include/pnmcc.h.
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <cmath>
#include <cstring>
#include <cstdio>
#include <cstdint>

#include "pnm_context.cuh"

static thread_local std::string g_last_error;

void pnm_set_error(int code, const std::string& msg) {
  g_last_error = "pnmcc error " + std::to_string(code) + ": " + msg;
}

template <typename F>
static int guarded(F&& f) {
  try {
    return f();
  } catch (const PnmError& e) {
    pnm_set_error(e.code, e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    pnm_set_error(PNM_ENOMEM, "host allocation failed");
    return PNM_ENOMEM;
  } catch (...) {
    pnm_set_error(PNM_EINVAL, "unexpected failure");
    return PNM_EINVAL;
  }
}

static cudaMemPool_t library_pool(int dev) {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  std::lock_guard<std::mutex> lock(mu);
  auto f = pools.find(dev);
  if (f != pools.end()) return f->second;
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool;
  CUDA_TRY(cudaMemPoolCreate(&pool, &props));
  uint64_t keep = ~0ull;  // freed blocks stay in the pool for reuse until the process ends
  CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
  pools[dev] = pool;
  return pool;
}

void pnm_smem_at_least(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<const void*, size_t> cur;
  std::lock_guard<std::mutex> lock(mu);
  size_t& c = cur[func];
  if (bytes <= c) return;
  CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  c = bytes;
}

void* pnm_pool_alloc(cudaStream_t s, size_t bytes) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  void* p = nullptr;
  if (cudaMallocFromPoolAsync(&p, bytes ? bytes : 1, library_pool(dev), s) != cudaSuccess) {
    cudaGetLastError();
    throw PnmError{PNM_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed"};
  }
  return p;
}

void pnm_pool_free(cudaStream_t s, void* p) {
  if (p) cudaFreeAsync(p, s);
}

void* pnm_ctx_alloc(pnm_ctx* ctx, size_t bytes) {
  void* p = pnm_pool_alloc(ctx->stream, bytes);
  ctx->owned.push_back(p);
  return p;
}

static void release(pnm_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.second);
  for (auto& g : ctx->graph_defs) cudaGraphDestroy(g.second);
  pnm_drop_solve_graphs(ctx);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  pnm_free_mixed(ctx);
  pnm_free_mlp(ctx);
  for (void* p : ctx->owned) pnm_pool_free(ctx->stream, p);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  for (int k = 0; k < 2; k++) {
    if (ctx->side[k]) cudaStreamDestroy(ctx->side[k]);
    if (ctx->ev_join[k]) cudaEventDestroy(ctx->ev_join[k]);
  }
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  for (auto& pr : ctx->prof_ev) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

static void check_sys(const pnm_ctx* ctx, int sys) {
  if (!ctx) throw PnmError{PNM_EINVAL, "null context"};
  if (sys < 0 || sys >= (int)ctx->sys.size()) throw PnmError{PNM_EINVAL, "system index out of range"};
}

extern "C" {

void pnm_default_opts(pnm_solve_opts* o) {
  if (!o) return;
  o->precision = PNM_PREC_FP64;
  o->mix_alpha = 0.5;
  o->tol_dE = 1e-10;
  o->tol_dE_per_N = 0.0;
  o->max_iter = 500;
  o->refine_sweeps = 0;
  o->init = PNM_INIT_MBPT2;
  o->host_loop = 0;
  o->terms = PNM_TERMS_FULL;
  o->refine_kernels = PNM_PREC_FP64;
}

const char* pnm_last_error(void) { return g_last_error.c_str(); }

int pnm_create_matter(int n, const int* N, const int* Z, const double* rho, const int* n2max,
                      const double* theta, const pnm_minnesota* params, void* stream,
                      pnm_ctx** out) {
  return guarded([&]() {
    if (!out || !N || !rho || !n2max || !params || n <= 0)
      throw PnmError{PNM_EINVAL, "null argument or empty batch"};
    *out = nullptr;
    pnm_ctx* ctx = new pnm_ctx();
    try {
      if (stream) {
        ctx->stream = (cudaStream_t)stream;
      } else {
        CUDA_TRY(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
      }
      for (auto& e : ctx->ev) CUDA_TRY(cudaEventCreate(&e));
      CUDA_TRY(cudaEventRecord(ctx->ev[2], ctx->stream));
      pnm_build(ctx, n, N, Z, rho, n2max, theta, *params);
      pnm_prepare_iteration(ctx);
      pnm_eref_all(ctx);
      CUDA_TRY(cudaEventRecord(ctx->ev[3], ctx->stream));
      CUDA_TRY(cudaStreamSynchronize(ctx->stream));
      float ms = 0;
      cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]);
      ctx->t_setup = ms;
    } catch (...) {
      release(ctx);
      throw;
    }
    *out = ctx;
    return PNM_OK;
  });
}

int pnm_create_twisted(int n, const int* N, const double* rho, const int* n2max,
                       const double* theta, const pnm_minnesota* params, void* stream,
                       pnm_ctx** out) {
  return pnm_create_matter(n, N, nullptr, rho, n2max, theta, params, stream, out);
}

int pnm_create_batch(int n, const int* N, const double* rho, const int* n2max,
                     const pnm_minnesota* params, void* stream, pnm_ctx** out) {
  return pnm_create_matter(n, N, nullptr, rho, n2max, nullptr, params, stream, out);
}

// Gauss-Legendre nodes and weights on [-1, 1]: Newton's method on P_n from the Chebyshev-like
// first guess cos(pi (i + 3/4) / (n + 1/2)); P_n and P_n' from the three-term recurrence
// (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}; w_i = 2 / ((1 - x_i^2) P_n'(x_i)^2).
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; i++) {
    double z = std::cos(PNM_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; it++) {
      double p0 = 1.0, p1 = 0.0;
      for (int k = 0; k < n; k++) {
        double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * k + 1.0) * z * p1 - k * p2) / (k + 1.0);
      }
      dp = n * (z * p0 - p1) / (z * z - 1.0);
      double dz = p0 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = 0.0;
    for (int k = 0; k < n; k++) {
      double p2 = p1;
      p1 = p0;
      p0 = ((2.0 * k + 1.0) * z * p1 - k * p2) / (k + 1.0);
    }
    dp = n * (z * p0 - p1) / (z * z - 1.0);
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

int pnm_twist_mesh(int nx, int ny, int nz, double* theta, double* weight) {
  return guarded([&]() {
    if (nx < 1 || ny < 1 || nz < 1 || nx > 64 || ny > 64 || nz > 64 || !theta || !weight)
      throw PnmError{PNM_EINVAL, "mesh sizes must be 1..64 per axis and outputs non-null"};
    int n3[3] = {nx, ny, nz};
    std::vector<double> th[3], wt[3];
    for (int a = 0; a < 3; a++) {
      std::vector<double> x, w;
      gauss_legendre(n3[a], x, w);
      th[a].resize(n3[a]);
      wt[a].resize(n3[a]);
      for (int i = 0; i < n3[a]; i++) {
        th[a][i] = 0.5 * PNM_PI * (x[i] + 1.0);
        wt[a][i] = 0.5 * w[i];  // (pi/2) w_i / pi: the 1/pi^3 of the average taken per axis
      }
    }
    long m = 0;
    for (int i = 0; i < nx; i++)
      for (int j = 0; j < ny; j++)
        for (int k = 0; k < nz; k++, m++) {
          theta[3 * m] = th[0][i];
          theta[3 * m + 1] = th[1][j];
          theta[3 * m + 2] = th[2][k];
          weight[m] = wt[0][i] * wt[1][j] * wt[2][k];
        }
    return PNM_OK;
  });
}

int pnm_create(int N, double rho, int n2max, const pnm_minnesota* params, void* stream,
               pnm_ctx** out) {
  return pnm_create_batch(1, &N, &rho, &n2max, params, stream, out);
}

int pnm_destroy(pnm_ctx* ctx) {
  return guarded([&]() {
    release(ctx);
    return PNM_OK;
  });
}

int pnm_num_systems(const pnm_ctx* ctx, int* n) {
  return guarded([&]() {
    if (!ctx || !n) throw PnmError{PNM_EINVAL, "null argument"};
    *n = (int)ctx->sys.size();
    return PNM_OK;
  });
}

int pnm_basis(const pnm_ctx* ctx, int sys, int* n_sp, int* n_holes, int8_t* nxyzs,
              double* eps_hf) {
  return guarded([&]() {
    check_sys(ctx, sys);
    const SysInfo& S = ctx->sys[sys];
    if (n_sp) *n_sp = S.nsp;
    if (n_holes) *n_holes = S.N;
    if (nxyzs)
      CUDA_TRY(cudaMemcpyAsync(nxyzs, ctx->d.nvec + S.sp_off, sizeof(char4) * S.nsp,
                               cudaMemcpyDeviceToHost, ctx->stream));
    if (eps_hf)
      CUDA_TRY(cudaMemcpyAsync(eps_hf, ctx->d.eps + S.sp_off, sizeof(double) * S.nsp,
                               cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return PNM_OK;
  });
}

int pnm_channels(const pnm_ctx* ctx, int sys, int kind, int* n_chan, int* n_pairs, int32_t* keys,
                 int32_t* sizes, int32_t* pairs) {
  return guarded([&]() {
    check_sys(ctx, sys);
    const SysInfo& S = ctx->sys[sys];
    cudaStream_t s = ctx->stream;
    if (kind == 0) {
      int c0 = S.ch_begin, c1 = S.ch_end;
      int nh = 0, np = 0;
      for (int c = c0; c < c1; c++) {
        nh += ctx->h_nhh[c];
        np += ctx->h_npp[c];
      }
      if (n_chan) *n_chan = c1 - c0;
      if (n_pairs) *n_pairs = nh + np;
      for (int c = c0; c < c1; c++) {
        if (keys) keys[c - c0] = ctx->h_key[c];
        if (sizes) {
          sizes[2 * (c - c0)] = ctx->h_nhh[c];
          sizes[2 * (c - c0) + 1] = ctx->h_npp[c];
        }
      }
      if (pairs && c1 > c0) {
        std::vector<int2> hh(nh), pp(np);
        CUDA_TRY(cudaMemcpyAsync(hh.data(), ctx->d.hh_pair + ctx->h_hh_off[c0], sizeof(int2) * nh,
                                 cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaMemcpyAsync(pp.data(), ctx->d.pp_pair + ctx->h_pp_off[c0], sizeof(int2) * np,
                                 cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        for (int k = 0; k < nh; k++) {
          pairs[2 * k] = hh[k].x - S.sp_off;
          pairs[2 * k + 1] = hh[k].y - S.sp_off;
        }
        for (int k = 0; k < np; k++) {
          pairs[2 * (nh + k)] = pp[k].x - S.sp_off;
          pairs[2 * (nh + k) + 1] = pp[k].y - S.sp_off;
        }
      }
    } else if (kind == 1) {
      int x0 = S.x_begin, x1 = S.x_end;
      int nph = 0, nhp = 0;
      for (int x = x0; x < x1; x++) {
        nph += ctx->h_x_nph[x];
        nhp += ctx->h_x_nhp[x];
      }
      if (n_chan) *n_chan = x1 - x0;
      if (n_pairs) *n_pairs = nph + nhp;
      if (keys && x1 > x0) {
        // keys are recomputed from the first row of each channel: key(n_a - n_i, s_a - s_i)
        std::vector<int2> ph(nph);
        CUDA_TRY(cudaMemcpyAsync(ph.data(), ctx->d.ph_pair + ctx->h_x_ph_off[x0],
                                 sizeof(int2) * nph, cudaMemcpyDeviceToHost, s));
        std::vector<char4> nv(S.nsp);
        CUDA_TRY(cudaMemcpyAsync(nv.data(), ctx->d.nvec + S.sp_off, sizeof(char4) * S.nsp,
                                 cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        for (int x = x0; x < x1; x++) {
          int2 pr = ph[ctx->h_x_ph_off[x] - ctx->h_x_ph_off[x0]];
          char4 a = nv[pr.x - S.sp_off], i = nv[pr.y - S.sp_off];
          int dw = a.w - i.w, slot, nq = S.species == 1 ? 3 : 9;
          if (S.species == 1) {
            slot = (dw + 2) / 2;
          } else {  // dw = (s_a - s_i) + 4 (t_a - t_i)
            int dt = dw >= 6 ? 2 : (dw <= -6 ? -2 : 0);
            slot = 3 * ((dw - 4 * dt + 2) / 2) + (dt + 2) / 2;
          }
          keys[x - x0] = (((a.x - i.x + S.m) * S.M + (a.y - i.y + S.m)) * S.M + (a.z - i.z + S.m)) * nq + slot;
        }
      }
      if (sizes)
        for (int x = x0; x < x1; x++) {
          sizes[2 * (x - x0)] = ctx->h_x_nph[x];
          sizes[2 * (x - x0) + 1] = ctx->h_x_nhp[x];
        }
      if (pairs && x1 > x0) {
        std::vector<int2> ph(nph), hp(nhp);
        CUDA_TRY(cudaMemcpyAsync(ph.data(), ctx->d.ph_pair + ctx->h_x_ph_off[x0],
                                 sizeof(int2) * nph, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaMemcpyAsync(hp.data(), ctx->d.hp_pair + ctx->h_x_hp_off[x0],
                                 sizeof(int2) * nhp, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        for (int k = 0; k < nph; k++) {
          pairs[2 * k] = ph[k].x - S.sp_off;
          pairs[2 * k + 1] = ph[k].y - S.sp_off;
        }
        for (int k = 0; k < nhp; k++) {
          pairs[2 * (nph + k)] = hp[k].x - S.sp_off;
          pairs[2 * (nph + k) + 1] = hp[k].y - S.sp_off;
        }
      }
    } else {
      throw PnmError{PNM_EINVAL, "kind must be 0 (direct) or 1 (cross)"};
    }
    return PNM_OK;
  });
}

int pnm_eref(const pnm_ctx* ctx, double* e_ref) {
  return guarded([&]() {
    if (!ctx || !e_ref) throw PnmError{PNM_EINVAL, "null argument"};
    for (size_t k = 0; k < ctx->sys.size(); k++) e_ref[k] = ctx->sys[k].eref;
    return PNM_OK;
  });
}

int pnm_mbpt2(pnm_ctx* ctx, double* dE) {
  return guarded([&]() {
    if (!ctx || !dE) throw PnmError{PNM_EINVAL, "null argument"};
    pnm_mbpt2_all(ctx, dE);
    return PNM_OK;
  });
}

int pnm_ladder_sizes(const pnm_ctx* ctx, int sys, int* n_chan, int32_t* nlad) {
  return guarded([&]() {
    check_sys(ctx, sys);
    const SysInfo& S = ctx->sys[sys];
    if (n_chan) *n_chan = S.ch_end - S.ch_begin;
    if (nlad)
      for (int c = S.ch_begin; c < S.ch_end; c++) nlad[c - S.ch_begin] = ctx->h_vpp[c] ? ctx->h_nlad[c] : 0;
    return PNM_OK;
  });
}

int pnm_mbpt3(pnm_ctx* ctx, double* e3) {
  return guarded([&]() {
    if (!ctx || !e3) throw PnmError{PNM_EINVAL, "null argument"};
    pnm_mbpt3_all(ctx, e3);
    return PNM_OK;
  });
}

int pnm_ccd_solve(pnm_ctx* ctx, const pnm_solve_opts* opts, double* dE, int* iters,
                  double* resid) {
  return guarded([&]() {
    if (!ctx || !opts) throw PnmError{PNM_EINVAL, "null argument"};
    return pnm_solve(ctx, *opts, dE, iters, resid);
  });
}

int pnm_energy_history(const pnm_ctx* ctx, int sys, double* hist, int cap, int* n) {
  return guarded([&]() {
    check_sys(ctx, sys);
    if (!ctx->hist) throw PnmError{PNM_EINVAL, "no solve has run"};
    SysCtl sc;
    CUDA_TRY(cudaMemcpyAsync(&sc, ctx->sysctl + sys, sizeof(SysCtl), cudaMemcpyDeviceToHost,
                             ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    int cnt = std::min(sc.iters + 1, ctx->hist_cap);
    cnt = std::min(cnt, cap);
    if (n) *n = cnt;
    if (hist && cnt > 0)
      CUDA_TRY(cudaMemcpyAsync(hist, ctx->hist + (long)sys * ctx->hist_cap, sizeof(double) * cnt,
                               cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return PNM_OK;
  });
}

int pnm_amplitude_labels(const pnm_ctx* ctx, int sys, size_t* n, int32_t* abij) {
  return guarded([&]() {
    check_sys(ctx, sys);
    const SysInfo& S = ctx->sys[sys];
    if (n) *n = (size_t)(S.t_end - S.t_begin);
    if (abij) {
      int c0 = S.ch_begin, c1 = S.ch_end;
      if (c1 == c0) return PNM_OK;
      int nh = ctx->h_hh_off[c1 - 1] + ctx->h_nhh[c1 - 1] - ctx->h_hh_off[c0];
      int np = ctx->h_pp_off[c1 - 1] + ctx->h_npp[c1 - 1] - ctx->h_pp_off[c0];
      std::vector<int2> hh(nh), pp(np);
      CUDA_TRY(cudaMemcpyAsync(hh.data(), ctx->d.hh_pair + ctx->h_hh_off[c0], sizeof(int2) * nh,
                               cudaMemcpyDeviceToHost, ctx->stream));
      CUDA_TRY(cudaMemcpyAsync(pp.data(), ctx->d.pp_pair + ctx->h_pp_off[c0], sizeof(int2) * np,
                               cudaMemcpyDeviceToHost, ctx->stream));
      CUDA_TRY(cudaStreamSynchronize(ctx->stream));
      size_t z = 0;
      for (int c = c0; c < c1; c++) {
        int hb = ctx->h_hh_off[c] - ctx->h_hh_off[c0], pb = ctx->h_pp_off[c] - ctx->h_pp_off[c0];
        for (int ij = 0; ij < ctx->h_nhh[c]; ij++)
          for (int ab = 0; ab < ctx->h_npp[c]; ab++, z++) {
            abij[4 * z + 0] = pp[pb + ab].x - S.sp_off;
            abij[4 * z + 1] = pp[pb + ab].y - S.sp_off;
            abij[4 * z + 2] = hh[hb + ij].x - S.sp_off;
            abij[4 * z + 3] = hh[hb + ij].y - S.sp_off;
          }
      }
    }
    return PNM_OK;
  });
}

int pnm_get_amplitudes(const pnm_ctx* ctx, int sys, double* t, size_t n) {
  return guarded([&]() {
    check_sys(ctx, sys);
    const SysInfo& S = ctx->sys[sys];
    if (!t || n != (size_t)(S.t_end - S.t_begin)) throw PnmError{PNM_EINVAL, "size mismatch"};
    CUDA_TRY(cudaMemcpyAsync(t, ctx->d.t0 + S.t_begin, sizeof(double) * n, cudaMemcpyDeviceToHost,
                             ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return PNM_OK;
  });
}

int pnm_set_amplitudes(pnm_ctx* ctx, int sys, const double* t, size_t n) {
  return guarded([&]() {
    check_sys(ctx, sys);
    const SysInfo& S = ctx->sys[sys];
    if (!t || n != (size_t)(S.t_end - S.t_begin)) throw PnmError{PNM_EINVAL, "size mismatch"};
    CUDA_TRY(cudaMemcpyAsync(ctx->d.t0 + S.t_begin, t, sizeof(double) * n, cudaMemcpyHostToDevice,
                             ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return PNM_OK;
  });
}

// FNV-1a, 64 bit: offset basis 14695981039346656037, prime 1099511628211.
static uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; i++) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

static pnm_checkpoint_header header_of(const pnm_ctx* ctx, int sys) {
  const SysInfo& S = ctx->sys[sys];
  pnm_checkpoint_header h;
  std::memset(&h, 0, sizeof(h));
  h.N = S.N - S.Z;
  h.Z = S.Z;
  h.n2max = S.n2max;
  h.rho = S.rho;
  for (int a = 0; a < 3; a++) h.twist[a] = S.phi[a];
  h.n_amplitudes = S.t_end - S.t_begin;
  int nch = 0, npairs = 0;
  int rc = pnm_channels(ctx, sys, 0, &nch, &npairs, nullptr, nullptr, nullptr);
  if (rc != PNM_OK) throw PnmError{rc, "channel tables unavailable"};
  std::vector<int32_t> keys(std::max(nch, 1)), sizes(2 * std::max(nch, 1)), pairs(2 * std::max(npairs, 1));
  rc = pnm_channels(ctx, sys, 0, &nch, &npairs, keys.data(), sizes.data(), pairs.data());
  if (rc != PNM_OK) throw PnmError{rc, "channel tables unavailable"};
  uint64_t x = 14695981039346656037ull;
  for (int c = 0; c < nch; c++) {
    x = fnv1a(x, &keys[c], sizeof(int32_t));
    x = fnv1a(x, &sizes[2 * c], 2 * sizeof(int32_t));
  }
  x = fnv1a(x, pairs.data(), sizeof(int32_t) * 2 * (size_t)npairs);
  h.channel_hash = x;
  return h;
}

int pnm_checkpoint_header_of(const pnm_ctx* ctx, int sys, pnm_checkpoint_header* h) {
  return guarded([&]() {
    check_sys(ctx, sys);
    if (!h) throw PnmError{PNM_EINVAL, "null argument"};
    *h = header_of(ctx, sys);
    return PNM_OK;
  });
}

static const char kCkptMagic[8] = {'P', 'N', 'M', 'C', 'K', 'P', 'T', '1'};

int pnm_checkpoint_save(const pnm_ctx* ctx, const char* path) {
  return guarded([&]() {
    if (!ctx || !path) throw PnmError{PNM_EINVAL, "null argument"};
    const int nsys = (int)ctx->sys.size();
    std::vector<pnm_checkpoint_header> hs(nsys);
    for (int k = 0; k < nsys; k++) hs[k] = header_of(ctx, k);
    std::vector<double> t((size_t)std::max<long>(ctx->nt, 1));
    CUDA_TRY(cudaMemcpyAsync(t.data(), ctx->d.t0, sizeof(double) * ctx->nt, cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    FILE* f = std::fopen(path, "wb");
    if (!f) throw PnmError{PNM_EINVAL, std::string("cannot open ") + path + " for writing"};
    const int32_t head[2] = {nsys, 0};
    bool ok = std::fwrite(kCkptMagic, 1, 8, f) == 8 && std::fwrite(head, sizeof(int32_t), 2, f) == 2 &&
              std::fwrite(hs.data(), sizeof(pnm_checkpoint_header), nsys, f) == (size_t)nsys;
    for (int k = 0; k < nsys && ok; k++) {
      const SysInfo& S = ctx->sys[k];
      const size_t n = (size_t)(S.t_end - S.t_begin);
      ok = std::fwrite(t.data() + S.t_begin, sizeof(double), n, f) == n;
    }
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) throw PnmError{PNM_EINVAL, std::string("writing ") + path + " failed"};
    return PNM_OK;
  });
}

int pnm_checkpoint_load(pnm_ctx* ctx, const char* path) {
  return guarded([&]() {
    if (!ctx || !path) throw PnmError{PNM_EINVAL, "null argument"};
    const int nsys = (int)ctx->sys.size();
    FILE* f = std::fopen(path, "rb");
    if (!f) throw PnmError{PNM_EINVAL, std::string("cannot open ") + path};
    struct Closer {
      FILE* f;
      ~Closer() { std::fclose(f); }
    } closer{f};
    char magic[8];
    int32_t head[2];
    if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, kCkptMagic, 8) != 0)
      throw PnmError{PNM_EINVAL, "not a checkpoint file"};
    if (std::fread(head, sizeof(int32_t), 2, f) != 2) throw PnmError{PNM_EINVAL, "truncated checkpoint"};
    if (head[0] != nsys) throw PnmError{PNM_EINVAL, "checkpoint holds another number of systems"};
    std::vector<pnm_checkpoint_header> hs(nsys);
    if (std::fread(hs.data(), sizeof(pnm_checkpoint_header), nsys, f) != (size_t)nsys)
      throw PnmError{PNM_EINVAL, "truncated checkpoint"};
    for (int k = 0; k < nsys; k++) {
      const pnm_checkpoint_header own = header_of(ctx, k);
      if (std::memcmp(&own, &hs[k], sizeof(own)) != 0)
        throw PnmError{PNM_EINVAL, "checkpoint header of system " + std::to_string(k) +
                                       " does not match the context (N, Z, n2max, rho, twist or channel tables)"};
    }
    std::vector<double> t((size_t)std::max<long>(ctx->nt, 1));
    for (int k = 0; k < nsys; k++) {
      const SysInfo& S = ctx->sys[k];
      const size_t n = (size_t)(S.t_end - S.t_begin);
      if (std::fread(t.data() + S.t_begin, sizeof(double), n, f) != n) throw PnmError{PNM_EINVAL, "truncated checkpoint"};
    }
    CUDA_TRY(cudaMemcpyAsync(ctx->d.t0, t.data(), sizeof(double) * ctx->nt, cudaMemcpyHostToDevice, ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return PNM_OK;
  });
}

int pnm_get_timings(const pnm_ctx* ctx, double* ms, int n) {
  return guarded([&]() {
    if (!ctx || !ms) throw PnmError{PNM_EINVAL, "null argument"};
    double v[7] = {ctx->t_setup, ctx->t_mbpt2, ctx->t_solve, ctx->t_mixed, ctx->t_refine,
                   (double)ctx->mlp_fallback, ctx->t_prepare};
    for (int k = 0; k < n && k < 7; k++) ms[k] = v[k];
    return PNM_OK;
  });
}

int pnm_v_element(const pnm_ctx* ctx, int sys, int p, int q, int r, int s, double* out);

int pnm_apply_pp_ladder(pnm_ctx* ctx, int sys, int precision, const double* t, double* r, size_t n) {
  return guarded([&]() {
    check_sys(ctx, sys);
    if (!t || !r) throw PnmError{PNM_EINVAL, "null argument"};
    if (precision != PNM_PREC_FP64 && precision != PNM_PREC_BF16X3 && precision != PNM_PREC_F32PAIR)
      throw PnmError{PNM_EINVAL, "unknown precision mode"};
    pnm_apply_pp(ctx, sys, precision, t, r, n);
    return PNM_OK;
  });
}

int pnm_apply_ph_term(pnm_ctx* ctx, int sys, int precision, const double* t, double* r, size_t n) {
  return guarded([&]() {
    check_sys(ctx, sys);
    if (!t || !r) throw PnmError{PNM_EINVAL, "null argument"};
    if (precision != PNM_PREC_FP64 && precision != PNM_PREC_BF16X3 && precision != PNM_PREC_F32PAIR)
      throw PnmError{PNM_EINVAL, "unknown precision mode"};
    pnm_apply_ph(ctx, sys, precision, t, r, n);
    return PNM_OK;
  });
}

int pnm_get_tuning(const pnm_ctx* ctx, int* ksplit, int* stages, float* us, int* serial_mask) {
  return guarded([&]() {
    if (!ctx) throw PnmError{PNM_EINVAL, "null context"};
    pnm_mixed_tuning(ctx, ksplit, stages, us, serial_mask);
    return PNM_OK;
  });
}

int pnm_selftest_timeout(pnm_ctx* ctx) {
  return guarded([&]() {
    if (!ctx) throw PnmError{PNM_EINVAL, "null context"};
    pnm_selftest_wait(ctx);
    return PNM_OK;
  });
}

int pnm_set_profiling(pnm_ctx* ctx, int on) {
  return guarded([&]() {
    if (!ctx) throw PnmError{PNM_EINVAL, "null context"};
    ctx->prof_on = on != 0;
    for (int k = 0; k < PNM_NKERNELS; k++) {
      ctx->prof_ms[k] = 0.0;
      ctx->prof_n[k] = 0;
    }
    return PNM_OK;
  });
}

int pnm_kernel_stats(const pnm_ctx* ctx, int id, const char** name, double* total_ms, int* launches) {
  return guarded([&]() {
    if (!ctx) throw PnmError{PNM_EINVAL, "null context"};
    if (id < 0 || id >= PNM_NKERNELS) throw PnmError{PNM_EINVAL, "kernel id out of range"};
    if (name) *name = pnm_kernel_names[id];
    if (total_ms) *total_ms = ctx->prof_ms[id];
    if (launches) *launches = ctx->prof_n[id];
    return PNM_OK;
  });
}

}  // extern "C"
