// mlp.cu -- learned warm start for the CCD iteration (not in the paper; it starts the
// Jacobi iteration of Eq. ccd3 from a prediction instead of the MBPT2 guess of Eq. ccdGuess).
//
// Network: 32 features -> 128 -> 128 -> 128 (GELU) -> 1, weights and layer inputs in BF16,
// FP32 accumulation.  Prediction per restricted amplitude:
//   t_start = t_MBPT2 + sigma_sys * y_scale * net(features),
// with sigma_sys the RMS of the system's MBPT2 amplitudes.  Features are dimensionless:
// momenta in units of k_F, spins, eps_ij^ab / eps_F, N <ab|v|ij> / eps_F, t_MBPT2 / sigma_sys,
// rho, k_F, N.  Training (SIMT kernels, Adam) uses amplitudes the solver itself converged;
// inference is one fused tcgen05 kernel: the four layers of a 128-sample tile run back to
// back with the weights resident in shared memory and the accumulator in tensor memory.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>

#include "pnm_context.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int MF = 32, MH = 128, MHEADER = 2 * MF + 4;
constexpr int O_MU = 0, O_IS = MF, O_YS = 2 * MF;
constexpr int O_W1 = MHEADER, O_B1 = O_W1 + MH * MF, O_W2 = O_B1 + MH, O_B2 = O_W2 + MH * MH;
constexpr int O_W3 = O_B2 + MH, O_B3 = O_W3 + MH * MH, O_W4 = O_B3 + MH, O_B4 = O_W4 + MH;
constexpr int NPARAM = O_B4 + 1;
constexpr int NFEAT = 22;  // real features; columns NFEAT..MF-1 are zero

// GELU in its tanh form, gelu(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))) (Hendrycks and
// Gimpel), and its derivative; training uses the accurate tanhf.
constexpr float GELU_C0 = 0.7978845608028654f, GELU_C1 = 0.7978845608028654f * 0.044715f;
__device__ __forceinline__ float gelu_f(float z) {
  float th = tanhf(z * fmaf(GELU_C1, z * z, GELU_C0));
  return 0.5f * z * (1.0f + th);
}
__device__ __forceinline__ float gelu_prime_f(float z) {
  float th = tanhf(z * fmaf(GELU_C1, z * z, GELU_C0));
  return 0.5f * (1.0f + th) + 0.5f * z * (1.0f - th * th) * fmaf(3.0f * GELU_C1, z * z, GELU_C0);
}
// Inference: the same function with the hardware tanh approximation (relative error about
// 2^-11, below the BF16 rounding of the activations that follows).
__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float gelu_fast(float z) {
  float hz = 0.5f * z;
  return fmaf(hz, tanh_fast(z * fmaf(GELU_C1, z * z, GELU_C0)), hz);
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ------------------------------------------------------------------------ features
struct FeatSys {
  double kscale;  // (2 pi / L) / k_F
  double epsF;    // hbar^2 k_F^2 / 2m
  double rho, kF;
  int N;
  double inv_epsF, v_scale;   // 1 / epsF and N / epsF
  float f19, f20, f21;        // rho / 0.16, k_F, N / 66
};

// t_MBPT2 per amplitude (stored when tm2 is given) and partial sums of its square (one per
// update item).
__global__ void k_tm2(DevState D, const int4* __restrict__ items, double* __restrict__ tm2,
                      double* __restrict__ parts) {
  __shared__ double sh32[32];
  int4 it = items[blockIdx.x];
  int c = it.x, ij = it.y;
  int npp = D.ch_npp[c];
  int ab = it.z + threadIdx.x;
  double s = 0.0;
  if (ab < npp && threadIdx.x < 128) {
    long z = D.ch_t_off[c] + (long)ij * npp + ab;
    double t = D.v_pphh[z] * D.inv_den[z];  // the MBPT2 amplitude v / eps_ij^ab
    if (tm2) tm2[z] = t;
    s = t * t;
  }
  s = block_sum(s, sh32);
  if (threadIdx.x == 0) parts[blockIdx.x] = s;
}

__global__ void k_sigma(const double* __restrict__ parts, const int* __restrict__ lo,
                        const int* __restrict__ hi, const long* __restrict__ count,
                        double* __restrict__ sigma) {
  __shared__ double sh32[32];
  int s = blockIdx.x;
  double acc = 0.0;
  for (int k = lo[s] + threadIdx.x; k < hi[s]; k += blockDim.x) acc += parts[k];
  acc = block_sum(acc, sh32);
  if (threadIdx.x == 0) {
    sigma[s] = sqrt(acc / (double)max(1L, count[s]));
    sigma[gridDim.x + s] = 1.0 / sigma[s];
  }
}

// Features [16 h, 16 h + 16) of the restricted amplitude z = (channel c, hole pair ij, particle
// pair ab): h = 0 the momenta of a, b, i, j in units of k_F and their spins; h = 1
// eps_ij^ab / eps_F, N <ab|v|ij> / eps_F, t_MBPT2 / sigma_sys (t_MBPT2 = v / eps, the product
// k_tm2 forms), rho / 0.16, k_F, N / 66, zeros.  FP64 only where the inputs are FP64: three
// products (reciprocals prepared per system) and their conversions.
__device__ __forceinline__ void feature_half(const DevState& D, const FeatSys& f, double inv_sigma, int c,
                                             int ij, int ab, long z, int h, float (&x)[16]) {
  if (h == 0) {
    const int2 hp = D.hh_pair[D.ch_hh_off[c] + ij];
    const int2 pp = D.pp_pair[D.ch_pp_off[c] + ab];
    const char4 sa = D.nvec[pp.x], sb = D.nvec[pp.y], si = D.nvec[hp.x], sj = D.nvec[hp.y];
    const float k = (float)f.kscale;
    x[0] = k * sa.x; x[1] = k * sa.y; x[2] = k * sa.z;
    x[3] = k * sb.x; x[4] = k * sb.y; x[5] = k * sb.z;
    x[6] = k * si.x; x[7] = k * si.y; x[8] = k * si.z;
    x[9] = k * sj.x; x[10] = k * sj.y; x[11] = k * sj.z;
    x[12] = sa.w; x[13] = sb.w; x[14] = si.w; x[15] = sj.w;
  } else {
    const double v = D.v_pphh[z];
    const double tm2 = v * D.inv_den[z];
    x[0] = (float)(D.den[z] * f.inv_epsF);
    x[1] = (float)(v * f.v_scale);
    x[2] = (float)(tm2 * inv_sigma);
    x[3] = f.f19;
    x[4] = f.f20;
    x[5] = f.f21;
#pragma unroll
    for (int q = 6; q < 16; q++) x[q] = 0.0f;
  }
}

__global__ void k_features(DevState D, const int4* __restrict__ items, const FeatSys* __restrict__ fs,
                           const double* __restrict__ inv_sigma, float* __restrict__ X) {
  int4 it = items[blockIdx.x];
  int c = it.x, ij = it.y;
  int npp = D.ch_npp[c];
  int ab = it.z + threadIdx.x;
  if (ab >= npp || threadIdx.x >= 128) return;
  int sys = D.ch_sys[c];
  long z = D.ch_t_off[c] + (long)ij * npp + ab;
  float* x = X + z * MF;
  for (int h = 0; h < 2; h++) {
    float xh[16];
    feature_half(D, fs[sys], inv_sigma[sys], c, ij, ab, z, h, xh);
#pragma unroll
    for (int q = 0; q < 16; q++) x[16 * h + q] = xh[q];
  }
}

// The learned start's sample list: rep[off + k] = (z, c) for the amplitudes z = t_off[c] +
// ij npp + ab0 + k of the row chunks items (c, ij, ab0, off) (up to 128 columns each).
__global__ void k_rep_fill(DevState D, const int4* __restrict__ items, int2* __restrict__ rep) {
  const int4 it = items[blockIdx.x];
  const int npp = D.ch_npp[it.x];
  const int ab = it.z + threadIdx.x;
  if (ab >= npp || threadIdx.x >= 128) return;
  rep[it.w + threadIdx.x] = make_int2((int)(D.ch_t_off[it.x] + (long)it.y * npp + ab), it.x);
}

// Training targets y = (t - t_MBPT2) / sigma_sys from the held amplitudes t0.
__global__ void k_targets(DevState D, const int4* __restrict__ items, const double* __restrict__ tm2,
                          const double* __restrict__ sigma, float* __restrict__ T) {
  int4 it = items[blockIdx.x];
  int c = it.x, ij = it.y;
  int npp = D.ch_npp[c];
  int ab = it.z + threadIdx.x;
  if (ab >= npp || threadIdx.x >= 128) return;
  long z = D.ch_t_off[c] + (long)ij * npp + ab;
  T[z] = (float)((D.t0[z] - tm2[z]) / sigma[D.ch_sys[c]]);
}

// ------------------------------------------------------------------- SIMT training
// C[M][N] (+)= op(A)[M][K] op(B)[K][N], row-major; op(A)(m,k) = tA ? A[k lda + m] : A[m lda + k].
__global__ void __launch_bounds__(256) k_sgemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                               int tA, const float* __restrict__ B, int ldb, int tB,
                                               float* __restrict__ C, int ldc, int acc) {
  __shared__ float As[16][68], Bs[16][68];
  int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float c[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      int kk = e >> 6, mm = e & 63;
      int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < K) ? (tA ? A[(long)k * lda + m] : A[(long)m * lda + k]) : 0.0f;
      int n = n0 + mm;
      Bs[kk][mm] = (n < N && k < K) ? (tB ? B[(long)n * ldb + k] : B[(long)k * ldb + n]) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; kk++) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; i++) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) c[i][j] = fmaf(a[i], b[j], c[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
      if (m < M && n < N) C[(long)m * ldc + n] = (acc ? C[(long)m * ldc + n] : 0.0f) + c[i][j];
    }
}

void sgemm(cudaStream_t s, int M, int N, int K, const float* A, int lda, int tA, const float* B, int ldb,
           int tB, float* C, int ldc, int acc) {
  dim3 g((N + 63) / 64, (M + 63) / 64);
  k_sgemm<<<g, 256, 0, s>>>(M, N, K, A, lda, tA, B, ldb, tB, C, ldc, acc);
}

// ------------------------------------------------------------ tensor-core training GEMM
// The k_sgemm contract, C[M][N] (+)= op(A)[M][K] op(B)[K][N], on the tcgen05 tensor cores for the
// BF16 training mode: each operand element is split as it is staged into BF16 hi + lo (exact for
// the BF16-rounded weights and layer inputs, whose lo part is zero; 2^-18 relative for the FP32
// error signals of the backward pass), three products per 16-wide k step (hi hi + hi lo +
// lo hi) accumulate in FP32 in tensor memory.  One CTA (four warps) per 128 x bn tile of C and
// k-range blockIdx.z (K split into gridDim.z ranges of whole 64-wide stages, results to
// C + blockIdx.z * cz, summed in order by k_sum_splits); all threads stage a 64-wide k slice of
// both operands into shared memory in the K-major core-matrix layout, thread 0 issues the MMAs
// and commits them to an mbarrier (bounded wait: on timeout the CTA stops, writes nothing and
// sets *err), and each thread drains its TMEM lane (row of C).
constexpr int TG_BM = 128, TG_BN = 128, TG_BK = 64;
constexpr int TG_PLANE_A = TG_BM * TG_BK, TG_PLANE_B = TG_BN * TG_BK;  // BF16 elements per plane
constexpr size_t TG_SMEM = 1024 + 2 * (size_t)(TG_PLANE_A + TG_PLANE_B) * sizeof(__nv_bfloat16);
constexpr int TG_MAX_SPLIT = 16, TG_BATCH = 16;

__device__ __forceinline__ void tg_split(float x, __nv_bfloat16* hi, __nv_bfloat16* lo, int o) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  hi[o] = h;
  lo[o] = __float2bfloat16_rn(x - __bfloat162float(h));
}

__global__ void __launch_bounds__(128) k_gemm_tc(int M, int N, int K, const float* __restrict__ A, int lda, int tA,
                                                 const float* __restrict__ B, int ldb, int tB,
                                                 float* __restrict__ C, int ldc, long cz, int acc, int bn,
                                                 int* __restrict__ err_flag) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 8);
  __nv_bfloat16* Ah = reinterpret_cast<__nv_bfloat16*>(smem + 1024);
  __nv_bfloat16* Al = Ah + TG_PLANE_A;
  __nv_bfloat16* Bh = Al + TG_PLANE_A;
  __nv_bfloat16* Bl = Bh + TG_PLANE_B;
  __shared__ int bad;
  const int m0 = blockIdx.y * TG_BM, n0 = blockIdx.x * bn;  // bn: 32, 64 or TG_BN columns per CTA
  const int nt = min(bn, N - n0);
  const int np = (nt + 15) & ~15;  // the MMA's N: a multiple of 16
  // this CTA's k-range: whole stages
  const int nstage = (K + TG_BK - 1) / TG_BK;
  const int per = (nstage + gridDim.z - 1) / gridDim.z;
  const int kb = blockIdx.z * per * TG_BK, ke = min(K, (int)(blockIdx.z + 1) * per * TG_BK);
  float* __restrict__ Cz = C + blockIdx.z * cz;
  if (threadIdx.x == 0) {
    bad = 0;
    tc::mbar_init(bar, 1);
    tc::mbar_fence_init();
  }
  if (threadIdx.x < 32) {
    tc::tmem_alloc(tslot, 128);
    tc::tmem_relinquish();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t idesc = tc::idesc_bf16(TG_BM, np);
  const uint32_t sbo = (TG_BK / 8) * 128;
  uint32_t phase = 0, fail_parity = 0;
  bool issued = false;
  for (int k0 = kb; k0 < ke; k0 += TG_BK) {
    __syncthreads();
    const int stop = bad;
    __syncthreads();
    if (stop) break;
    // coalesced along each operand's contiguous index; TG_BATCH independent loads in flight
    // per thread before their splits are stored
    for (int e0 = 0; e0 < TG_BM * TG_BK; e0 += TG_BATCH * 128) {
      float x[TG_BATCH];
#pragma unroll
      for (int j = 0; j < TG_BATCH; j++) {
        const int e = e0 + j * 128 + threadIdx.x;
        const int r = tA ? e % TG_BM : e / TG_BK, k = tA ? e / TG_BM : e % TG_BK;
        const int m = m0 + r, kk = k0 + k;
        x[j] = (m < M && kk < ke) ? (tA ? A[(long)kk * lda + m] : A[(long)m * lda + kk]) : 0.0f;
      }
#pragma unroll
      for (int j = 0; j < TG_BATCH; j++) {
        const int e = e0 + j * 128 + threadIdx.x;
        const int r = tA ? e % TG_BM : e / TG_BK, k = tA ? e / TG_BM : e % TG_BK;
        tg_split(x[j], Ah, Al, tc::core_off(r, k, TG_BK / 8));
      }
    }
    for (int e0 = 0; e0 < np * TG_BK; e0 += TG_BATCH * 128) {
      float x[TG_BATCH];
#pragma unroll
      for (int j = 0; j < TG_BATCH; j++) {
        const int e = e0 + j * 128 + threadIdx.x;
        const int r = tB ? e / TG_BK : e % np, k = tB ? e % TG_BK : e / np;
        const int kk = k0 + k;
        x[j] = (e < np * TG_BK && r < nt && kk < ke)
                   ? (tB ? B[(long)(n0 + r) * ldb + kk] : B[(long)kk * ldb + n0 + r])
                   : 0.0f;
      }
#pragma unroll
      for (int j = 0; j < TG_BATCH; j++) {
        const int e = e0 + j * 128 + threadIdx.x;
        if (e < np * TG_BK) {
          const int r = tB ? e / TG_BK : e % np, k = tB ? e % TG_BK : e / np;
          tg_split(x[j], Bh, Bl, tc::core_off(r, k, TG_BK / 8));
        }
      }
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (threadIdx.x == 0) {
      for (int ks = 0; ks < TG_BK / 16; ks++) {
        const uint64_t ah = tc::smem_desc(reinterpret_cast<const unsigned char*>(Ah) + ks * 256, 128, sbo);
        const uint64_t al = tc::smem_desc(reinterpret_cast<const unsigned char*>(Al) + ks * 256, 128, sbo);
        const uint64_t bh = tc::smem_desc(reinterpret_cast<const unsigned char*>(Bh) + ks * 256, 128, sbo);
        const uint64_t bl = tc::smem_desc(reinterpret_cast<const unsigned char*>(Bl) + ks * 256, 128, sbo);
        tc::mma_bf16(tbase, ah, bh, idesc, (issued || ks > 0) ? 1u : 0u);
        tc::mma_bf16(tbase, ah, bl, idesc, 1u);
        tc::mma_bf16(tbase, al, bh, idesc, 1u);
      }
      tc::commit(bar);
    }
    issued = true;
    __syncwarp();
    // every thread waits: the next stage overwrites the operands the MMAs read
    if (!tc::mbar_wait(bar, phase & 1)) {
      bad = 1;
      fail_parity = phase & 1;
    }
    phase++;
    tc::fence_after();
  }
  __syncthreads();
  const int ok = !bad;
  // after a wait that ran out, give the MMAs still in flight one more bounded wait before the
  // tensor memory they write is freed
  if (!ok && threadIdx.x == 0) tc::mbar_wait(bar, fail_parity);
  // epilogue through shared memory (the operand planes are free once the last wait passed), 64
  // columns at a time: thread = TMEM lane = row of the tile into Cs, then rows of C written with
  // consecutive threads on consecutive columns (an empty k-range leaves zeros)
  constexpr int CS_LD = 65;
  float* Cs = reinterpret_cast<float*>(smem + 1024);  // 128 x CS_LD floats
  const int r = threadIdx.x;
  const uint32_t lane_addr = tbase + ((uint32_t)((threadIdx.x >> 5) * 32) << 16);
  for (int c0 = 0; c0 < np; c0 += 64) {
    const int cw = min(64, np - c0);
    __syncthreads();
    if (ok) {
      for (int cc = 0; cc < cw; cc += 16) {
        uint32_t v[16];
        tc::tmem_ld16(lane_addr + c0 + cc, v);
#pragma unroll
        for (int j = 0; j < 16; j++) Cs[r * CS_LD + cc + j] = issued ? __uint_as_float(v[j]) : 0.0f;
      }
    }
    __syncthreads();
    if (ok) {
      for (int e = threadIdx.x; e < TG_BM * cw; e += blockDim.x) {
        const int rr = e / cw, c = e % cw;
        const int m = m0 + rr, n = c0 + c;
        if (m < M && n < nt) {
          float* dst = Cz + (long)m * ldc + n0 + n;
          const float y = Cs[rr * CS_LD + c];
          *dst = acc ? *dst + y : y;
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (threadIdx.x < 32) tc::tmem_dealloc(tbase, 128);
  if (threadIdx.x == 0 && !ok) atomicExch(err_flag, 1);
}

// C (+)= sum over z of W[z] (M x N, row stride N), in the order z = 0, 1, ...
__global__ void k_sum_splits(const float* __restrict__ W, int nz, int M, int N, float* __restrict__ C, int ldc,
                             int acc) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)M * N) return;
  const int m = (int)(e / N), n = (int)(e % N);
  float s = acc ? C[(long)m * ldc + n] : 0.0f;
  for (int z = 0; z < nz; z++) s += W[(long)z * M * N + e];
  C[(long)m * ldc + n] = s;
}

// h0 = bf16((x - mu) * inv_std) for the rows idx[0..B) of X (rnd = 0: FP32 debug mode, no
// BF16 rounding).
__global__ void k_prep(const float* __restrict__ X, const int* __restrict__ idx, int B,
                       const float* __restrict__ blob, float* __restrict__ H0, int rnd) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * MF) return;
  int r = e / MF, q = e % MF;
  long row = idx ? idx[r] : r;
  float x = (X[row * MF + q] - blob[O_MU + q]) * blob[O_IS + q];
  H0[e] = rnd ? bf16r(x) : x;
}

// z = acc + b; keep z; h = bf16(gelu(z)) (rnd = 0: FP32 debug mode, h = gelu(z)).
__global__ void k_bias_gelu(float* __restrict__ Z, const float* __restrict__ b, float* __restrict__ Hn, int B,
                            int rnd) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * MH) return;
  float z = Z[e] + b[e % MH];
  Z[e] = z;
  float h = gelu_f(z);
  Hn[e] = rnd ? bf16r(h) : h;
}

// y = h3 . w4 + b4, residual, loss partial and dy = 2 (y - t) / B.  One warp per row.
__global__ void k_out(const float* __restrict__ H3, const float* __restrict__ w4q, const float* __restrict__ b4,
                      const float* __restrict__ T, const int* __restrict__ idx, int B, float* __restrict__ Y,
                      float* __restrict__ dY, double* __restrict__ loss_acc) {
  int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (r >= B) return;
  float s = 0.0f;
  for (int q = lane; q < MH; q += 32) s += H3[(long)r * MH + q] * w4q[q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    float y = s + b4[0];
    if (Y) Y[r] = y;
    if (T) {
      float t = T[idx ? idx[r] : r];
      float d = y - t;
      dY[r] = 2.0f * d / (float)B;
      atomicAdd(loss_acc, (double)d * d);
    }
  }
}

__global__ void k_dz(const float* __restrict__ dH, const float* __restrict__ Z, float* __restrict__ dZ, int n) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) dZ[e] = dH[e] * gelu_prime_f(Z[e]);
}

// Column sums of a (B x ncol) matrix into g (fixed order per column).
// g[col] = sum_r w[r] A[r][col] (w == nullptr: w = 1), one block per column.
__global__ void k_colsum(const float* __restrict__ A, int B, int ncol, float* __restrict__ g,
                         const float* __restrict__ w = nullptr) {
  __shared__ float sh[256];
  int col = blockIdx.x;
  float s = 0.0f;
  if (w)
    for (int r = threadIdx.x; r < B; r += blockDim.x) s = fmaf(w[r], A[(long)r * ncol + col], s);
  else
    for (int r = threadIdx.x; r < B; r += blockDim.x) s += A[(long)r * ncol + col];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) g[col] = sh[0];
}

// Adam on the parameters (header entries are constants); q = BF16-rounded copy of weights.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float* __restrict__ q, float lr, float b1, float b2,
                       float c1, float c2, float eps) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < MHEADER || e >= NPARAM) return;
  float ge = g[e];
  float me = b1 * m[e] + (1.0f - b1) * ge;
  float ve = b2 * v[e] + (1.0f - b2) * ge * ge;
  m[e] = me;
  v[e] = ve;
  float we = w[e] - lr * (me / c1) / (sqrtf(ve / c2) + eps);
  w[e] = we;
  bool is_w = (e >= O_W1 && e < O_B1) || (e >= O_W2 && e < O_B2) || (e >= O_W3 && e < O_B3) ||
              (e >= O_W4 && e < O_B4);
  q[e] = is_w ? bf16r(we) : we;
}

// q = the parameters as the forward pass uses them: weights rounded to BF16 (rnd = 0: FP32
// debug mode, unrounded).
__global__ void k_quantize(const float* __restrict__ w, float* __restrict__ q, int rnd = 1) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NPARAM) return;
  bool is_w = (e >= O_W1 && e < O_B1) || (e >= O_W2 && e < O_B2) || (e >= O_W3 && e < O_B3) ||
              (e >= O_W4 && e < O_B4);
  q[e] = (is_w && rnd) ? bf16r(w[e]) : w[e];
}

// Per-column sums and squares of X (n x 32) for the feature normalisation.
__global__ void k_featstats(const float* __restrict__ X, long n, double* __restrict__ out) {
  __shared__ double s1[256], s2[256];
  int q = blockIdx.x;
  double a = 0.0, b = 0.0;
  for (long r = threadIdx.x; r < n; r += blockDim.x) {
    double x = X[r * MF + q];
    a += x;
    b += x * x;
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s1[threadIdx.x] += s1[threadIdx.x + w];
      s2[threadIdx.x] += s2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * q] = s1[0];
    out[2 * q + 1] = s2[0];
  }
}

__global__ void k_scale(float* __restrict__ T, long n, float s) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) T[e] *= s;
}

// ------------------------------------------------------------- tensor-core inference
// Packed BF16 weights in the K-major core-matrix layout: W1 (128 x 32), W2, W3 (128 x 128),
// W4 (16 x 128, rows 1..15 zero).
constexpr int PW1 = MH * MF, PW2 = MH * MH, PW4 = 16 * MH;
constexpr int PW_TOTAL = PW1 + 2 * PW2 + PW4;

__global__ void k_pack_weights(const float* __restrict__ q, __nv_bfloat16* __restrict__ pw) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < PW1) {
    int r = e / MF, k = e % MF;
    pw[tc::core_off(r, k, MF / 8)] = __float2bfloat16_rn(q[O_W1 + e]);
  } else if (e < PW1 + PW2) {
    int f = e - PW1, r = f / MH, k = f % MH;
    pw[PW1 + tc::core_off(r, k, MH / 8)] = __float2bfloat16_rn(q[O_W2 + f]);
  } else if (e < PW1 + 2 * PW2) {
    int f = e - PW1 - PW2, r = f / MH, k = f % MH;
    pw[PW1 + PW2 + tc::core_off(r, k, MH / 8)] = __float2bfloat16_rn(q[O_W3 + f]);
  } else if (e < PW_TOTAL) {
    int f = e - PW1 - 2 * PW2, r = f / MH, k = f % MH;
    float w = (r == 0) ? q[O_W4 + k] : 0.0f;
    pw[PW1 + 2 * PW2 + tc::core_off(r, k, MH / 8)] = __float2bfloat16_rn(w);
  }
}

constexpr int MLP_THREADS = 256;
constexpr int MLP_PAR = 3 * MH + 1 + 2 * MF;  // b1, b2, b3, b4, mu, inv_std
constexpr uint32_t MLP_SMEM = 1024 + PW_TOTAL * 2 + MH * MH * 2 + ((MLP_PAR * 4 + 1023) / 1024) * 1024;

// Where the inference writes: raw outputs Y, and/or the learned start amplitudes
// t0 = t_MBPT2 + sigma_sys * y_scale * y of every system (t_begin: first amplitude of each
// system, nsys + 1 entries).
struct MlpOut {
  float* Y;
  double* t0;
  const double* tm2;
  const double* sigma;
  const long* t_begin;
  int nsys;
  float y_scale;
  const int* idx;  // sample r is amplitude idx[r] (nullptr: amplitude r)
};

// Inputs of the learned start with the features formed in the kernel: sample r is amplitude
// rep[r].x of channel rep[r].y; its features come from D (feature_half), its t_MBPT2 is
// v / eps formed as k_tm2 forms it.
struct MlpFused {
  DevState D;
  const int2* rep;
  const FeatSys* fs;
  const double* inv_sigma;
};

// One CTA (8 warps) loops over 128-sample tiles; two CTAs share an SM, so one CTA's
// epilogue overlaps the other's MMAs.  Warp w reads TMEM lanes 32 (w % 4) ... + 31 (its
// row quarter) and columns 64 (w / 4) ... + 63 (its column half); thread (w, lane) owns
// sample row 32 (w % 4) + lane of the tile.
// FUSED: the samples' features are formed from the context (MlpFused) instead of read from X.
template <bool FUSED>
__global__ void __launch_bounds__(MLP_THREADS, 2) k_mlp_tc(const float* __restrict__ X, long n,
                                                           const float* __restrict__ q,
                                                           const __nv_bfloat16* __restrict__ pw, MlpOut out,
                                                           MlpFused fin, int* __restrict__ err_flag) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bar_w = reinterpret_cast<uint64_t*>(smem);
  uint64_t* bar_mma = bar_w + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar_w + 2);
  __nv_bfloat16* W = reinterpret_cast<__nv_bfloat16*>(smem + 1024);
  __nv_bfloat16* A = W + PW_TOTAL;
  float* par = reinterpret_cast<float*>(A + MH * MH);  // b1 b2 b3 | b4 | mu | inv_std
  const float* mu = par + 3 * MH + 1;
  const float* istd = mu + MF;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3, half = warp >> 2;
  const int row = quarter * 32 + lane;
  __shared__ int bad;
  if (threadIdx.x == 0) {
    bad = 0;
    tc::mbar_init(bar_w, 1);
    tc::mbar_init(bar_mma, 1);
    tc::mbar_fence_init();
  }
  if (warp == 2) {
    tc::tmem_alloc(tslot, MH);
    tc::tmem_relinquish();
  }
  for (int k = threadIdx.x; k < MH; k += blockDim.x) {
    par[k] = q[O_B1 + k];
    par[MH + k] = q[O_B2 + k];
    par[2 * MH + k] = q[O_B3 + k];
  }
  for (int k = threadIdx.x; k < MF; k += blockDim.x) {
    par[3 * MH + 1 + k] = q[O_MU + k];
    par[3 * MH + 1 + MF + k] = q[O_IS + k];
  }
  if (threadIdx.x == 0) par[3 * MH] = q[O_B4];
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;
  if (threadIdx.x == 0) {
    tc::mbar_expect_tx(bar_w, PW_TOTAL * 2);
    tc::bulk_g2s(W, pw, PW_TOTAL * 2, bar_w);
  }
  if (!tc::mbar_wait(bar_w, 0)) bad = 1;
  uint32_t phase = 0;
  const long ntiles = (n + MH - 1) / MH;
  const uint32_t lane_addr = tbase + ((uint32_t)(quarter * 32) << 16);
  // features [16 half, 16 half + 16) of this thread's row of a tile (zeros past n); the next
  // tile's are loaded while the current one runs through the layers
  const int k0 = 16 * half;
  auto load_x = [&](long tile, float4 (&xr)[4]) {
    long rg = tile * MH + row;
    if (tile < ntiles && rg < n) {
      if constexpr (FUSED) {
        const int2 zc = fin.rep[rg];
        const int npp = fin.D.ch_npp[zc.y];
        const int rel = (int)(zc.x - fin.D.ch_t_off[zc.y]);
        const int ij = rel / npp, ab = rel - ij * npp;
        const int sy = fin.D.ch_sys[zc.y];
        float xh[16];
        feature_half(fin.D, fin.fs[sy], fin.inv_sigma[sy], zc.y, ij, ab, zc.x, half, xh);
#pragma unroll
        for (int j = 0; j < 4; j++) xr[j] = make_float4(xh[4 * j], xh[4 * j + 1], xh[4 * j + 2], xh[4 * j + 3]);
      } else {
        const long zg = out.idx ? (long)out.idx[rg] : rg;
        const float4* xp = reinterpret_cast<const float4*>(X + zg * MF + k0);
#pragma unroll
        for (int j = 0; j < 4; j++) xr[j] = __ldg(xp + j);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 4; j++) xr[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
  };
  float4 xnext[4];
  load_x(blockIdx.x, xnext);
  for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // every thread leaves together after a failed wait (no thread may skip a barrier)
    __syncthreads();
    const int stop = bad;
    __syncthreads();
    if (stop) break;
    const long r_glob = tile * MH + row;
    const bool ok = r_glob < n;
    float xv[16];
#pragma unroll
    for (int j = 0; j < 4; j++) {
      xv[4 * j] = xnext[j].x; xv[4 * j + 1] = xnext[j].y; xv[4 * j + 2] = xnext[j].z; xv[4 * j + 3] = xnext[j].w;
    }
    load_x(tile + gridDim.x, xnext);
    // layer-1 input: normalised, BF16
    {
#pragma unroll
      for (int k = 0; k < 16; k++) xv[k] = ok ? (xv[k] - mu[k0 + k]) * istd[k0 + k] : 0.0f;
#pragma unroll
      for (int h = 0; h < 16; h += 8) {
        __align__(16) __nv_bfloat162 v4[4];
#pragma unroll
        for (int j = 0; j < 4; j++) v4[j] = __floats2bfloat162_rn(xv[h + 2 * j], xv[h + 2 * j + 1]);
        *reinterpret_cast<uint4*>(A + tc::core_off(row, k0 + h, MF / 8)) = *reinterpret_cast<uint4*>(v4);
      }
    }
    for (int layer = 0; layer < 4; layer++) {
      tc::fence_async_smem();
      tc::fence_before();
      __syncthreads();
      tc::fence_after();
      const int K = layer == 0 ? MF : MH;
      const int N = layer == 3 ? 16 : MH;
      if (threadIdx.x == 0) {
        const __nv_bfloat16* Wl = W + (layer == 0 ? 0 : layer == 1 ? PW1 : layer == 2 ? PW1 + PW2 : PW1 + 2 * PW2);
        const uint32_t sbo = (K / 8) * 128;
        const uint32_t idesc = tc::idesc_bf16(MH, N);
        for (int ks = 0; ks < K / 16; ks++) {
          uint64_t ad = tc::smem_desc(reinterpret_cast<const unsigned char*>(A) + ks * 256, 128, sbo);
          uint64_t bd = tc::smem_desc(reinterpret_cast<const unsigned char*>(Wl) + ks * 256, 128, sbo);
          tc::mma_bf16(tbase, ad, bd, idesc, ks > 0 ? 1u : 0u);
        }
        tc::commit(bar_mma);
      }
      __syncwarp();
      if (!tc::mbar_wait(bar_mma, phase & 1)) bad = 1;
      phase++;
      tc::fence_after();
      if (layer < 3) {
        // bias + GELU of this thread's 64 columns, BF16, into the next layer's A operand
        const float* b = par + layer * MH;
        const int cbase = 64 * half;
        uint32_t r[64];
        tc::tmem_ld16_nowait(lane_addr + cbase, *reinterpret_cast<uint32_t(*)[16]>(r));
        tc::tmem_ld16_nowait(lane_addr + cbase + 16, *reinterpret_cast<uint32_t(*)[16]>(r + 16));
        tc::tmem_ld16_nowait(lane_addr + cbase + 32, *reinterpret_cast<uint32_t(*)[16]>(r + 32));
        tc::tmem_ld16_nowait(lane_addr + cbase + 48, *reinterpret_cast<uint32_t(*)[16]>(r + 48));
        tc::tmem_wait_ld();
#pragma unroll
        for (int h = 0; h < 64; h += 8) {
          __align__(16) __nv_bfloat162 v4[4];
#pragma unroll
          for (int j = 0; j < 4; j++) {
            float z0 = __uint_as_float(r[h + 2 * j]) + b[cbase + h + 2 * j];
            float z1 = __uint_as_float(r[h + 2 * j + 1]) + b[cbase + h + 2 * j + 1];
            v4[j] = __floats2bfloat162_rn(gelu_fast(z0), gelu_fast(z1));
          }
          *reinterpret_cast<uint4*>(A + tc::core_off(row, cbase + h, MH / 8)) = *reinterpret_cast<uint4*>(v4);
        }
      } else if (half == 0) {
        uint32_t r[16];
        tc::tmem_ld16(lane_addr, r);
        if (ok) {
          float y = __uint_as_float(r[0]) + par[3 * MH];
          if (out.Y) out.Y[r_glob] = y;
          if (out.t0) {
            long z;
            int sy = 0;
            double t;
            if constexpr (FUSED) {
              const int2 zc = fin.rep[r_glob];
              z = zc.x;
              sy = fin.D.ch_sys[zc.y];
              t = fin.D.v_pphh[z] * fin.D.inv_den[z];
            } else {
              z = out.idx ? (long)out.idx[r_glob] : r_glob;
              while (sy + 1 < out.nsys && z >= out.t_begin[sy + 1]) sy++;
              t = out.tm2[z];
            }
            if (isfinite(y)) t += out.sigma[sy] * (double)out.y_scale * (double)y;
            out.t0[z] = t;
          }
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 2) tc::tmem_dealloc(tbase, MH);
  if (threadIdx.x == 0 && bad) atomicExch(err_flag, 1);
}

template <typename T>
T* xalloc(size_t n, std::vector<void*>& owned) {
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    throw PnmError{PNM_ENOMEM, "cudaMalloc (warm-start network) failed"};
  }
  owned.push_back(p);
  return (T*)p;
}

struct Scratch {
  std::vector<void*> owned;
  ~Scratch() {
    for (void* p : owned) cudaFree(p);
  }
};

// Training/inference buffers for a batch of B rows.
struct Net {
  float *w, *q, *g, *m, *v;  // parameters, BF16-rounded copy, gradient, Adam moments
  float *H0, *Z1, *H1, *Z2, *H2, *Z3, *H3, *Y, *dY, *dA, *dB;
  int B;
  // tc = 1: the matrix products on the tensor cores (k_gemm_tc; BF16 mode only); ws holds the
  // partial tiles of a k-split product, err the kernel's timeout flag
  int tc = 0;
  float* ws = nullptr;
  long ws_cap = 0;
  int* err = nullptr;
  void alloc(int b, Scratch& s, int use_tc = 0, cudaStream_t st = nullptr) {
    B = b;
    tc = use_tc;
    if (tc) {
      ws_cap = (long)TG_MAX_SPLIT * std::max(b, MH) * MH;
      ws = xalloc<float>(ws_cap, s.owned);
      err = xalloc<int>(1, s.owned);
      CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
      smem_at_least(k_gemm_tc, TG_SMEM);
    }
    w = xalloc<float>(NPARAM, s.owned);
    q = xalloc<float>(NPARAM, s.owned);
    g = xalloc<float>(NPARAM, s.owned);
    m = xalloc<float>(NPARAM, s.owned);
    v = xalloc<float>(NPARAM, s.owned);
    H0 = xalloc<float>((size_t)b * MF, s.owned);
    Z1 = xalloc<float>((size_t)b * MH, s.owned);
    H1 = xalloc<float>((size_t)b * MH, s.owned);
    Z2 = xalloc<float>((size_t)b * MH, s.owned);
    H2 = xalloc<float>((size_t)b * MH, s.owned);
    Z3 = xalloc<float>((size_t)b * MH, s.owned);
    H3 = xalloc<float>((size_t)b * MH, s.owned);
    Y = xalloc<float>(b, s.owned);
    dY = xalloc<float>(b, s.owned);
    dA = xalloc<float>((size_t)b * MH, s.owned);
    dB = xalloc<float>((size_t)b * MH, s.owned);
  }
};

// A matrix product of the training passes: on the tensor cores when nt.tc is set and both output
// dimensions are at least 16 (the output layer's vector products stay on k_sgemm), with the k
// range split over up to TG_MAX_SPLIT CTAs when the output has few tiles.
void gemm(cudaStream_t s, const Net& nt, int M, int N, int K, const float* A, int lda, int tA, const float* B,
          int ldb, int tB, float* C, int ldc, int acc) {
  if (!nt.tc || M < 16 || N < 16) {
    sgemm(s, M, N, K, A, lda, tA, B, ldb, tB, C, ldc, acc);
    return;
  }
  // about 64 CTAs: narrower column tiles first (the row tiles are fixed at 128), then the k split
  const int gy = (M + TG_BM - 1) / TG_BM;
  int bn = TG_BN;
  while (bn > 32 && ((N + bn - 1) / bn) * gy < 64) bn >>= 1;
  const int gx = (N + bn - 1) / bn;
  const int nstage = (K + TG_BK - 1) / TG_BK;
  int kz = 1;
  if (gx * gy < 64) kz = std::max(1, std::min(std::min(TG_MAX_SPLIT, nstage), 64 / (gx * gy)));
  while (kz > 1 && (long)kz * M * N > nt.ws_cap) kz--;
  if (kz == 1) {
    k_gemm_tc<<<dim3(gx, gy, 1), 128, TG_SMEM, s>>>(M, N, K, A, lda, tA, B, ldb, tB, C, ldc, 0, acc, bn, nt.err);
  } else {
    k_gemm_tc<<<dim3(gx, gy, kz), 128, TG_SMEM, s>>>(M, N, K, A, lda, tA, B, ldb, tB, nt.ws, N, (long)M * N, 0,
                                                     bn, nt.err);
    k_sum_splits<<<(unsigned)(((long)M * N + 255) / 256), 256, 0, s>>>(nt.ws, kz, M, N, C, ldc, acc);
  }
}

// rnd = 0: the FP32 debug mode (no BF16 rounding of the layer inputs).
void net_forward(cudaStream_t s, Net& nt, const float* X, const int* idx, int B, int rnd = 1) {
  k_prep<<<(B * MF + 255) / 256, 256, 0, s>>>(X, idx, B, nt.q, nt.H0, rnd);
  gemm(s, nt, B, MH, MF, nt.H0, MF, 0, nt.q + O_W1, MF, 1, nt.Z1, MH, 0);
  k_bias_gelu<<<(B * MH + 255) / 256, 256, 0, s>>>(nt.Z1, nt.q + O_B1, nt.H1, B, rnd);
  gemm(s, nt, B, MH, MH, nt.H1, MH, 0, nt.q + O_W2, MH, 1, nt.Z2, MH, 0);
  k_bias_gelu<<<(B * MH + 255) / 256, 256, 0, s>>>(nt.Z2, nt.q + O_B2, nt.H2, B, rnd);
  gemm(s, nt, B, MH, MH, nt.H2, MH, 0, nt.q + O_W3, MH, 1, nt.Z3, MH, 0);
  k_bias_gelu<<<(B * MH + 255) / 256, 256, 0, s>>>(nt.Z3, nt.q + O_B3, nt.H3, B, rnd);
}

// Backward pass from dY; writes the gradient blob nt.g (header entries zero).
void net_backward(cudaStream_t s, Net& nt, int B) {
  CUDA_TRY(cudaMemsetAsync(nt.g, 0, sizeof(float) * NPARAM, s));
  // output layer: dw4 = dY^T H3 (a weighted column sum), db4 = sum dY, dH3 = dY w4
  k_colsum<<<MH, 256, 0, s>>>(nt.H3, B, MH, nt.g + O_W4, nt.dY);
  k_colsum<<<1, 256, 0, s>>>(nt.dY, B, 1, nt.g + O_B4);
  gemm(s, nt, B, MH, 1, nt.dY, 1, 0, nt.q + O_W4, MH, 0, nt.dA, MH, 0);
  const float* Zs[3] = {nt.Z1, nt.Z2, nt.Z3};
  const float* Hin[3] = {nt.H0, nt.H1, nt.H2};
  const int Ow[3] = {O_W1, O_W2, O_W3}, Ob[3] = {O_B1, O_B2, O_B3}, Kin[3] = {MF, MH, MH};
  for (int l = 2; l >= 0; l--) {
    k_dz<<<(B * MH + 255) / 256, 256, 0, s>>>(nt.dA, Zs[l], nt.dB, B * MH);
    gemm(s, nt, MH, Kin[l], B, nt.dB, MH, 1, Hin[l], Kin[l], 0, nt.g + Ow[l], Kin[l], 0);
    k_colsum<<<MH, 256, 0, s>>>(nt.dB, B, MH, nt.g + Ob[l]);
    if (l > 0) gemm(s, nt, B, MH, MH, nt.dB, MH, 0, nt.q + Ow[l], MH, 0, nt.dA, MH, 0);
  }
}

unsigned long long g_seed_mix(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

}  // namespace

// ------------------------------------------------------------------- context glue
struct MlpState {
  float* X = nullptr;       // features of every amplitude (library order; training and pnm_mlp_features)
  double* tm2 = nullptr;    // MBPT2 amplitudes (idem)
  double* sigma = nullptr;  // per system, then 1 / sigma per system
  long* t_begin = nullptr;  // first amplitude of each system, then the total
  FeatSys* fs = nullptr;    // per-system feature constants
  float* q = nullptr;       // model parameters (BF16-rounded weights)
  __nv_bfloat16* pw = nullptr;
  int* err = nullptr;
  int2* rep = nullptr;      // (amplitude, channel) of the rows the updates compute (learned start)
  long n_rep = 0;
  float y_scale = 1.0f;
  bool have_model = false;
};

// Per-system constants of the features: sigma_sys (RMS of the MBPT2 amplitudes), k_F, eps_F,
// ... (once per context, stream-ordered, no host synchronisation).
static void mlp_systems(pnm_ctx* ctx) {
  if (!ctx->mlp) ctx->mlp = new MlpState();
  MlpState* M = ctx->mlp;
  if (M->sigma) return;
  cudaStream_t s = ctx->stream;
  int nsys = (int)ctx->sys.size();
  M->sigma = ctx_alloc<double>(ctx, 2 * nsys);
  std::vector<long> tb(nsys + 1);
  for (int k = 0; k < nsys; k++) tb[k] = ctx->sys[k].t_begin;
  tb[nsys] = ctx->nt;
  M->t_begin = ctx_alloc<long>(ctx, nsys + 1);
  CUDA_TRY(cudaMemcpyAsync(M->t_begin, tb.data(), sizeof(long) * (nsys + 1), cudaMemcpyHostToDevice, s));
  double* parts = ctx_alloc<double>(ctx, ctx->n_upd_items);
  std::vector<long> cnt(nsys);
  std::vector<FeatSys> fs(nsys);
  for (int k = 0; k < nsys; k++) {
    const SysInfo& S = ctx->sys[k];
    cnt[k] = S.t_end - S.t_begin;
    double kF = std::cbrt(3.0 * PNM_PI * PNM_PI * S.rho);
    fs[k].kF = kF;
    fs[k].rho = S.rho;
    fs[k].N = S.N;
    fs[k].kscale = (2.0 * PNM_PI / S.L) / kF;
    fs[k].epsF = ctx->hbar2_2m * kF * kF;
    fs[k].inv_epsF = 1.0 / fs[k].epsF;
    fs[k].v_scale = S.N / fs[k].epsF;
    fs[k].f19 = (float)(S.rho / 0.16);
    fs[k].f20 = (float)kF;
    fs[k].f21 = (float)(S.N / 66.0);
  }
  long* dcnt = ctx_alloc<long>(ctx, nsys);
  M->fs = ctx_alloc<FeatSys>(ctx, nsys);
  // pageable sources: each copy has left the host vector when cudaMemcpyAsync returns
  CUDA_TRY(cudaMemcpyAsync(dcnt, cnt.data(), sizeof(long) * nsys, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(M->fs, fs.data(), sizeof(FeatSys) * nsys, cudaMemcpyHostToDevice, s));
  k_tm2<<<ctx->n_upd_items, 128, 0, s>>>(ctx->d, ctx->upd_items, nullptr, parts);
  k_sigma<<<nsys, 256, 0, s>>>(parts, ctx->upd_lo_d, ctx->upd_hi_d, dcnt, M->sigma);
  CUDA_TRY(cudaGetLastError());
}

// The feature matrix X and t_MBPT2 of every amplitude, for training and pnm_mlp_features (the
// learned start forms its features in the inference kernel instead).
static void mlp_features(pnm_ctx* ctx) {
  mlp_systems(ctx);
  MlpState* M = ctx->mlp;
  if (M->X) return;
  cudaStream_t s = ctx->stream;
  int nsys = (int)ctx->sys.size();
  M->X = ctx_alloc<float>(ctx, (size_t)ctx->nt * MF);
  M->tm2 = ctx_alloc<double>(ctx, ctx->nt);
  double* parts = ctx_alloc<double>(ctx, ctx->n_upd_items);
  k_tm2<<<ctx->n_upd_items, 128, 0, s>>>(ctx->d, ctx->upd_items, M->tm2, parts);
  k_features<<<ctx->n_upd_items, 128, 0, s>>>(ctx->d, ctx->upd_items, M->fs, M->sigma + nsys, M->X);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(s));
}

static void mlp_tc_attributes() {
  smem_at_least(k_mlp_tc<false>, MLP_SMEM);
  smem_at_least(k_mlp_tc<true>, MLP_SMEM);
  CUDA_TRY(cudaFuncSetAttribute(k_mlp_tc<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  CUDA_TRY(cudaFuncSetAttribute(k_mlp_tc<true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
}

static void check_blob_header(const float* blob) {
  for (int k = 0; k < NPARAM; k++)
    if (!std::isfinite(blob[k])) throw PnmError{PNM_EINVAL, "non-finite parameter"};
}

static void set_model(pnm_ctx* ctx, const float* blob) {
  check_blob_header(blob);
  if (!ctx->mlp) ctx->mlp = new MlpState();
  MlpState* M = ctx->mlp;
  cudaStream_t s = ctx->stream;
  if (!M->q) {
    M->q = ctx_alloc<float>(ctx, NPARAM);
    M->pw = ctx_alloc<__nv_bfloat16>(ctx, PW_TOTAL);
    M->err = ctx_alloc<int>(ctx, 1);
    mlp_tc_attributes();
  }
  float* w = ctx_alloc<float>(ctx, NPARAM);
  CUDA_TRY(cudaMemcpyAsync(w, blob, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, s));
  k_quantize<<<(NPARAM + 255) / 256, 256, 0, s>>>(w, M->q);
  k_pack_weights<<<(PW_TOTAL + 255) / 256, 256, 0, s>>>(M->q, M->pw);
  CUDA_TRY(cudaMemsetAsync(M->err, 0, sizeof(int), s));
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(s));
  M->y_scale = blob[O_YS];
  M->have_model = true;
  pnm_drop_solve_graphs(ctx);  // the learned start's kernels hold y_scale as an argument
}

// One CTA pair per SM over the 128-sample tiles (fin.rep set: features formed in the kernel).
static void tc_infer(cudaStream_t s, const float* X, long n, const float* q, const __nv_bfloat16* pw,
                     const MlpOut& out, int* err, const MlpFused* fin = nullptr) {
  long ntiles = (n + MH - 1) / MH;
  int dev = 0, nsm = 148;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  int grid = (int)std::min<long>(ntiles, 2L * nsm);
  if (grid <= 0) return;
  if (fin) k_mlp_tc<true><<<grid, MLP_THREADS, MLP_SMEM, s>>>(X, n, q, pw, out, *fin, err);
  else k_mlp_tc<false><<<grid, MLP_THREADS, MLP_SMEM, s>>>(X, n, q, pw, out, MlpFused{}, err);
}

// One-time state of the learned start (per-system constants and the sample list).
void pnm_mlp_prepare(pnm_ctx* ctx) {
  if (!ctx->mlp || !ctx->mlp->have_model) throw PnmError{PNM_EINVAL, "no warm-start model set (pnm_mlp_set_model)"};
  mlp_systems(ctx);
  MlpState* M = ctx->mlp;
  cudaStream_t s = ctx->stream;
  if (!M->rep) {
    // the start is made flip-symmetric: the network is evaluated on the rows the updates
    // compute (about half the amplitudes) and the rest is copied from their spin flips.  The
    // sample list is filled on the device from row chunks (channel, ij, first column, offset).
    std::vector<int4> chunks;
    long off = 0;
    for (int r = 0; r < ctx->nrows; r++) {
      if (!ctx->h_row_mode[r]) continue;
      int2 row = ctx->h_rows[r];
      const int npp = ctx->h_npp[row.x];
      for (int ab0 = 0; ab0 < npp; ab0 += 128) {
        chunks.push_back(make_int4(row.x, row.y, ab0, (int)off));
        off += std::min(128, npp - ab0);
      }
    }
    if (ctx->nt > INT_MAX) throw PnmError{PNM_EINVAL, "too many amplitudes for the learned start"};
    M->n_rep = off;
    M->rep = ctx_alloc<int2>(ctx, std::max<long>(1, off));
    if (!chunks.empty()) {
      int4* dch = ctx_alloc<int4>(ctx, chunks.size());
      CUDA_TRY(cudaMemcpyAsync(dch, chunks.data(), sizeof(int4) * chunks.size(), cudaMemcpyHostToDevice, s));
      k_rep_fill<<<(unsigned)chunks.size(), 128, 0, s>>>(ctx->d, dch, M->rep);
      CUDA_TRY(cudaGetLastError());
    }
  }
}

// The learned start's kernels (after pnm_mlp_prepare): inference into t0, then the spin flips.
void pnm_mlp_enqueue(pnm_ctx* ctx) {
  MlpState* M = ctx->mlp;
  cudaStream_t s = ctx->stream;
  // the network output goes straight into t0 (t_MBPT2 + sigma_sys * y_scale * y)
  const int nsys = (int)ctx->sys.size();
  const MlpFused fin{ctx->d, M->rep, M->fs, M->sigma + nsys};
  tc_infer(s, nullptr, M->n_rep, M->q, M->pw,
           MlpOut{nullptr, ctx->d.t0, nullptr, M->sigma, M->t_begin, nsys, M->y_scale, nullptr}, M->err, &fin);
  pnm_flip_copy(ctx, ctx->d.t0, s);
  CUDA_TRY(cudaGetLastError());
}

// Learned start into t0 (every system), used by the solver for PNM_INIT_MLP.
void pnm_mlp_start(pnm_ctx* ctx) {
  pnm_mlp_prepare(ctx);
  pnm_mlp_enqueue(ctx);
}

// Device flag the inference kernel sets when one of its bounded waits ran out (nullptr without
// a model).
int* pnm_mlp_err(pnm_ctx* ctx) { return ctx->mlp ? ctx->mlp->err : nullptr; }

void pnm_free_mlp(pnm_ctx* ctx) {
  delete ctx->mlp;
  ctx->mlp = nullptr;
}

// -------------------------------------------------------------------------- C ABI
extern "C" {

int pnm_mlp_num_params(int* n) {
  if (!n) return PNM_EINVAL;
  *n = NPARAM;
  return PNM_OK;
}

int pnm_mlp_init(float* blob, unsigned long long seed) {
  if (!blob) return PNM_EINVAL;
  std::mt19937_64 rng(g_seed_mix(seed));
  std::normal_distribution<double> nd(0.0, 1.0);
  std::memset(blob, 0, sizeof(float) * NPARAM);
  for (int k = 0; k < MF; k++) blob[O_IS + k] = 1.0f;
  blob[O_YS] = 1.0f;
  for (int k = 0; k < MH * MF; k++) blob[O_W1 + k] = (float)(nd(rng) * std::sqrt(2.0 / NFEAT));
  for (int k = 0; k < MH * MH; k++) blob[O_W2 + k] = (float)(nd(rng) * std::sqrt(2.0 / MH));
  for (int k = 0; k < MH * MH; k++) blob[O_W3 + k] = (float)(nd(rng) * std::sqrt(2.0 / MH));
  for (int k = 0; k < MH; k++) blob[O_W4 + k] = (float)(nd(rng) * std::sqrt(1.0 / MH));
  return PNM_OK;
}

int pnm_mlp_features(pnm_ctx* ctx, int sys, float* X, double* t_mbpt2, double* sigma) {
  try {
    if (!ctx || sys < 0 || sys >= (int)ctx->sys.size()) throw PnmError{PNM_EINVAL, "bad argument"};
    mlp_features(ctx);
    const SysInfo& S = ctx->sys[sys];
    long n = S.t_end - S.t_begin;
    cudaStream_t s = ctx->stream;
    if (X) CUDA_TRY(cudaMemcpyAsync(X, ctx->mlp->X + S.t_begin * MF, sizeof(float) * n * MF, cudaMemcpyDeviceToHost, s));
    if (t_mbpt2) CUDA_TRY(cudaMemcpyAsync(t_mbpt2, ctx->mlp->tm2 + S.t_begin, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    if (sigma) CUDA_TRY(cudaMemcpyAsync(sigma, ctx->mlp->sigma + sys, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return PNM_OK;
  } catch (const PnmError& e) {
    pnm_set_error(e.code, e.msg);
    return e.code;
  }
}

int pnm_mlp_set_model(pnm_ctx* ctx, const float* blob) {
  try {
    if (!ctx || !blob) throw PnmError{PNM_EINVAL, "null argument"};
    set_model(ctx, blob);
    return PNM_OK;
  } catch (const PnmError& e) {
    pnm_set_error(e.code, e.msg);
    return e.code;
  }
}

int pnm_mlp_predict(pnm_ctx* ctx) {
  try {
    if (!ctx) throw PnmError{PNM_EINVAL, "null argument"};
    pnm_mlp_start(ctx);
    int h_err = 0;
    CUDA_TRY(cudaMemcpyAsync(&h_err, ctx->mlp->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (h_err) {
      CUDA_TRY(cudaMemsetAsync(ctx->mlp->err, 0, sizeof(int), ctx->stream));
      throw PnmError{PNM_ETIMEOUT, "a device-side wait ran out of its budget"};
    }
    return PNM_OK;
  } catch (const PnmError& e) {
    pnm_set_error(e.code, e.msg);
    return e.code;
  }
}

int pnm_mlp_forward(const float* blob, const float* X, long n, float* Y, int mode, void* stream) {
  try {
    if (!blob || !X || !Y || n < 0) throw PnmError{PNM_EINVAL, "bad argument"};
    if (mode != PNM_MLP_SIMT && mode != PNM_MLP_TENSOR_CORES && mode != PNM_MLP_SIMT_FP32)
      throw PnmError{PNM_EINVAL, "unknown forward mode"};
    const bool use_tensor_cores = mode == PNM_MLP_TENSOR_CORES;
    const int rnd = mode == PNM_MLP_SIMT_FP32 ? 0 : 1;
    check_blob_header(blob);
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc;
    float* w = xalloc<float>(NPARAM, sc.owned);
    float* q = xalloc<float>(NPARAM, sc.owned);
    float* dX = xalloc<float>((size_t)n * MF, sc.owned);
    float* dY = xalloc<float>(n, sc.owned);
    CUDA_TRY(cudaMemcpyAsync(w, blob, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(dX, X, sizeof(float) * n * MF, cudaMemcpyHostToDevice, s));
    k_quantize<<<(NPARAM + 255) / 256, 256, 0, s>>>(w, q, rnd);
    if (use_tensor_cores) {
      __nv_bfloat16* pw = xalloc<__nv_bfloat16>(PW_TOTAL, sc.owned);
      int* err = xalloc<int>(1, sc.owned);
      CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
      mlp_tc_attributes();
      k_pack_weights<<<(PW_TOTAL + 255) / 256, 256, 0, s>>>(q, pw);
      tc_infer(s, dX, n, q, pw, MlpOut{dY, nullptr, nullptr, nullptr, nullptr, 0, 1.0f}, err);
      int h_err = 0;
      CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaStreamSynchronize(s));
      if (h_err) throw PnmError{PNM_ETIMEOUT, "a device-side wait ran out of its budget"};
    } else {
      const long chunk = 8192;
      Net nt;
      nt.alloc((int)std::min(chunk, std::max(1L, n)), sc);
      CUDA_TRY(cudaMemcpyAsync(nt.q, q, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, s));
      for (long r0 = 0; r0 < n; r0 += chunk) {
        int B = (int)std::min(chunk, n - r0);
        net_forward(s, nt, dX + r0 * MF, nullptr, B, rnd);
        k_out<<<(B * 32 + 255) / 256, 256, 0, s>>>(nt.H3, nt.q + O_W4, nt.q + O_B4, nullptr, nullptr, B,
                                                   dY + r0, nullptr, nullptr);
      }
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(Y, dY, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return PNM_OK;
  } catch (const PnmError& e) {
    pnm_set_error(e.code, e.msg);
    return e.code;
  }
}

int pnm_mlp_loss_grad(const float* blob, const float* X, const float* T, int n, float* loss, float* grad,
                      int fp32, void* stream) {
  try {
    if (!blob || !X || !T || n <= 0) throw PnmError{PNM_EINVAL, "bad argument"};
    check_blob_header(blob);
    cudaStream_t s = (cudaStream_t)stream;
    if (fp32 < 0 || fp32 > 2) throw PnmError{PNM_EINVAL, "unknown gradient mode"};
    Scratch sc;
    Net nt;
    nt.alloc(n, sc, fp32 == 0 ? 1 : 0, s);  // 0: BF16 on the tensor cores, 2: BF16 on k_sgemm
    float* dX = xalloc<float>((size_t)n * MF, sc.owned);
    float* dT = xalloc<float>(n, sc.owned);
    double* lacc = xalloc<double>(1, sc.owned);
    CUDA_TRY(cudaMemcpyAsync(nt.w, blob, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(dX, X, sizeof(float) * (size_t)n * MF, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(dT, T, sizeof(float) * n, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemsetAsync(lacc, 0, sizeof(double), s));
    const int rnd = fp32 == 1 ? 0 : 1;
    k_quantize<<<(NPARAM + 255) / 256, 256, 0, s>>>(nt.w, nt.q, rnd);
    net_forward(s, nt, dX, nullptr, n, rnd);
    k_out<<<(n * 32 + 255) / 256, 256, 0, s>>>(nt.H3, nt.q + O_W4, nt.q + O_B4, dT, nullptr, n, nt.Y, nt.dY, lacc);
    net_backward(s, nt, n);
    CUDA_TRY(cudaGetLastError());
    double l = 0;
    int h_err = 0;
    CUDA_TRY(cudaMemcpyAsync(&l, lacc, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (grad) CUDA_TRY(cudaMemcpyAsync(grad, nt.g, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, s));
    if (nt.err) CUDA_TRY(cudaMemcpyAsync(&h_err, nt.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (h_err) throw PnmError{PNM_ETIMEOUT, "a device-side wait of the training products ran out of its budget"};
    if (loss) *loss = (float)(l / n);
    return PNM_OK;
  } catch (const PnmError& e) {
    pnm_set_error(e.code, e.msg);
    return e.code;
  }
}

int pnm_mlp_train(pnm_ctx* const* ctxs, int nctx, const pnm_mlp_opts* o, float* blob, float* loss_hist,
                  int cap, int* n_hist) {
  try {
    if (!ctxs || nctx <= 0 || !o || !blob) throw PnmError{PNM_EINVAL, "bad argument"};
    if (o->epochs < 0 || o->batch <= 0 || !(o->lr > 0)) throw PnmError{PNM_EINVAL, "bad options"};
    check_blob_header(blob);
    cudaStream_t s = ctxs[0]->stream;
    long ntot = 0;
    for (int k = 0; k < nctx; k++) {
      if (!ctxs[k]) throw PnmError{PNM_EINVAL, "null context"};
      ntot += ctxs[k]->nt;
    }
    Scratch sc;
    float* X = xalloc<float>((size_t)ntot * MF, sc.owned);
    float* T = xalloc<float>(ntot, sc.owned);
    long off = 0;
    for (int k = 0; k < nctx; k++) {
      pnm_ctx* c = ctxs[k];
      mlp_features(c);
      CUDA_TRY(cudaStreamSynchronize(c->stream));
      k_targets<<<c->n_upd_items, 128, 0, c->stream>>>(c->d, c->upd_items, c->mlp->tm2, c->mlp->sigma, T + off);
      CUDA_TRY(cudaMemcpyAsync(X + off * MF, c->mlp->X, sizeof(float) * c->nt * MF, cudaMemcpyDeviceToDevice,
                               c->stream));
      CUDA_TRY(cudaStreamSynchronize(c->stream));
      off += c->nt;
    }
    // normalisation from the training data
    double* st = xalloc<double>(2 * MF + 2, sc.owned);
    k_featstats<<<MF, 256, 0, s>>>(X, ntot, st);
    std::vector<double> hs(2 * MF + 2);
    CUDA_TRY(cudaMemcpyAsync(hs.data(), st, sizeof(double) * 2 * MF, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    for (int q = 0; q < MF; q++) {
      double mu = hs[2 * q] / ntot, var = hs[2 * q + 1] / ntot - mu * mu;
      blob[O_MU + q] = (float)mu;
      blob[O_IS + q] = var > 1e-12 ? (float)(1.0 / std::sqrt(var)) : 0.0f;
    }
    {
      std::vector<float> ht(ntot);
      CUDA_TRY(cudaMemcpyAsync(ht.data(), T, sizeof(float) * ntot, cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaStreamSynchronize(s));
      double a = 0, b = 0;
      for (float v : ht) {
        a += v;
        b += (double)v * v;
      }
      double var = b / ntot - (a / ntot) * (a / ntot);
      double ys = var > 1e-30 ? std::sqrt(var) : 1.0;
      blob[O_YS] = (float)ys;
      k_scale<<<(unsigned)((ntot + 255) / 256), 256, 0, s>>>(T, ntot, (float)(1.0 / ys));
    }
    int B = (int)std::min<long>(o->batch, ntot);
    Net nt;
    nt.alloc(B, sc, 1, s);  // BF16 training: the matrix products on the tensor cores
    int* idx = xalloc<int>(ntot, sc.owned);
    double* lacc = xalloc<double>(1, sc.owned);
    CUDA_TRY(cudaMemcpyAsync(nt.w, blob, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemsetAsync(nt.m, 0, sizeof(float) * NPARAM, s));
    CUDA_TRY(cudaMemsetAsync(nt.v, 0, sizeof(float) * NPARAM, s));
    k_quantize<<<(NPARAM + 255) / 256, 256, 0, s>>>(nt.w, nt.q);
    std::vector<int> perm(ntot);
    std::iota(perm.begin(), perm.end(), 0);
    std::mt19937_64 rng(g_seed_mix(o->seed));
    long step = 0;
    const long nsteps = (long)o->epochs * (ntot / B);
    const double lr_end = o->lr_final > 0.0 ? o->lr_final : o->lr;
    int nh = 0;
    const float b1 = 0.9f, b2 = 0.999f;
    for (int ep = 0; ep < o->epochs; ep++) {
      std::shuffle(perm.begin(), perm.end(), rng);
      CUDA_TRY(cudaMemcpyAsync(idx, perm.data(), sizeof(int) * ntot, cudaMemcpyHostToDevice, s));
      CUDA_TRY(cudaMemsetAsync(lacc, 0, sizeof(double), s));
      long nb = 0;
      for (long r0 = 0; r0 + B <= ntot; r0 += B, nb++) {
        net_forward(s, nt, X, idx + r0, B);
        k_out<<<(B * 32 + 255) / 256, 256, 0, s>>>(nt.H3, nt.q + O_W4, nt.q + O_B4, T, idx + r0, B, nt.Y, nt.dY,
                                                   lacc);
        net_backward(s, nt, B);
        // half-cosine decay from lr to lr_final over the steps (constant when they are equal)
        const double frac = nsteps > 1 ? (double)step / (double)(nsteps - 1) : 0.0;
        const double lr = lr_end + 0.5 * (o->lr - lr_end) * (1.0 + std::cos(PNM_PI * frac));
        step++;
        float c1 = 1.0f - std::pow(b1, (float)step), c2 = 1.0f - std::pow(b2, (float)step);
        k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(nt.w, nt.g, nt.m, nt.v, nt.q, (float)lr, b1, b2, c1, c2,
                                                    1e-8f);
      }
      CUDA_TRY(cudaGetLastError());
      double l = 0;
      int h_err = 0;
      CUDA_TRY(cudaMemcpyAsync(&l, lacc, sizeof(double), cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaMemcpyAsync(&h_err, nt.err, sizeof(int), cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaStreamSynchronize(s));
      if (h_err) throw PnmError{PNM_ETIMEOUT, "a device-side wait of the training products ran out of its budget"};
      if (loss_hist && nh < cap) loss_hist[nh] = (float)(l / std::max(1L, nb * B));
      nh++;
    }
    std::vector<float> w(NPARAM);
    CUDA_TRY(cudaMemcpyAsync(w.data(), nt.w, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    for (int k = MHEADER; k < NPARAM; k++) blob[k] = w[k];
    if (n_hist) *n_hist = nh;
    return PNM_OK;
  } catch (const PnmError& e) {
    pnm_set_error(e.code, e.msg);
    return e.code;
  }
}

}  // extern "C"
