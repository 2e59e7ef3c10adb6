// iterate.cu -- one CCD update, Eq. (ccd3) of arXiv:1611.06765 written with the
// intermediates of Sec. "Developing a CCD code":
//
//   0 = v_ab^ij + P(ab) chi_b^c t_ac^ij - P(ij) chi_k^j t_ab^ik + 1/2 <ab|chi|cd> t_cd^ij
//       + 1/2 t_ab^kl <kl|chi|ij> + P(ij)P(ab) t_ik^ac <kb|chi|cj>
//
// with chi_b^c, chi_k^j diagonal here (momentum and S_z conservation), blocked per direct
// channel (restricted pairs) and per cross channel (ordered ph/hp pairs).  Kernels:
//   k_tstats   row and column sums of t o v (one-body intermediates) and
//              <kl|chi|ij> = <kl|v|ij> + 1/2 <kl|v|cd> t_ij^cd per direct channel
//   k_dchi     chi_p - eps_p per state, gathered over the pairs holding p
//   k_ph       T_x = remap(t); C_x = V1_x + 1/2 W_x T_x; Q_x = T_x C_x per cross channel
//   k_pp64     1/2 sum_cd <ab|v|cd> t_cd^ij, grouped over all channels with a V_pppp block (FP64)
//   k_update   Jacobi step t_new = (v + rest) / eps_ij^ab, mixing, energy/residual partials
//   finalize   (last block of k_update) Eq. (ccdcorr) energy per system, |dE| test,
//              device-side loop condition
#include <cmath>
#include <cstdio>
#include <map>
#include <algorithm>
#include <chrono>
#include <mutex>
#include <type_traits>

#include "pnm_context.cuh"

#ifndef PNM_UPD_HH_UNROLL
#define PNM_UPD_HH_UNROLL 4
#endif
constexpr int UPD_HH_UNROLL = PNM_UPD_HH_UNROLL;  // loads of the mixed update's hh-ladder pass in flight


// ----------------------------------------------------------------------------- stats
// Element type T_: double for the FP64 iteration (t, v_pphh, v_hhhh, chi_hh, sij, sab), float
// for the mixed-precision one (their FP32 copies).
template <typename T_>
struct StatsIO {
  const T_ *t, *v, *vhh;
  T_ *chi, *sij, *sab;
  __device__ StatsIO(const DevState& D, const LoopCtl* ctl) {
    if constexpr (std::is_same<T_, double>::value) {
      t = cur_t(D, ctl); v = D.v_pphh; vhh = D.v_hhhh; chi = D.chi_hh; sij = D.sij; sab = D.sab;
    } else {
      t = cur_t32(D, ctl); v = D.v32; vhh = D.vhh32; chi = D.chi32; sij = D.sij32; sab = D.sab32;
    }
  }
};

// Blocks [0, nrows): row (c, kl): sij[kl] = sum_ab t v; chi_hh[kl][ij] for the ij the updates
// compute.
// Blocks [nrows, ...): column chunk (c, ab0): sab[ab] = sum_ij t v.
// PAIR (FP64 only): the contractions in FP32-pair arithmetic from the pair copies tp of t and vp
// of v_pphh (the refinement sweeps): chi_hh, and the one-body sums as per-thread pair partials
// added in FP64.
template <typename T_, bool PAIR = false>
__global__ void __launch_bounds__(128) k_tstats(DevState D, const LoopCtl* __restrict__ ctl,
                                                int nrows, const int2* __restrict__ ab_items,
                                                const f2* __restrict__ tp = nullptr,
                                                const f2* __restrict__ vp = nullptr) {
  __shared__ T_ sh32[32];
  StatsIO<T_> io(D, ctl);
  const T_* __restrict__ t = io.t;
  if ((int)blockIdx.x < nrows) {
    int2 it = D.row_item[blockIdx.x];
    int c = it.x, kl = it.y;
    if (sys_done(D, ctl, D.ch_sys[c])) return;
    int npp = D.ch_npp[c], nh = D.ch_nhh[c];
    long base = D.ch_t_off[c];
    const T_* tr = t + base + (long)kl * npp;
    const T_* vr = io.v + base + (long)kl * npp;
    T_ s = 0;
    if constexpr (PAIR) {
      // per-thread partial sums in FP32 pairs, the block sum in FP64
      const f2* __restrict__ tpr = tp + base + (long)kl * npp;
      const f2* __restrict__ vpr = vp + base + (long)kl * npp;
      f2 a2 = Arith<f2>::zero();
      for (int ab = threadIdx.x; ab < npp; ab += blockDim.x) Arith<f2>::mac(a2, tpr[ab], vpr[ab]);
      s = Arith<f2>::to_double(a2);
    } else {
      for (int ab = threadIdx.x; ab < npp; ab += blockDim.x) s += tr[ab] * vr[ab];
    }
    s = block_sum(s, sh32);
    if (threadIdx.x == 0) io.sij[D.ch_hh_off[c] + kl] = s;
    // chi is read only in the columns ij of the rows the updates compute (the list upd_row)
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int* __restrict__ rl = D.upd_row + D.ch_uoff[c];
    const int nr = D.ch_uoff[c + 1] - D.ch_uoff[c];
    for (int k = warp; k < nr; k += blockDim.x >> 5) {
      const int ij = rl[k];
      T_ acc = 0;
      if constexpr (PAIR) {
        const f2* __restrict__ vk = vp + base + (long)kl * npp;
        const f2* __restrict__ tj = tp + base + (long)ij * npp;
        f2 a2 = Arith<f2>::zero();
        for (int cd = lane; cd < npp; cd += 32) Arith<f2>::mac(a2, vk[cd], tj[cd]);
        for (int o = 16; o; o >>= 1)
          a2 = Arith<f2>::add(a2, f2{__shfl_xor_sync(0xffffffffu, a2.hi, o),
                                     __shfl_xor_sync(0xffffffffu, a2.lo, o)});
        acc = Arith<f2>::to_double(a2);
      } else {
        const T_* tj = t + base + (long)ij * npp;
        for (int cd = lane; cd < npp; cd += 32) acc += vr[cd] * tj[cd];
        acc = warp_sum(acc);
      }
      if (lane == 0) {
        long e = D.ch_vhh_off[c] + (long)kl * nh + ij;
        io.chi[e] = io.vhh[e] + acc;
      }
    }
  } else {
    int2 it = ab_items[blockIdx.x - nrows];
    int c = it.x, ab = it.y + threadIdx.x;
    if (sys_done(D, ctl, D.ch_sys[c])) return;
    int npp = D.ch_npp[c], nh = D.ch_nhh[c];
    if (ab < npp) {
      long base = D.ch_t_off[c] + ab;
      T_ s = 0;
      if constexpr (PAIR) {
        f2 a2 = Arith<f2>::zero();
        for (int ij = 0; ij < nh; ij++) Arith<f2>::mac(a2, tp[base + (long)ij * npp], vp[base + (long)ij * npp]);
        s = Arith<f2>::to_double(a2);
      } else {
        for (int ij = 0; ij < nh; ij++) s += t[base + (long)ij * npp] * io.v[base + (long)ij * npp];
      }
      io.sab[D.ch_pp_off[c] + ab] = s;
    }
  }
}

// chi_b - eps_b = -sum_d sum_{k<l} t_kl^bd v_kl^bd   (particles)
// chi_j - eps_j = +sum_l sum_{c<d} v_jl^cd t_jl^cd   (holes)
template <typename T_>
__global__ void k_dchi(DevState D, int nsp_total) {
  int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (p >= nsp_total) return;
  constexpr bool F64 = std::is_same<T_, double>::value;
  int lo = D.occ_off[p], hi = D.occ_off[p + 1];
  bool hole = D.sp_hole[p] != 0;
  const T_* src;
  if constexpr (F64) src = hole ? D.sij : D.sab;
  else src = hole ? D.sij32 : D.sab32;
  T_ s = 0;
  for (int k = lo + lane; k < hi; k += 32) s += src[D.occ_idx[k]];
  s = warp_sum(s);
  if (lane == 0) {
    if constexpr (F64) D.dchi[p] = hole ? s : -s;
    else D.dchi32[p] = hole ? s : -s;
  }
}

// ----------------------------------------------------------------------------- ph term
// Global spin flip: Q is formed for the cross channels with S_z > 0 and for the spin-up rows of
// the S_z = 0 channels; the update reads every other position at its flip (same value for
// flip-symmetric amplitudes; qmap holds the formed positions only).  In an
// S_z = 0 channel, with rows ordered (spin-up rows u, their flips F u) and columns alike,
// every matrix of the term has the block form [[A, B], [B, A]] (A = M[u][v], B = M[u][F v]);
// products of such matrices are formed from the half-size sums A + B and differences A - B,
//   (A_1 + B_1)(A_2 + B_2) = A_3 + B_3,  (A_1 - B_1)(A_2 - B_2) = A_3 - B_3,
// which is a quarter of the flops of the full channel.
template <typename T_, int TS>
struct VecT;
template <>
struct VecT<double, 2> {
  __device__ __forceinline__ static void ld(const double* p, double (&v)[2]) {
    double2 a = *reinterpret_cast<const double2*>(p);
    v[0] = a.x; v[1] = a.y;
  }
};
template <>
struct VecT<float, 2> {
  __device__ __forceinline__ static void ld(const float* p, float (&v)[2]) {
    float2 a = *reinterpret_cast<const float2*>(p);
    v[0] = a.x; v[1] = a.y;
  }
};
template <>
struct VecT<float, 4> {
  __device__ __forceinline__ static void ld(const float* p, float (&v)[4]) {
    float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
};
template <>
struct VecT<f2, 2> {
  __device__ __forceinline__ static void ld(const f2* p, f2 (&v)[2]) {
    float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = f2{q.x, q.y}; v[1] = f2{q.z, q.w};
  }
};

// Element e of a cross channel's T: read from the FP32 copy in the cross-channel layout that
// the mixed update scatters (xt), or gathered through the signed index map from the current
// amplitudes (tcur): FP64, or their FP32-pair copy for the FP32-pair kernels.
template <typename T_>
__device__ __forceinline__ T_ ph_t(const DevState& D, const T_* __restrict__ tcur,
                                   const T_* __restrict__ xt, long e) {
  using A = Arith<T_>;
  if (xt) return xt[e];
  int cd = D.xmap[e];
  if (cd == 0) return A::zero();
  T_ g = tcur[cd > 0 ? cd - 1 : -cd - 1];
  return cd < 0 ? A::neg(g) : g;
}

// Bytes reserved for the index tables at the start of a k_ph CTA's shared memory (R4 + 2 H4
// ints are used; 2 (R4 + H4) with R4, H4 even keeps the reservation a multiple of 16 bytes).
__host__ __device__ __forceinline__ size_t ph_index_bytes(int R4, int H4) { return sizeof(int) * 2 * (size_t)(R4 + H4); }

// One CTA (NT threads) per cross channel.  NM = 1: a channel with S_z > 0.  NM = 2: an S_z = 0
// channel as the pair (sum, difference) of half-size problems, Q written on its spin-up rows.
// Per problem, in shared memory zero-padded to multiples of TS (R rows (a,i), H columns (k,c)):
//   Ts = T (R x H), Xt = W^T staged as W (R x H), then T^T (H x R), Cs = C (H x H);
//   C[(k,c)][(j,b)] = <kb|v|cj> + 1/2 sum_(e,l) <kl|v|ce> t_lj^eb   (xw == nullptr: <kb|v|cj>)
//   Q[(a,i)][(j,b)] = sum_(k,c) t_ik^ac C[(k,c)][(j,b)]
// Each thread accumulates TS x TS outputs of every problem per tile.  Element arithmetic is
// that of Arith<T_> (FP64, FP32, or FP32 pairs with FP64 results).
template <typename T_, int NT, int TS, int NM>
__device__ __forceinline__ void ph_block(const DevState& D, int x, unsigned char* smraw,
                                         const T_* __restrict__ tcur, const T_* __restrict__ xt,
                                         const T_* __restrict__ xw, const T_* __restrict__ xv1,
                                         typename Arith<T_>::Out* __restrict__ xq) {
  using A = Arith<T_>;
  const int nph = D.x_nph[x], nhp = D.x_nhp[x];
  const int R = NM == 2 ? nph >> 1 : nph, H = NM == 2 ? nhp >> 1 : nhp;
  // padded to multiples of the register tile (zeros): the padding costs FMAs in the tiles
  const int R4 = (R + TS - 1) & ~(TS - 1), H4 = (H + TS - 1) & ~(TS - 1);
  const int RH = R4 * H4, HH = H4 * H4;
  // NM = 2: index tables in shared memory first (no chains of dependent global loads below):
  // sra[u] = spin-up row, sca[v] = spin-up column, scb[v] = its flip
  int* sra = reinterpret_cast<int*>(smraw);
  int* sca = sra + R4;
  int* scb = sca + H4;
  T_* Ts = reinterpret_cast<T_*>(smraw + ph_index_bytes(R4, H4));
  T_* Xt = Ts + NM * RH;
  T_* Cs = Xt + NM * RH;
  const long to = D.x_t_off[x], wo = D.x_w_off[x], co = D.x_c_off[x];
  if constexpr (NM == 2) {
    const int* __restrict__ fcol = D.x_fcol + D.x_hp_off[x];
    const int* __restrict__ rrow = D.x_rrow + D.x_ph_off[x];
    const int* __restrict__ rcol = D.x_rcol + D.x_hp_off[x];
    for (int k = threadIdx.x; k < R4; k += NT) sra[k] = k < R ? rrow[k] : 0;
    for (int k = threadIdx.x; k < H4; k += NT) {
      int a = k < H ? rcol[k] : 0;
      sca[k] = a;
      scb[k] = k < H ? fcol[a] : 0;
    }
    __syncthreads();
  }
  const bool quad = xw != nullptr;
  // element e = u H4 + s of the staging loops: (u, s) advanced by NT per step without a division
  const int du = NT / H4, ds = NT % H4;
  int u = threadIdx.x / H4, s = threadIdx.x % H4;
#pragma unroll 4
  for (int e = threadIdx.x; e < RH; e += NT) {
    T_ t0 = A::zero(), t1 = A::zero(), w0 = A::zero(), w1 = A::zero();
    if (u < R && s < H) {
      if constexpr (NM == 1) {
        long o = (long)u * nhp + s;
        t0 = ph_t<T_>(D, tcur, xt, to + o);
        if (quad) w0 = xw[wo + o];
      } else {
        int row = sra[u], ca = sca[s], cb = scb[s];
        long oa = (long)row * nhp + ca, ob = (long)row * nhp + cb;
        T_ ta = ph_t<T_>(D, tcur, xt, to + oa), tb = ph_t<T_>(D, tcur, xt, to + ob);
        t0 = A::add(ta, tb);
        t1 = A::sub(ta, tb);
        if (quad) {
          T_ wa = xw[wo + oa], wb = xw[wo + ob];
          w0 = A::add(wa, wb);
          w1 = A::sub(wa, wb);
        }
      }
    }
    Ts[e] = t0;
    Xt[e] = w0;
    if constexpr (NM == 2) {
      Ts[RH + e] = t1;
      Xt[RH + e] = w1;
    }
    u += du;
    s += ds;
    if (s >= H4) {
      s -= H4;
      u++;
    }
  }
  int r = threadIdx.x / H4, c = threadIdx.x % H4;
#pragma unroll 4
  for (int e = threadIdx.x; e < HH; e += NT) {
    T_ v0 = A::zero(), v1 = A::zero();
    if (r < H && c < H) {
      if constexpr (NM == 1) {
        v0 = xv1[co + (long)r * nhp + c];
      } else {
        const long ra = co + (long)sca[r] * nhp;
        T_ va = xv1[ra + sca[c]], vb = xv1[ra + scb[c]];
        v0 = A::add(va, vb);
        v1 = A::sub(va, vb);
      }
    }
    Cs[e] = v0;
    if constexpr (NM == 2) Cs[HH + e] = v1;
    r += du;
    c += ds;
    if (c >= H4) {
      c -= H4;
      r++;
    }
  }
  __syncthreads();
  const int th = H4 / TS;
  if (quad) {
    // C += 1/2 W^T T (padded rows and columns stay zero)
    for (int tile = threadIdx.x; tile < NM * th * th; tile += NT) {
      const int mtx = tile / (th * th), tt = tile % (th * th);
      const int r0 = (tt / th) * TS, s0 = (tt % th) * TS;
      const T_* X = Xt + mtx * RH;
      const T_* Tm = Ts + mtx * RH;
      T_ acc[TS][TS];
#pragma unroll
      for (int i = 0; i < TS; i++)
#pragma unroll
        for (int j = 0; j < TS; j++) acc[i][j] = A::zero();
      for (int u = 0; u < R; u++) {
        T_ a[TS], b[TS];
        VecT<T_, TS>::ld(X + u * H4 + r0, a);
        VecT<T_, TS>::ld(Tm + u * H4 + s0, b);
#pragma unroll
        for (int i = 0; i < TS; i++)
#pragma unroll
          for (int j = 0; j < TS; j++) A::mac(acc[i][j], a[i], b[j]);
      }
      T_* Cm = Cs + mtx * HH;
#pragma unroll
      for (int i = 0; i < TS; i++)
#pragma unroll
        for (int j = 0; j < TS; j++) {
          T_& cv = Cm[(r0 + i) * H4 + s0 + j];
          cv = A::add(cv, A::half(acc[i][j]));
        }
    }
    __syncthreads();
  }
  // T transposed into Xt: Xt[s][u] = T[u][s]
  for (int e = threadIdx.x; e < NM * RH; e += NT) {
    const int mtx = e / RH, f = e % RH;
    Xt[mtx * RH + (f % H4) * R4 + f / H4] = Ts[e];
  }
  __syncthreads();
  const int tr = R4 / TS;
  for (int tile = threadIdx.x; tile < tr * th; tile += NT) {
    const int r0 = (tile / th) * TS, s0 = (tile % th) * TS;
    T_ acc[NM][TS][TS];
#pragma unroll
    for (int m = 0; m < NM; m++)
#pragma unroll
      for (int i = 0; i < TS; i++)
#pragma unroll
        for (int j = 0; j < TS; j++) acc[m][i][j] = A::zero();
    for (int u = 0; u < H; u++) {
#pragma unroll
      for (int mtx = 0; mtx < NM; mtx++) {
        T_ a[TS], b[TS];
        VecT<T_, TS>::ld(Xt + mtx * RH + u * R4 + r0, a);
        VecT<T_, TS>::ld(Cs + mtx * HH + u * H4 + s0, b);
#pragma unroll
        for (int i = 0; i < TS; i++)
#pragma unroll
          for (int j = 0; j < TS; j++) A::mac(acc[mtx][i][j], a[i], b[j]);
      }
    }
#pragma unroll
    for (int i = 0; i < TS; i++) {
      const int r = r0 + i;
      if (r >= R) continue;
      if constexpr (NM == 1) {
        const long qr = to + (long)r * nhp;
#pragma unroll
        for (int j = 0; j < TS; j++)
          if (s0 + j < H) xq[qr + s0 + j] = A::out(acc[0][i][j]);
      } else {
        // the spin-up row's two blocks; the flipped rows are never read (see qpos)
        const long qa = to + (long)sra[r] * nhp;
#pragma unroll
        for (int j = 0; j < TS; j++) {
          const int s = s0 + j;
          if (s < H) {
            xq[qa + sca[s]] = A::out(A::half(A::add(acc[0][i][j], acc[1][i][j])));
            xq[qa + scb[s]] = A::out(A::half(A::sub(acc[0][i][j], acc[1][i][j])));
          }
        }
      }
    }
  }
}

// Cross channels of at most PH_WARP_DIM rows and columns (of their halves for S_z = 0): one
// warp per channel with its own shared buffers (stride PH_WARP_DIM), no block-wide
// synchronisation; the same two bodies as the CTA path, one output element per lane and step.
constexpr int PH_WARPS = PH_THREADS / 32;
template <typename T_>
__device__ __forceinline__ void ph_warp_body(const DevState& D, int x, int w, int lane, unsigned char* smraw,
                                             const T_* __restrict__ tcur, const T_* __restrict__ xt,
                                             const T_* __restrict__ xw, const T_* __restrict__ xv1,
                                             typename Arith<T_>::Out* __restrict__ xq) {
  using A = Arith<T_>;
  constexpr int S = PH_WARP_DIM;
  const int nph = D.x_nph[x], nhp = D.x_nhp[x];
  const bool two = D.x_cls[x] == 0;
  const int nm = two ? 2 : 1;
  const int R = two ? nph >> 1 : nph, H = two ? nhp >> 1 : nhp;
  const long to = D.x_t_off[x], wo = D.x_w_off[x], co = D.x_c_off[x];
  T_* Ts = reinterpret_cast<T_*>(smraw) + (size_t)w * 6 * S * S;  // [m][u][s]
  T_* Ws = Ts + 2 * S * S;                                         // [m][u][r] = W[u][r]
  T_* Cs = Ws + 2 * S * S;                                         // [m][r][s]
  int* sra = reinterpret_cast<int*>(reinterpret_cast<T_*>(smraw) + (size_t)PH_WARPS * 6 * S * S) + w * 3 * S;
  int* sca = sra + S;
  int* scb = sca + S;
  if (two) {
    const int* __restrict__ fcol = D.x_fcol + D.x_hp_off[x];
    const int* __restrict__ rrow = D.x_rrow + D.x_ph_off[x];
    const int* __restrict__ rcol = D.x_rcol + D.x_hp_off[x];
    if (lane < R) sra[lane] = rrow[lane];
    if (lane < H) {
      int a = rcol[lane];
      sca[lane] = a;
      scb[lane] = fcol[a];
    }
  }
  __syncwarp();
  const bool quad = xw != nullptr;
  for (int e = lane; e < R * H; e += 32) {
    int u = e / H, c = e % H;
    if (two) {
      long oa = (long)sra[u] * nhp + sca[c], ob = (long)sra[u] * nhp + scb[c];
      T_ ta = ph_t<T_>(D, tcur, xt, to + oa), tb = ph_t<T_>(D, tcur, xt, to + ob);
      Ts[u * S + c] = A::add(ta, tb);
      Ts[S * S + u * S + c] = A::sub(ta, tb);
      T_ wa = quad ? xw[wo + oa] : A::zero(), wb = quad ? xw[wo + ob] : A::zero();
      Ws[u * S + c] = A::add(wa, wb);
      Ws[S * S + u * S + c] = A::sub(wa, wb);
    } else {
      long o = (long)u * nhp + c;
      Ts[u * S + c] = ph_t<T_>(D, tcur, xt, to + o);
      Ws[u * S + c] = quad ? xw[wo + o] : A::zero();
    }
  }
  __syncwarp();
  for (int e = lane; e < H * H; e += 32) {
    int r = e / H, c = e % H;
    for (int m = 0; m < nm; m++) {
      T_ v;
      if (two) {
        const long ra = co + (long)sca[r] * nhp;
        T_ va = xv1[ra + sca[c]], vb = xv1[ra + scb[c]];
        v = m == 0 ? A::add(va, vb) : A::sub(va, vb);
      } else {
        v = xv1[co + (long)r * nhp + c];
      }
      T_ acc = A::zero();
      for (int u = 0; u < R && quad; u++) A::mac(acc, Ws[m * S * S + u * S + r], Ts[m * S * S + u * S + c]);
      Cs[m * S * S + r * S + c] = A::add(v, A::half(acc));
    }
  }
  __syncwarp();
  for (int e = lane; e < R * H; e += 32) {
    int r = e / H, c = e % H;
    T_ acc[2] = {A::zero(), A::zero()};
    for (int m = 0; m < nm; m++)
      for (int u = 0; u < H; u++) A::mac(acc[m], Ts[m * S * S + r * S + u], Cs[m * S * S + u * S + c]);
    if (two) {
      const long qa = to + (long)sra[r] * nhp;
      xq[qa + sca[c]] = A::out(A::half(A::add(acc[0], acc[1])));
      xq[qa + scb[c]] = A::out(A::half(A::sub(acc[0], acc[1])));
    } else {
      xq[to + (long)r * nhp + c] = A::out(acc[0]);
    }
  }
}

// The current amplitudes the ph kernels gather T from (not used when T is read from the
// scattered FP32 copy): FP64, or the FP32-pair copy made at the start of the sweep.
template <typename T_>
__device__ __forceinline__ const T_* ph_tcur(const DevState& D, const LoopCtl* ctl, const T_* tpair) {
  if constexpr (std::is_same<T_, double>::value) return cur_t(D, ctl);
  else return tpair;
}

// The ph term over the S_z >= 0 cross channels (xlist): the first nblk CTAs take one channel
// each (the costliest first), with the S_z > 0 or the S_z = 0 body chosen per channel; the
// remaining CTAs take PH_WARPS small channels each, one per warp.  Channels are launched in two
// size classes with their own shared memory (the larger ones by k_ph_big).
template <typename T_, int NT, int TS>
__global__ void __launch_bounds__(NT) k_ph(DevState D, const LoopCtl* __restrict__ ctl,
                                           const int* __restrict__ xlist, int nblk, int nwarp,
                                           const T_* __restrict__ tpair, const T_* __restrict__ xt,
                                           const T_* __restrict__ xw, const T_* __restrict__ xv1,
                                           typename Arith<T_>::Out* __restrict__ xq) {
  static_assert(NT == PH_WARPS * 32, "one warp per small channel");
  extern __shared__ __align__(16) unsigned char smraw[];
  const T_* tcur = xt ? nullptr : ph_tcur<T_>(D, ctl, tpair);
  if ((int)blockIdx.x < nblk) {
    const int x = xlist[blockIdx.x];
    if (sys_done(D, ctl, D.x_sys[x])) return;  // CTA-uniform
    if (D.x_cls[x] == 0)
      ph_block<T_, NT, TS, 2>(D, x, smraw, tcur, xt, xw, xv1, xq);
    else
      ph_block<T_, NT, TS, 1>(D, x, smraw, tcur, xt, xw, xv1, xq);
    return;
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int idx = ((int)blockIdx.x - nblk) * PH_WARPS + w;
  if (idx >= nwarp) return;  // whole warps leave; the warp path never synchronises the block
  const int x = xlist[nblk + idx];
  if (sys_done(D, ctl, D.x_sys[x])) return;  // warp-uniform
  ph_warp_body<T_>(D, x, w, lane, smraw, tcur, xt, xw, xv1, xq);
}

// The channels of the larger size class: one CTA of PH_BIG_THREADS per channel.
constexpr int PH_BIG_THREADS = 256;
template <typename T_, int TS>
__global__ void __launch_bounds__(PH_BIG_THREADS) k_ph_big(DevState D, const LoopCtl* __restrict__ ctl,
                                                           const int* __restrict__ xlist,
                                                           const T_* __restrict__ tpair, const T_* __restrict__ xt,
                                                           const T_* __restrict__ xw, const T_* __restrict__ xv1,
                                                           typename Arith<T_>::Out* __restrict__ xq) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int x = xlist[blockIdx.x];
  if (sys_done(D, ctl, D.x_sys[x])) return;  // CTA-uniform
  const T_* tcur = xt ? nullptr : ph_tcur<T_>(D, ctl, tpair);
  if (D.x_cls[x] == 0)
    ph_block<T_, PH_BIG_THREADS, TS, 2>(D, x, smraw, tcur, xt, xw, xv1, xq);
  else
    ph_block<T_, PH_BIG_THREADS, TS, 1>(D, x, smraw, tcur, xt, xw, xv1, xq);
}

static size_t ph_warp_smem(size_t elem) {
  return (size_t)PH_WARPS * (6 * PH_WARP_DIM * PH_WARP_DIM * elem + 3 * PH_WARP_DIM * sizeof(int));
}

// Shared memory of a k_ph CTA for channels of at most max_dim (NM = 1) or 2 max_dim (NM = 2)
// rows and columns: the index tables, then NM problems of Ts, Xt (R x H) and Cs (H x H).
size_t ph_smem_bytes(int max_dim, int nm, size_t elem) {
  int m4 = (max_dim + 3) & ~3;
  return ph_index_bytes(m4, m4) + elem * 3 * (size_t)nm * m4 * m4;
}

// Shared memory of the launches: the larger size class alone (k_ph_big); for the 8-byte types
// the middle and the small class each alone and the warp path alone (PNM_PH_CLASSES = 4), or
// the smaller classes with the warp path in one launch (2, the default: the tails of the extra
// launches cost more than their higher occupancy gains); FP32 in one launch.
#ifndef PNM_PH_CLASSES
#define PNM_PH_CLASSES 2
#endif
template <typename T_>
static size_t ph_smem_of(const pnm_ctx* ctx) {
  size_t b = sizeof(T_) == 8 ? std::max(ctx->ph_smem64, ctx->ph_mid_smem64)
                             : std::max(std::max(ctx->ph_smem32, ctx->ph_mid_smem32), ctx->ph_big_smem32);
  return ctx->n_ph_warp > 0 ? std::max(b, ph_warp_smem(sizeof(T_))) : b;
}
template <typename T_>
static size_t ph_big_smem_of(const pnm_ctx* ctx) {
  return sizeof(T_) == 8 ? ctx->ph_big_smem64 : ctx->ph_big_smem32;
}

// Register tile of the ph kernels: 2 x 2 for FP64 (little padding; the FP64 pipe bounds the
// kernel) and FP32 pairs, 4 x 4 for FP32 (fewer shared-memory loads per FMA).
#ifndef PNM_PH32_TILE
#define PNM_PH32_TILE 4
#endif
template <typename T_>
constexpr int ph_tile() { return std::is_same<T_, float>::value ? PNM_PH32_TILE : 2; }

// The ph term: one launch over the S_z >= 0 cross channels (ph_list, costliest first).
// The 8-byte element types (FP64, FP32 pairs) are limited by shared memory: the larger channels
// go to k_ph_big with their own allocation so that the others fit more CTAs per SM.  FP32 is
// limited by registers: one launch, the larger channels first.
template <typename T_>
static void launch_ph_list(pnm_ctx* ctx, const T_* tpair, const T_* xt, const T_* xw, const T_* xv1,
                           typename Arith<T_>::Out* xq, cudaStream_t s) {
  constexpr int TS = ph_tile<T_>();
  constexpr bool split = sizeof(T_) == 8;
  const int nwb = (ctx->n_ph_warp + PH_WARPS - 1) / PH_WARPS;
  if (!split) {
    // FP32: every channel in one launch, the larger first
    const int nblk = ctx->n_ph_big + ctx->n_ph_mid + ctx->n_ph;
    if (nblk + nwb > 0)
      k_ph<T_, PH_THREADS, TS><<<nblk + nwb, PH_THREADS, ph_smem_of<T_>(ctx), s>>>(
          ctx->d, ctx->ctl, ctx->ph_list, nblk, ctx->n_ph_warp, tpair, xt, xw, xv1, xq);
    return;
  }
  if (ctx->n_ph_big > 0)
    k_ph_big<T_, TS><<<ctx->n_ph_big, PH_BIG_THREADS, ph_big_smem_of<T_>(ctx), s>>>(
        ctx->d, ctx->ctl, ctx->ph_list, tpair, xt, xw, xv1, xq);
  const int* mid = ctx->ph_list + ctx->n_ph_big;
  if (PNM_PH_CLASSES == 4) {
    const int* small = mid + ctx->n_ph_mid;
    const int* warp = small + ctx->n_ph;
    if (ctx->n_ph_mid > 0)
      k_ph<T_, PH_THREADS, TS><<<ctx->n_ph_mid, PH_THREADS, ctx->ph_mid_smem64, s>>>(
          ctx->d, ctx->ctl, mid, ctx->n_ph_mid, 0, tpair, xt, xw, xv1, xq);
    if (ctx->n_ph > 0)
      k_ph<T_, PH_THREADS, TS><<<ctx->n_ph, PH_THREADS, ctx->ph_smem64, s>>>(
          ctx->d, ctx->ctl, small, ctx->n_ph, 0, tpair, xt, xw, xv1, xq);
    if (nwb > 0)
      k_ph<T_, PH_THREADS, TS><<<nwb, PH_THREADS, ph_warp_smem(sizeof(T_)), s>>>(
          ctx->d, ctx->ctl, warp, 0, ctx->n_ph_warp, tpair, xt, xw, xv1, xq);
  } else {
    const int nblk = ctx->n_ph_mid + ctx->n_ph;
    if (nblk + nwb > 0)
      k_ph<T_, PH_THREADS, TS><<<nblk + nwb, PH_THREADS, ph_smem_of<T_>(ctx), s>>>(
          ctx->d, ctx->ctl, mid, nblk, ctx->n_ph_warp, tpair, xt, xw, xv1, xq);
  }
}

template <typename T_>
static void ph_attributes(const pnm_ctx* ctx) {
  smem_at_least(k_ph<T_, PH_THREADS, ph_tile<T_>()>, ph_smem_of<T_>(ctx));
  smem_at_least(k_ph_big<T_, ph_tile<T_>()>, ph_big_smem_of<T_>(ctx));
}

// FP64 ph: T gathered from the current FP64 amplitudes (linear: without the quadratic part).
void launch_ph64(pnm_ctx* ctx, cudaStream_t s, bool linear) {
  launch_ph_list<double>(ctx, nullptr, nullptr, linear ? nullptr : ctx->d.x_w, ctx->d.x_v1, ctx->d.xq, s);
}

// The same term with FP32-pair arithmetic (T gathered from the FP32-pair copy of the current
// amplitudes, W and <kb|v|cj> split into FP32 pairs once per context, Q stored as FP32 pairs in
// the 8-byte slots of the FP64 Q): the contractions of the refinement sweeps.
void launch_ph_f2(pnm_ctx* ctx, const f2* tpair, const f2* xw, const f2* xv1, cudaStream_t s) {
  launch_ph_list<f2>(ctx, tpair, nullptr, xw, xv1, reinterpret_cast<f2*>(ctx->d.xq), s);
}

// Mixed ph: T read from the FP32 cross-channel copy the update scatters, Q in FP32 at its
// cross-channel positions (the update gathers the four terms of each amplitude).
void launch_ph_mix(pnm_ctx* ctx, const float* xt, const float* xw, const float* xv1, float* xq, cudaStream_t s) {
  launch_ph_list<float>(ctx, nullptr, xt, xw, xv1, xq, s);
}

void pnm_ph_attributes(const pnm_ctx* ctx) {
  ph_attributes<double>(ctx);
  ph_attributes<float>(ctx);
  ph_attributes<f2>(ctx);
}

// ------------------------------------------------------------------------ ladder basis
// s(ij, q) = sum over the (one or two) pairs of vector q of sign * t(ij, pair), from the current
// amplitudes (FP64, tsrc == nullptr) or their FP32-pair copy (tsrc); one CTA per (channel, ij)
// row of a channel with V_pppp.
template <typename T_>
__global__ void __launch_bounds__(128) k_lad_gather(DevState D, const LoopCtl* __restrict__ ctl,
                                                    const int2* __restrict__ rows, const T_* __restrict__ tsrc,
                                                    T_* __restrict__ out) {
  using A = Arith<T_>;
  int2 it = rows[blockIdx.x];
  int c = it.x, ij = it.y;
  if (sys_done(D, ctl, D.ch_sys[c])) return;
  const T_* __restrict__ t;
  if constexpr (std::is_same<T_, double>::value) t = cur_t(D, ctl);
  else t = tsrc;
  int npp = D.ch_npp[c], nl = D.ch_nlad[c], off = D.ch_pp_off[c];
  const T_* tr = t + D.ch_t_off[c] + (long)ij * npp;
  T_* o = out + D.ch_s_off[c] + (long)ij * nl;
  for (int q = threadIdx.x; q < nl; q += blockDim.x) {
    int2 m = D.lad_mem[off + q];
    T_ a = tr[(m.x > 0 ? m.x : -m.x) - 1];
    T_ v = m.x > 0 ? a : A::neg(a);
    if (m.y != 0) {
      T_ b = tr[(m.y > 0 ? m.y : -m.y) - 1];
      v = A::add(v, m.y > 0 ? b : A::neg(b));
    }
    o[q] = v;
  }
}

// FP32-pair copy of the current amplitudes (the start of a sweep with FP32-pair contractions).
__global__ void k_split_cur(DevState D, const LoopCtl* __restrict__ ctl, f2* __restrict__ tp, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) tp[i] = Arith<f2>::from_double(cur_t(D, ctl)[i]);
}

void pnm_split_cur(pnm_ctx* ctx, cudaStream_t s) {
  if (ctx->nt > 0)
    k_split_cur<<<(unsigned)((ctx->nt + 255) / 256), 256, 0, s>>>(ctx->d, ctx->ctl, ctx->t_pair, ctx->nt);
}

// The pp ladder in the amplitude layout, from its ladder-layout value (planes summed): zero in
// channels without V_pppp.  One CTA per (channel, ij) row.
template <typename T_>
__global__ void __launch_bounds__(128) k_lad_expand(DevState D, const T_* __restrict__ rs, int planes,
                                                    long pstride, double* __restrict__ out) {
  using A = Arith<T_>;
  int2 it = D.row_item[blockIdx.x];
  int c = it.x, ij = it.y;
  int npp = D.ch_npp[c];
  bool vpp = D.ch_vpp[c] != 0;
  double* o = out + D.ch_t_off[c] + (long)ij * npp;
  for (int ab = threadIdx.x; ab < npp; ab += blockDim.x) {
    double v = 0.0;
    if (vpp) {
      int sg;
      long z = lad_index(D, c, ij, ab, sg);
      T_ a = A::zero();
      for (int p = 0; p < planes; p++) a = A::add(a, rs[p * pstride + z]);
      v = sg > 0 ? A::to_double(a) : -A::to_double(a);
    }
    o[ab] = v;
  }
}

// ---------------------------------------------------------------------- pp ladder FP64
// R^T(ij, ab) = sum_cd t(ij, cd) <cd|v|ab>, restricted pairs (1/2 sum over ordered cd of a
// pair-antisymmetric product = sum over c<d).  One CTA per work item (channel, 32 pp
// columns); its 8 warps split the cd range, lane = column, so each warp streams coalesced
// rows of the symmetric V block.  hh rows go in groups of 8 staged in shared memory; the 8
// partial sums per output are added in a fixed order (deterministic).  Element arithmetic is
// that of Arith<T_>: FP64, or FP32 pairs (V split once per context, the staged amplitudes
// split on the way into shared memory, FP64 result).
constexpr int PP64_COLS = 32, PP64_WARPS = 8, PP64_ROWS = 8;
static size_t pp64_smem(int npp) {
  return sizeof(double) * ((size_t)PP64_ROWS * npp + PP64_WARPS * PP64_ROWS * 32);
}

template <typename T_>
__global__ void __launch_bounds__(PP64_WARPS * 32) k_pp(DevState D, const LoopCtl* __restrict__ ctl,
                                                        const int2* __restrict__ items, int rep_only,
                                                        const T_* __restrict__ vpp) {
  using A = Arith<T_>;
  extern __shared__ __align__(16) unsigned char smpp[];  // ts[PP64_ROWS][npp], red[PP64_WARPS][PP64_ROWS][32]
  int2 it = items[blockIdx.x];
  int c = it.x, ab0 = it.y;
  if (sys_done(D, ctl, D.ch_sys[c])) return;
  // rep_only: the rows the updates compute (the list upd_row), else every hole pair
  const int* __restrict__ rows = rep_only ? D.upd_row + D.ch_uoff[c] : nullptr;
  int npp = D.ch_npp[c], nh = rep_only ? D.ch_uoff[c + 1] - D.ch_uoff[c] : D.ch_nhh[c];
  long tb = D.ch_t_off[c];
  // the ladder-basis amplitudes (FP64, or FP32 pairs in the same 8-byte slots)
  const T_* __restrict__ t = reinterpret_cast<const T_*>(cur_t(D, ctl));
  T_* ts = reinterpret_cast<T_*>(smpp);
  T_* red = ts + PP64_ROWS * npp;
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int ab = ab0 + lane;
  bool col = ab < npp;
  int chunk = (npp + PP64_WARPS - 1) / PP64_WARPS;
  int lo = warp * chunk, hi = min(npp, lo + chunk);
  const T_* __restrict__ V = vpp + D.ch_vpp_off[c] + (col ? ab : 0);
  for (int g0 = 0; g0 < nh; g0 += PP64_ROWS) {
    int nr = min(PP64_ROWS, nh - g0);
    __syncthreads();
    for (int e = threadIdx.x; e < nr * npp; e += blockDim.x) {
      int g = g0 + e / npp;
      ts[e] = t[tb + (long)(rows ? rows[g] : g) * npp + e % npp];
    }
    __syncthreads();
    T_ acc[PP64_ROWS];
#pragma unroll
    for (int r = 0; r < PP64_ROWS; r++) acc[r] = A::zero();
    if (col) {
      int cd = lo;
      for (; cd + 4 <= hi; cd += 4) {
        T_ v0 = V[(long)cd * npp], v1 = V[(long)(cd + 1) * npp];
        T_ v2 = V[(long)(cd + 2) * npp], v3 = V[(long)(cd + 3) * npp];
#pragma unroll
        for (int r = 0; r < PP64_ROWS; r++) {
          if (r < nr) {
            const T_* tr = ts + r * npp + cd;
            A::mac(acc[r], tr[0], v0);
            A::mac(acc[r], tr[1], v1);
            A::mac(acc[r], tr[2], v2);
            A::mac(acc[r], tr[3], v3);
          }
        }
      }
      for (; cd < hi; cd++) {
        T_ v0 = V[(long)cd * npp];
#pragma unroll
        for (int r = 0; r < PP64_ROWS; r++)
          if (r < nr) A::mac(acc[r], ts[r * npp + cd], v0);
      }
    }
#pragma unroll
    for (int r = 0; r < PP64_ROWS; r++) red[(warp * PP64_ROWS + r) * 32 + lane] = acc[r];
    __syncthreads();
    if ((int)threadIdx.x < nr * 32) {
      int r = threadIdx.x >> 5, l = threadIdx.x & 31;
      T_ s = A::zero();
#pragma unroll
      for (int w = 0; w < PP64_WARPS; w++) s = A::add(s, red[(w * PP64_ROWS + r) * 32 + l]);
      if (ab0 + l < npp)
        reinterpret_cast<typename A::Out*>(D.rpp)[tb + (long)(rows ? rows[g0 + r] : g0 + r) * npp + ab0 + l] = A::out(s);
    }
  }
}

// W in the ladder basis split into FP32 pairs (the refinement sweeps' copy of v_pppp).
__global__ void k_split_f2(const double* __restrict__ a, f2* __restrict__ b, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = Arith<f2>::from_double(a[i]);
}

void pnm_split_f2(const double* a, f2* b, long n, cudaStream_t s) {
  if (n > 0) k_split_f2<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, b, n);
}

// ----------------------------------------------------------------------- finalize
// End of one update: energy (Eq. ccdcorr, sum of v t over restricted amplitudes) and
// residual norm per system from the block partials in a fixed order, the |dE| test, the
// energy history, and the loop condition of the device-side loop.
__device__ void finalize_systems(const FinArgs& f, LoopCtl* ctl) {
  __shared__ double sh32f[32];
  __shared__ int all_done, bad;
  if (threadIdx.x == 0) {
    all_done = 1;
    bad = 0;
  }
  __syncthreads();
  for (int s = 0; s < f.nsys; s++) {
    double e = 0.0, r = 0.0;
    for (int k = f.lo[s] + threadIdx.x; k < f.hi[s]; k += blockDim.x) {
      e += __ldcg(f.eparts + k);
      r += __ldcg(f.rparts + k);
    }
    e = block_sum(e, sh32f);
    r = block_sum(r, sh32f);
    if (threadIdx.x == 0) {
      SysCtl& S = f.sc[s];
      if (!S.done) {
        S.iters += 1;
        S.e_new = e;
        S.resid = sqrt(r);
        if (S.iters < f.hist_cap) f.hist[(long)s * f.hist_cap + S.iters] = e;
        double diff = fabs(e - S.e_old);
        S.e_old = e;
        S.grow = (diff > 2.0 * S.d_old && diff > S.tol) ? S.grow + 1 : 0;
        S.d_old = diff;
        if (!isfinite(e) || !isfinite(r) || S.grow >= PNM_DIVERGE_STEPS) bad = 1;
        if (diff < S.tol && ctl->iter + 1 >= ctl->min_iter) {
          S.done = 1;
          S.frozen_at = ctl->iter;
        }
      }
      if (!S.done) all_done = 0;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ctl->iter += 1;
    int cont = 1;
    if (ctl->dev_error) {
      ctl->status = PNM_ETIMEOUT;
      cont = 0;
    } else if (bad) {
      ctl->status = PNM_EDIVERGED;
      cont = 0;
    } else if (all_done) {
      ctl->status = 1;
      cont = 0;
    } else if (ctl->iter >= ctl->max_iter) {
      ctl->status = PNM_ENOTCONV;
      cont = 0;
    }
    if (f.use_cond) cudaGraphSetConditional(f.handle, cont ? 1u : 0u);
  }
}

// The last block of a grid to finish runs the finalize step (no waiting: the blocks count
// themselves out with an atomic after a fence, as in the CUDA threadfence reduction).
__device__ void last_block_finalize(const FinArgs& f, LoopCtl* ctl) {
  // only thread 0 wrote the block's partials: its fence orders them before the count
  __shared__ int is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = (atomicAdd(&ctl->blocks_done, 1) == (int)gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  finalize_systems(f, ctl);
  if (threadIdx.x == 0) ctl->blocks_done = 0;
}

// ---------------------------------------------------------------------------- update
// One CTA per item (channel, up to UPD_ROWS hole pairs ij, 128 pp columns).  Jacobi step of
// Eq. (ccd3): the bracket collects v, the non-eps parts of the one-body terms, the pp and hh
// ladders and P(ij)P(ab) Q; then t_new = bracket / eps_ij^ab and t = alpha t_new + (1 - alpha) t_old.
// The residual of the amplitude equation is R = bracket - eps_ij^ab t.  The hh ladder is
// summed in the element arithmetic of T_: FP64, or FP32 pairs from the pair copy of the
// amplitudes (the sweeps with FP32-pair contractions); everything else is FP64.
// With FP32 pairs the pp ladder, the hh ladder and the ph term arrive as pairs (the 8-byte
// slots of rpp and xq) and their sum is formed on the FP32 pipe and converted to FP64 once; the
// denominator, residual, step (alpha / eps_ij^ab prepared per solve, aw) and energy stay FP64.
template <typename T_>
__global__ void __launch_bounds__(128) k_update(DevState D, LoopCtl* __restrict__ ctl,
                                                const int4* __restrict__ items, FinArgs fa,
                                                const T_* __restrict__ tpair, const double* __restrict__ aw) {
  constexpr bool PAIR = std::is_same<T_, f2>::value;
  using A = Arith<T_>;
  // the hh-ladder factor chi_kl^ij of the item's rows: chs[kl][g], zero for rows past ng;
  // per row: its hole pair ij and d_i + d_j of the one-body term
  __shared__ T_ chs[UPD_MAX_NHH][UPD_ROWS];
  __shared__ double row_dij[UPD_ROWS];
  __shared__ int row_ij[UPD_ROWS];
  __shared__ double sh32[32];
  int4 it = items[blockIdx.x];
  int c = it.x, ng = it.w;
  int npp = D.ch_npp[c], nh = D.ch_nhh[c];
  int ab = it.z + threadIdx.x;
  bool frozen = fa.sc[D.ch_sys[c]].done != 0;
  if (sys_settled(fa.sc[D.ch_sys[c]], ctl)) {
    // converged at least two steps ago: both amplitude buffers already hold its values
    if (threadIdx.x == 0) {
      D.eparts[blockIdx.x] = 0.0;
      D.rparts[blockIdx.x] = 0.0;
    }
    last_block_finalize(fa, ctl);
    return;
  }
  bool has_vpp = D.ch_vpp[c] != 0;
  double alpha = ctl->alpha;
  const double* __restrict__ t = cur_t(D, ctl);
  double* __restrict__ tn = next_t(D, ctl);
  long base = D.ch_t_off[c];
  long vho = D.ch_vhh_off[c];
  const UpdRow* __restrict__ rt = D.upd_rowinfo + (long)blockIdx.x * UPD_ROWS;
  if ((int)threadIdx.x < UPD_ROWS) {
    const UpdRow ri = rt[threadIdx.x];
    row_ij[threadIdx.x] = ri.ij;
    row_dij[threadIdx.x] = D.dchi[ri.hx] + D.dchi[ri.hy];
  }
  // chi's columns of the item's rows from the row table (one barrier covers both)
  for (int e = threadIdx.x; e < nh * UPD_ROWS; e += blockDim.x) {
    int kl = e / UPD_ROWS, g = e % UPD_ROWS;
    chs[kl][g] = g < ng ? A::from_double(D.chi_hh[vho + (long)kl * nh + rt[g].ij]) : A::zero();
  }
  __syncthreads();
  double esum = 0.0, rsum = 0.0;
  if (ab < npp) {
    // hh ladder sum_kl t_ab^kl chi_kl^ij for all rows of the item: one pass over the t column
    T_ hs[UPD_ROWS];
#pragma unroll
    for (int g = 0; g < UPD_ROWS; g++) hs[g] = A::zero();
    if (!frozen) {
      const long col = base + ab;
      const T_* __restrict__ tc;
      if constexpr (PAIR) tc = tpair;
      else tc = t;
#pragma unroll 4
      for (int kl = 0; kl < nh; kl++) {
        const T_ tk = tc[col + (long)kl * npp];
#pragma unroll
        for (int g = 0; g < UPD_ROWS; g++) A::mac(hs[g], tk, chs[kl][g]);
      }
    }
    int2 p = D.pp_pair[D.ch_pp_off[c] + ab];
    // one-body part of the bracket: (d_a + d_b - d_i - d_j) t with d_p = chi_p - eps_p
    double da = D.dchi[p.x] + D.dchi[p.y];
#pragma unroll
    for (int g = 0; g < UPD_ROWS; g++) {
      if (g >= ng) break;
      long z = base + (long)row_ij[g] * npp + ab;
      // one amplitude of each spin-flip pair is computed (the one with the smaller index) and
      // written to both; the pair counts twice in the energy and the residual norm
      const int fc = D.fmap[z];
      const long f = (long)(fc > 0 ? fc : -fc) - 1;
      if (f < z) continue;
      const double wgt = f == z ? 1.0 : 2.0;
      double tz = t[z];
      double out = tz;
      double v = D.v_pphh[z];
      if (!frozen) {
        int4 q = D.qmap[z];
        if constexpr (PAIR) {
          // pp ladder + hh ladder + P(ij)P(ab) Q in FP32 pairs, converted once
          const f2* __restrict__ rp = reinterpret_cast<const f2*>(D.rpp);
          const f2* __restrict__ xqp = reinterpret_cast<const f2*>(D.xq);
          f2 corr = hs[g];
          if (has_vpp) {
            int sg;
            const f2 rl = rp[lad_index(D, c, row_ij[g], ab, sg)];
            corr = A::add(corr, sg > 0 ? rl : A::neg(rl));
          }
          if (q.x >= 0) corr = A::add(corr, xqp[q.x]);
          if (q.y >= 0) corr = A::sub(corr, xqp[q.y]);
          if (q.z >= 0) corr = A::sub(corr, xqp[q.z]);
          if (q.w >= 0) corr = A::add(corr, xqp[q.w]);
          const double num = fma(da - row_dij[g], tz, v) + A::to_double(corr);
          const double R = fma(-D.den[z], tz, num);  // bracket - eps_ij^ab t
          rsum = fma(wgt * R, R, rsum);
          out = fma(R, aw[z], tz);                   // t + alpha R / eps_ij^ab
        } else {
          double num = v + (da - row_dij[g]) * tz;
          if (has_vpp) {
            int sg;
            double rl = D.rpp[lad_index(D, c, row_ij[g], ab, sg)];
            num += sg > 0 ? rl : -rl;
          }
          num += A::to_double(hs[g]);
          double ph = 0.0;
          if (q.x >= 0) ph += D.xq[q.x];
          if (q.y >= 0) ph -= D.xq[q.y];
          if (q.z >= 0) ph -= D.xq[q.z];
          if (q.w >= 0) ph += D.xq[q.w];
          num += ph;
          double tnew = num * D.inv_den[z];
          double R = num - D.den[z] * tz;
          rsum += wgt * (R * R);
          out = alpha * tnew + (1.0 - alpha) * tz;
        }
      }
      tn[z] = out;
      if (f != z) tn[f] = fc > 0 ? out : -out;
      esum = fma(wgt * v, out, esum);
    }
  }
  block_sum2(esum, rsum, sh32);
  if (threadIdx.x == 0) {
    D.eparts[blockIdx.x] = esum;
    D.rparts[blockIdx.x] = rsum;
  }
  last_block_finalize(fa, ctl);
}

void launch_update64(pnm_ctx* ctx, int use_cond, cudaGraphConditionalHandle h, bool pair) {
  if (pair)
    k_update<f2><<<ctx->n_grp_items, 128, 0, ctx->stream>>>(ctx->d, ctx->ctl, ctx->grp_items,
                                                            fin_args(ctx, use_cond, h, false), ctx->t_pair,
                                                            pnm_mixed_aw(ctx));
  else
    k_update<double><<<ctx->n_grp_items, 128, 0, ctx->stream>>>(ctx->d, ctx->ctl, ctx->grp_items,
                                                                fin_args(ctx, use_cond, h, false), nullptr,
                                                                nullptr);
}

// Mixed-precision update.  One CTA per item (channel, up to UPD_ROWS hole pairs ij of the rows
// the updates compute, 128 pp columns); each thread owns one column ab and the item's rows.
//   hh ladder   sum_kl t_ab^kl chi_kl^ij in FP32 for all rows of the item from one pass over
//               the FP32 t column (chi's columns of the item's rows staged in shared memory)
//   bracket     corrections in FP32: one-body (d_a + d_b - d_i - d_j) t, pp ladder (ladder
//               layout, k-split planes summed), hh ladder, and the ph term
//               Q_ij^ab - Q_ji^ab - Q_ij^ba + Q_ji^ba gathered from the cross-channel Q (qmap)
//   T scatter   the new FP32 amplitude to its four places in the ph term's T (the positions of
//               the four Q terms, qmap; formed positions only, so the same for the amplitude
//               and its spin flip), which the next ph kernel reads row by row
//   FP64        denominator eps_a + eps_b - eps_i - eps_j, residual R = v + bracket - eps_ij^ab t,
//               step t + alpha R / eps_ij^ab (alpha / eps_ij^ab prepared per solve), energy and
//               residual partial sums; v = <ab|v|ij> regenerated from the system's interaction
//               table (bit for bit the stored element, one FP64 addition) instead of streamed
// Arrays read once per update (t, alpha / eps, flip and Q maps) and the FP64 amplitudes written
// for the next update are streamed with the evict-first policy, so that the ph term's T and Q
// (50 MB each for the held-out batch, read and written at random) and the FP32 amplitudes the
// next update's contractions read stay in L2.
// The FP64 unit of a GB300 runs at about 1/64 of its FP32 rate, so the FP64 work is held to
// eight instructions per amplitude; the new amplitude goes to t (FP64) for itself and to t32 for
// itself and, sign applied, for its spin flip.  The FP64 flips are not read before the mixed
// iteration ends (the update reads t at the amplitudes it computes only); one flip copy of the
// current buffer fills them then (pnm_flip_copy_current).  Rows go in batches of UPD_BATCH with
// all loads of a batch issued before any store (rows past ng repeat the last row and are
// discarded).
__global__ void __launch_bounds__(128, UPD_MIN_BLOCKS) k_update_mix(DevState D, LoopCtl* __restrict__ ctl,
                                                    const int4* __restrict__ items, FinArgs fa,
                                                    const float* __restrict__ rpp, const float* __restrict__ xq,
                                                    const double* __restrict__ aw, float* __restrict__ xt,
                                                    const int* __restrict__ lut_off, int nplanes, long pstride) {
  __shared__ float chs[UPD_MAX_NHH * UPD_ROWS];  // chi32[kl][ij of row g] at kl * UPD_ROWS + g
  __shared__ float row_dij[UPD_ROWS];
  __shared__ double row_eij[UPD_ROWS];
  __shared__ int row_ij[UPD_ROWS];
  __shared__ char4 row_si[UPD_ROWS], row_sj[UPD_ROWS];
  __shared__ double red[2][128];
  int4 it = items[blockIdx.x];
  int c = it.x, ng = it.w;
  int npp = D.ch_npp[c], nh = D.ch_nhh[c];
  int ab = it.z + threadIdx.x;
  const bool col = ab < npp;
  const bool has_vpp = D.ch_vpp[c] != 0;
  // the column's pair data does not depend on the rows: loaded beside the row setup
  int2 p = make_int2(0, 0);
  int lmap = 0;
  if (col) {
    p = D.pp_pair[D.ch_pp_off[c] + ab];
    if (has_vpp) lmap = D.lad_map[D.ch_pp_off[c] + ab];
  }
  const UpdRow* __restrict__ rt = D.upd_rowinfo + (long)blockIdx.x * UPD_ROWS;
  if ((int)threadIdx.x < UPD_ROWS) {
    const UpdRow ri = rt[threadIdx.x];
    row_ij[threadIdx.x] = ri.ij;
    row_dij[threadIdx.x] = D.dchi32[ri.hx] + D.dchi32[ri.hy];
    row_eij[threadIdx.x] = ri.eij;
    row_si[threadIdx.x] = ri.si;
    row_sj[threadIdx.x] = ri.sj;
  }
  float dab = 0.0f;
  double eab = 0.0;
  char4 sa = make_char4(0, 0, 0, 0), sb = sa;
  if (col) {
    dab = D.dchi32[p.x] + D.dchi32[p.y];
    eab = D.eps[p.x] + D.eps[p.y];
    sa = D.nvec[p.x];
    sb = D.nvec[p.y];
  }
  const bool frozen = fa.sc[D.ch_sys[c]].done != 0;
  if (sys_settled(fa.sc[D.ch_sys[c]], ctl)) {
    // converged at least two steps ago: both amplitude buffers already hold its values
    if (threadIdx.x == 0) {
      D.eparts[blockIdx.x] = 0.0;
      D.rparts[blockIdx.x] = 0.0;
    }
    last_block_finalize(fa, ctl);
    return;
  }
  // chi's columns of the item's rows, their indices read from the row table (no wait for the
  // row setup above: one barrier covers both)
  if (!frozen) {
    const float* __restrict__ chi = D.chi32 + D.ch_vhh_off[c];
    for (int e = threadIdx.x; e < nh * UPD_ROWS; e += blockDim.x) {
      const int kl = e / UPD_ROWS, g = e % UPD_ROWS;
      chs[e] = g < ng ? chi[(long)kl * nh + rt[g].ij] : 0.0f;
    }
  }
  __syncthreads();
  const double* __restrict__ t = cur_t(D, ctl);
  const float* __restrict__ t32 = cur_t32(D, ctl);
  double* __restrict__ tn = next_t(D, ctl);
  float* __restrict__ t32n = next_t32(D, ctl);
  const long base = D.ch_t_off[c];
  // energy and residual sums of the amplitudes whose spin flip is another amplitude (counted
  // twice) and of those that are their own flip (counted once)
  double e2 = 0.0, e1 = 0.0, r2 = 0.0, r1 = 0.0;
  if (col) {
    float hh[UPD_ROWS];
#pragma unroll
    for (int g = 0; g < UPD_ROWS; g++) hh[g] = 0.0f;
    if (!frozen) {
      const float* __restrict__ tc = t32 + base + ab;
#pragma unroll UPD_HH_UNROLL
      for (int kl = 0; kl < nh; kl++) {
        const float tk = tc[(long)kl * npp];
        const float4 c0 = *reinterpret_cast<const float4*>(chs + kl * UPD_ROWS);
        const float4 c1 = *reinterpret_cast<const float4*>(chs + kl * UPD_ROWS + 4);
        hh[0] = fmaf(tk, c0.x, hh[0]); hh[1] = fmaf(tk, c0.y, hh[1]);
        hh[2] = fmaf(tk, c0.z, hh[2]); hh[3] = fmaf(tk, c0.w, hh[3]);
        hh[4] = fmaf(tk, c1.x, hh[4]); hh[5] = fmaf(tk, c1.y, hh[5]);
        hh[6] = fmaf(tk, c1.z, hh[6]); hh[7] = fmaf(tk, c1.w, hh[7]);
      }
    }
    const double* __restrict__ lut = D.lut + lut_off[D.ch_sys[c]];
    // the pp ladder's element in the ladder layout: s_off + ij * n_lad + |m| - 1, sign of m
    long lad0 = 0;
    int nl = 0;
    bool lneg = false;
    if (has_vpp) {
      const int m = lmap;
      lneg = m < 0;
      nl = D.ch_nlad[c];
      lad0 = D.ch_s_off[c] + ((m > 0 ? m : -m) - 1);
    }
#pragma unroll
    for (int gb = 0; gb < UPD_ROWS; gb += UPD_BATCH) {
      if (gb >= ng) break;
      long z[UPD_BATCH];
      double tz[UPD_BATCH], wz[UPD_BATCH];
      int fc[UPD_BATCH];
      float t32z[UPD_BATCH], part[UPD_BATCH], qs[UPD_BATCH];
      int4 qm[UPD_BATCH];
#pragma unroll
      for (int j = 0; j < UPD_BATCH; j++) {
        const int g = min(gb + j, ng - 1);
        z[j] = base + (long)row_ij[g] * npp + ab;
        tz[j] = __ldcs(t + z[j]);
        wz[j] = __ldcs(aw + z[j]);
        fc[j] = __ldcs(D.fmap + z[j]);
        t32z[j] = t32[z[j]];
        qm[j] = __ldcs(D.qmap + z[j]);
        float rl = 0.0f;
        if (has_vpp) {
          const long zl = lad0 + (long)row_ij[g] * nl;
          for (int pl = 0; pl < nplanes; pl++) rl += rpp[pl * pstride + zl];
          if (lneg) rl = -rl;
        }
        part[j] = rl;
      }
#pragma unroll
      for (int j = 0; j < UPD_BATCH; j++) {
        // P(ij)P(ab) Q: Q_ij^ab - Q_ji^ab - Q_ij^ba + Q_ji^ba from the cross-channel layout
        const float a0 = qm[j].x >= 0 ? xq[qm[j].x] : 0.0f, a1 = qm[j].y >= 0 ? xq[qm[j].y] : 0.0f;
        const float a2 = qm[j].z >= 0 ? xq[qm[j].z] : 0.0f, a3 = qm[j].w >= 0 ? xq[qm[j].w] : 0.0f;
        qs[j] = (a0 - a1) - (a2 - a3);
      }
#pragma unroll
      for (int j = 0; j < UPD_BATCH; j++) {
        const int g = gb + j;
        if (g >= ng) break;
        // one amplitude of each spin-flip pair is computed (the smaller index) and written to both
        const long f = (long)(fc[j] > 0 ? fc[j] : -fc[j]) - 1;
        if (f < z[j]) continue;
        const double v = v_minnesota_as(sa, sb, row_si[g], row_sj[g], lut);
        double out = tz[j], R = 0.0;
        if (!frozen) {
          const float corr = (dab - row_dij[g]) * t32z[j] + (part[j] + hh[g]) + qs[j];
          R = fma(eab - row_eij[g], tz[j], v) + (double)corr;  // bracket - eps_ij^ab t
          out = fma(R, wz[j], tz[j]);
        }
        const float o32 = (float)out;
        __stcs(tn + z[j], out);
        t32n[z[j]] = o32;
        if (f != z[j]) {
          t32n[f] = fc[j] < 0 ? -o32 : o32;
          e2 = fma(v, out, e2);
          r2 = fma(R, R, r2);
        } else {
          e1 = fma(v, out, e1);
          r1 = fma(R, R, r1);
        }
        if (!frozen) {
          // the T positions of t_ij^ab, t_ji^ab, t_ij^ba, t_ji^ba (the Q positions of the same
          // amplitude; stores only, nothing waits on them)
          if (qm[j].x >= 0) xt[qm[j].x] = o32;
          if (qm[j].y >= 0) xt[qm[j].y] = -o32;
          if (qm[j].z >= 0) xt[qm[j].z] = -o32;
          if (qm[j].w >= 0) xt[qm[j].w] = o32;
        }
      }
    }
  }
  // block sums: per thread in FP64, then 128 values per sum added by one warp
  red[0][threadIdx.x] = fma(2.0, e2, e1);
  red[1][threadIdx.x] = fma(2.0, r2, r1);
  __syncthreads();
  if (threadIdx.x < 32) {
    double es = (red[0][threadIdx.x] + red[0][threadIdx.x + 32]) + (red[0][threadIdx.x + 64] + red[0][threadIdx.x + 96]);
    double rs = (red[1][threadIdx.x] + red[1][threadIdx.x + 32]) + (red[1][threadIdx.x + 64] + red[1][threadIdx.x + 96]);
    es = warp_sum(es);
    rs = warp_sum(rs);
    if (threadIdx.x == 0) {
      D.eparts[blockIdx.x] = es;
      D.rparts[blockIdx.x] = rs;
    }
  }
  last_block_finalize(fa, ctl);
}

void launch_update_mix(pnm_ctx* ctx, const float* rpp, const float* xq, const double* aw, float* xt, int use_cond,
                       cudaGraphConditionalHandle h, int nplanes, long pstride) {
  k_update_mix<<<ctx->n_grp_items, 128, 0, ctx->stream>>>(ctx->d, ctx->ctl, ctx->grp_items,
                                                         fin_args(ctx, use_cond, h, false), rpp, xq, aw, xt,
                                                         ctx->lut_off_d, nplanes, pstride);
}

// alpha / eps_ij^ab per amplitude (the step of the mixed update).
__global__ void k_alpha_inv(const double* __restrict__ inv_den, double alpha, long n, double* __restrict__ aw) {
  long z = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (z < n) aw[z] = alpha * inv_den[z];
}

void pnm_alpha_inv(pnm_ctx* ctx, double alpha, double* aw) {
  if (ctx->nt > 0)
    k_alpha_inv<<<(unsigned)((ctx->nt + 255) / 256), 256, 0, ctx->stream>>>(ctx->d.inv_den, alpha, ctx->nt, aw);
  CUDA_TRY(cudaGetLastError());
}

// Per row (channel, ij) of the amplitudes: 2 if the spin flip maps it onto a later row (it is
// computed by the updates), 0 onto an earlier one (written by that row's update), 1 onto
// itself (its columns are paired among themselves).
__global__ void k_row_mode(DevState D, int nrows, int* __restrict__ mode) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  int2 it = D.row_item[r];
  int npp = D.ch_npp[it.x];
  long z0 = D.ch_t_off[it.x] + (long)it.y * npp;
  int cd = D.fmap[z0];
  long f0 = (long)(cd > 0 ? cd : -cd) - 1;
  mode[r] = (f0 >= z0 && f0 < z0 + npp) ? 1 : (f0 > z0 ? 2 : 0);
}

// t <- (t + F t) / 2 under the global spin flip F (fmap).  The solution is flip-symmetric
// and the ph term is formed for flip-symmetric amplitudes, so kept and learned starts are
// symmetrised first (MBPT2 and zero starts are symmetric already).  A pair (z, F z) is handled
// by the thread of its smaller index; fmap is an involution.
__global__ void k_flip_sym(const int* __restrict__ fmap, double* __restrict__ t, long n) {
  long z = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= n) return;
  int cd = fmap[z];
  long f = (long)(cd > 0 ? cd : -cd) - 1;
  if (f < z) return;
  double v = 0.5 * (t[z] + (cd > 0 ? t[f] : -t[f]));
  t[z] = v;
  if (f != z) t[f] = cd > 0 ? v : -v;
}

// t(F z) <- sign * t(z) for every z that comes before its flip (a start computed on the rows
// the updates compute, made flip-symmetric).
__global__ void k_flip_copy(const int* __restrict__ fmap, double* __restrict__ t, long n) {
  long z = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= n) return;
  int cd = fmap[z];
  long f = (long)(cd > 0 ? cd : -cd) - 1;
  if (f > z) t[f] = cd > 0 ? t[z] : -t[z];
}

void pnm_flip_copy(pnm_ctx* ctx, double* t, cudaStream_t s) {
  if (ctx->nt > 0)
    k_flip_copy<<<(unsigned)((ctx->nt + 255) / 256), 256, 0, s>>>(ctx->d.fmap, t, ctx->nt);
}

// The spin flips of the current FP64 amplitudes (t[iter & 1]) from the amplitudes the updates
// compute, after a mixed-precision iteration (whose updates write the FP64 values of the
// computed amplitudes only).
void pnm_flip_copy_current(pnm_ctx* ctx, int iter) {
  pnm_flip_copy(ctx, (iter & 1) ? ctx->d.t1 : ctx->d.t0, ctx->stream);
  CUDA_TRY(cudaGetLastError());
}

void pnm_flip_symmetrise(pnm_ctx* ctx, double* t, cudaStream_t s) {
  if (ctx->nt > 0)
    k_flip_sym<<<(unsigned)((ctx->nt + 255) / 256), 256, 0, s>>>(ctx->d.fmap, t, ctx->nt);
}

// Initial amplitudes (MBPT2 guess or zero) into t0 with energy partials.
__global__ void __launch_bounds__(128) k_init(DevState D, int init) {
  __shared__ double sh32[32];
  int2 it = D.row_item[blockIdx.x];
  int c = it.x, ij = it.y;
  int npp = D.ch_npp[c];
  long row = D.ch_t_off[c] + (long)ij * npp;
  int2 h = D.hh_pair[D.ch_hh_off[c] + ij];
  double ei = D.eps[h.x], ej = D.eps[h.y];
  double esum = 0.0;
  for (int ab = threadIdx.x; ab < npp; ab += blockDim.x) {
    long z = row + ab;
    double v = D.v_pphh[z];
    double t;
    if (init == PNM_INIT_MBPT2) {
      int2 p = D.pp_pair[D.ch_pp_off[c] + ab];
      t = v / (ei + ej - D.eps[p.x] - D.eps[p.y]);
      D.t0[z] = t;
    } else if (init == PNM_INIT_ZERO) {
      t = 0.0;
      D.t0[z] = t;
    } else {
      t = D.t0[z];
    }
    esum += v * t;
  }
  esum = block_sum(esum, sh32);
  if (threadIdx.x == 0) {
    D.eparts[blockIdx.x] = esum;
    D.rparts[blockIdx.x] = 0.0;
  }
}

// MBPT2 with v generated on the fly: sum over restricted pairs of v^2 / eps_ij^ab.
__global__ void __launch_bounds__(128) k_mbpt2(DevState D, const int* __restrict__ row_lut_off) {
  __shared__ double sh32[32];
  int2 it = D.row_item[blockIdx.x];
  int c = it.x, ij = it.y;
  int npp = D.ch_npp[c];
  const double* lut = D.lut + row_lut_off[D.ch_sys[c]];
  int2 h = D.hh_pair[D.ch_hh_off[c] + ij];
  char4 si = D.nvec[h.x], sj = D.nvec[h.y];
  double ei = D.eps[h.x], ej = D.eps[h.y];
  double s = 0.0;
  for (int ab = threadIdx.x; ab < npp; ab += blockDim.x) {
    int2 p = D.pp_pair[D.ch_pp_off[c] + ab];
    double v = v_minnesota_as(D.nvec[p.x], D.nvec[p.y], si, sj, lut);
    s += v * v / (ei + ej - D.eps[p.x] - D.eps[p.y]);
  }
  s = block_sum(s, sh32);
  if (threadIdx.x == 0) D.eparts[blockIdx.x] = s;
}

// Sum of row partials per system (fixed order), into out[sys].
__global__ void k_reduce_rows(const double* __restrict__ parts, const int* __restrict__ row_lo,
                              const int* __restrict__ row_hi, double* __restrict__ out) {
  __shared__ double sh32[32];
  int s = blockIdx.x;
  double acc = 0.0;
  for (int r = row_lo[s] + threadIdx.x; r < row_hi[s]; r += blockDim.x) acc += parts[r];
  acc = block_sum(acc, sh32);
  if (threadIdx.x == 0) out[s] = acc;
}

// Energy of the start amplitudes: history[0] per system, reset of the loop state.
__global__ void k_start(const double* __restrict__ parts, const int* __restrict__ row_lo,
                        const int* __restrict__ row_hi, int nsys, SysCtl* __restrict__ sc,
                        LoopCtl* __restrict__ ctl, double* __restrict__ hist, int hist_cap) {
  __shared__ double sh32[32];
  for (int s = 0; s < nsys; s++) {
    double acc = 0.0;
    for (int r = row_lo[s] + threadIdx.x; r < row_hi[s]; r += blockDim.x) acc += parts[r];
    acc = block_sum(acc, sh32);
    if (threadIdx.x == 0) {
      sc[s].e_old = acc;
      sc[s].e_new = acc;
      sc[s].resid = 0.0;
      sc[s].done = 0;
      sc[s].iters = 0;
      hist[(long)s * hist_cap] = acc;
    }
  }
  if (threadIdx.x == 0) {
    ctl->iter = 0;
    ctl->status = 0;
    ctl->blocks_done = 0;
    ctl->dev_error = 0;
  }
}

// ------------------------------------------------------------------------- host side

static void* dmalloc(pnm_ctx* ctx, size_t bytes) { return pnm_ctx_alloc(ctx, bytes); }

// Static row data of the update items: row g of item i is the (min(g, ng - 1))-th row of its run.
__global__ void k_rowinfo(DevState D, const int4* __restrict__ items, UpdRow* __restrict__ out) {
  const int g = threadIdx.x;
  if (g >= UPD_ROWS) return;
  const int4 it = items[blockIdx.x];
  const int c = it.x, ij = D.upd_row[it.y + min(g, it.w - 1)];
  const int2 h = D.hh_pair[D.ch_hh_off[c] + ij];
  UpdRow r;
  r.ij = ij;
  r.hx = h.x;
  r.hy = h.y;
  r.pad = 0;
  r.si = D.nvec[h.x];
  r.sj = D.nvec[h.y];
  r.eij = D.eps[h.x] + D.eps[h.y];
  out[(long)blockIdx.x * UPD_ROWS + g] = r;
}

void pnm_prepare_iteration(pnm_ctx* ctx) {
  cudaStream_t s = ctx->stream;
  int nsys = (int)ctx->sys.size();
  // per-system row ranges and LUT offsets
  std::vector<int> lo(nsys), hi(nsys), lut(nsys);
  for (int k = 0; k < nsys; k++) {
    lo[k] = ctx->sys[k].row_begin;
    hi[k] = ctx->sys[k].row_end;
    lut[k] = ctx->sys[k].lut_off;
  }
  int* d = (int*)dmalloc(ctx, sizeof(int) * 3 * nsys);
  CUDA_TRY(cudaMemcpyAsync(d, lo.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(d + nsys, hi.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(d + 2 * nsys, lut.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, s));
  ctx->row_lo_d = d;
  ctx->row_hi_d = d + nsys;
  ctx->lut_off_d = d + 2 * nsys;
  // pp work list (channels with a V_pppp block): one item per 32 columns of the ladder basis;
  // ladder rows (channel, ij) for the gather of the ladder-basis amplitudes
  std::vector<int2> items, abit, lrows;
  std::vector<int4> upd;
  std::vector<int> ulo(nsys), uhi(nsys);
  int max_npp = 0, max_nlad = 0;
  for (int c = 0; c < ctx->nch; c++) {
    int npp = ctx->h_npp[c];
    max_npp = std::max(max_npp, npp);
    for (int ab0 = 0; ab0 < npp; ab0 += 128) abit.push_back(make_int2(c, ab0));
    if (!ctx->h_vpp[c]) continue;
    int nl = ctx->h_nlad[c];
    max_nlad = std::max(max_nlad, nl);
    for (int q0 = 0; q0 < nl; q0 += PP64_COLS) items.push_back(make_int2(c, q0));
    for (int ij = 0; ij < ctx->h_nhh[c]; ij++) lrows.push_back(make_int2(c, ij));
  }
  // per-row items (channel, ij, first column), 128 columns each, grouped by system (the
  // learned-start kernels); update items (channel, first ij, first column, rows) with up to
  // UPD_ROWS hole pairs each, fewer when the grid would not fill the GPU
  for (int k = 0; k < nsys; k++) {
    ulo[k] = (int)upd.size();
    for (int r = ctx->sys[k].row_begin; r < ctx->sys[k].row_end; r++) {
      int2 row = ctx->h_rows[r];
      for (int ab0 = 0; ab0 < ctx->h_npp[row.x]; ab0 += 128) upd.push_back(make_int4(row.x, row.y, ab0, 0));
    }
    uhi[k] = (int)upd.size();
  }
  int dev = 0, nsm = 148;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // rows the updates compute: of two rows that the spin flip maps onto each other the one
  // whose amplitudes come first, and the rows it maps onto themselves (half of their
  // columns); per channel a run of the list upd_row, which update items index
  std::vector<int> rmode(ctx->nrows, 2);
  if (ctx->nrows > 0) {
    int* dm = (int*)dmalloc(ctx, sizeof(int) * ctx->nrows);
    k_row_mode<<<(ctx->nrows + 255) / 256, 256, 0, s>>>(ctx->d, ctx->nrows, dm);
    CUDA_TRY(cudaMemcpyAsync(rmode.data(), dm, sizeof(int) * ctx->nrows, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  ctx->h_row_mode = rmode;
  std::vector<int> urow, uoff(ctx->nch + 1, 0), ucnt(ctx->nch, 0);
  for (int r = 0; r < ctx->nrows; r++)
    if (rmode[r]) ucnt[ctx->h_rows[r].x]++;
  for (int c = 0; c < ctx->nch; c++) uoff[c + 1] = uoff[c] + ucnt[c];
  urow.resize(uoff[ctx->nch]);
  std::fill(ucnt.begin(), ucnt.end(), 0);
  for (int r = 0; r < ctx->nrows; r++)
    if (rmode[r]) {
      int c = ctx->h_rows[r].x;
      urow[uoff[c] + ucnt[c]++] = ctx->h_rows[r].y;
    }
  ctx->d.upd_row = (int*)dmalloc(ctx, sizeof(int) * std::max<size_t>(1, urow.size()));
  if (!urow.empty())
    CUDA_TRY(cudaMemcpyAsync(ctx->d.upd_row, urow.data(), sizeof(int) * urow.size(), cudaMemcpyHostToDevice, s));
  ctx->d.ch_uoff = (int*)dmalloc(ctx, sizeof(int) * (ctx->nch + 1));
  CUDA_TRY(cudaMemcpyAsync(ctx->d.ch_uoff, uoff.data(), sizeof(int) * (ctx->nch + 1), cudaMemcpyHostToDevice, s));
  auto group_items = [&](int G, std::vector<int4>* out, std::vector<int>* glo, std::vector<int>* ghi) {
    size_t n = 0;
    for (int k = 0; k < nsys; k++) {
      if (glo) (*glo)[k] = (int)(out ? out->size() : n);
      for (int c = ctx->sys[k].ch_begin; c < ctx->sys[k].ch_end; c++) {
        int nr = uoff[c + 1] - uoff[c], np = ctx->h_npp[c];
        for (int r0 = 0; r0 < nr; r0 += G)
          for (int ab0 = 0; ab0 < np; ab0 += 128) {
            if (out) out->push_back(make_int4(c, uoff[c] + r0, ab0, std::min(G, nr - r0)));
            n++;
          }
      }
      if (ghi) (*ghi)[k] = (int)(out ? out->size() : n);
    }
    return n;
  };
  int G = UPD_ROWS;
  while (G > 1 && group_items(G, nullptr, nullptr, nullptr) < (size_t)8 * nsm) G >>= 1;
  std::vector<int4> grp;
  std::vector<int> glo(nsys), ghi(nsys);
  group_items(G, &grp, &glo, &ghi);
  // static row data of every update item, filled on the device (pairs and energies live there)
  ctx->d.upd_rowinfo = (UpdRow*)dmalloc(ctx, sizeof(UpdRow) * UPD_ROWS * std::max<size_t>(1, grp.size()));
  ctx->upd_rows = G;
  ctx->max_npp = max_npp;
  ctx->max_nlad = max_nlad;
  ctx->n_lad_rows = (int)lrows.size();
  ctx->lad_rows = (int2*)dmalloc(ctx, sizeof(int2) * std::max<size_t>(1, lrows.size()));
  if (!lrows.empty())
    CUDA_TRY(cudaMemcpyAsync(ctx->lad_rows, lrows.data(), sizeof(int2) * lrows.size(), cudaMemcpyHostToDevice, s));
  ctx->n_pp_items = (int)items.size();
  ctx->pp_items = (int2*)dmalloc(ctx, sizeof(int2) * std::max<size_t>(1, items.size()));
  if (!items.empty())
    CUDA_TRY(cudaMemcpyAsync(ctx->pp_items, items.data(), sizeof(int2) * items.size(),
                             cudaMemcpyHostToDevice, s));
  std::vector<int> alo(nsys), ahi(nsys);
  int max_nhh = 1;
  for (size_t k = 0; k < abit.size(); k++) max_nhh = std::max(max_nhh, ctx->h_nhh[abit[k].x]);
  for (int k = 0; k < nsys; k++) {
    alo[k] = (int)abit.size();
    ahi[k] = 0;
  }
  for (size_t k = 0; k < abit.size(); k++) {
    int sy = ctx->h_ch_sys[abit[k].x];
    alo[sy] = std::min(alo[sy], (int)k);
    ahi[sy] = std::max(ahi[sy], (int)k + 1);
  }
  for (int k = 0; k < nsys; k++)
    if (ahi[k] == 0) alo[k] = 0;
  ctx->max_nhh = max_nhh;
  if (max_nhh > UPD_MAX_NHH) throw PnmError{PNM_EINVAL, "more hole pairs in one channel than the update supports"};
  int* ad = (int*)dmalloc(ctx, sizeof(int) * 2 * nsys);
  CUDA_TRY(cudaMemcpyAsync(ad, alo.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(ad + nsys, ahi.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, s));
  ctx->ab_lo_d = ad;
  ctx->ab_hi_d = ad + nsys;
  ctx->n_ab_items = (int)abit.size();
  ctx->ab_items = (int2*)dmalloc(ctx, sizeof(int2) * std::max<size_t>(1, abit.size()));
  if (!abit.empty())
    CUDA_TRY(cudaMemcpyAsync(ctx->ab_items, abit.data(), sizeof(int2) * abit.size(),
                             cudaMemcpyHostToDevice, s));
  ctx->n_upd_items = (int)upd.size();
  ctx->upd_items = (int4*)dmalloc(ctx, sizeof(int4) * std::max<size_t>(1, upd.size()));
  if (!upd.empty())
    CUDA_TRY(cudaMemcpyAsync(ctx->upd_items, upd.data(), sizeof(int4) * upd.size(),
                             cudaMemcpyHostToDevice, s));
  int* ud = (int*)dmalloc(ctx, sizeof(int) * 2 * nsys);
  CUDA_TRY(cudaMemcpyAsync(ud, ulo.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(ud + nsys, uhi.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, s));
  ctx->upd_lo_d = ud;
  ctx->upd_hi_d = ud + nsys;
  ctx->n_grp_items = (int)grp.size();
  ctx->grp_items = (int4*)dmalloc(ctx, sizeof(int4) * std::max<size_t>(1, grp.size()));
  if (!grp.empty()) {
    CUDA_TRY(cudaMemcpyAsync(ctx->grp_items, grp.data(), sizeof(int4) * grp.size(),
                             cudaMemcpyHostToDevice, s));
    k_rowinfo<<<(unsigned)grp.size(), 32, 0, s>>>(ctx->d, ctx->grp_items, ctx->d.upd_rowinfo);
    CUDA_TRY(cudaGetLastError());
  }
  int* gd = (int*)dmalloc(ctx, sizeof(int) * 2 * nsys);
  CUDA_TRY(cudaMemcpyAsync(gd, glo.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(gd + nsys, ghi.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, s));
  ctx->grp_lo_d = gd;
  ctx->grp_hi_d = gd + nsys;
  // partial sums: one per update item (at least one per row for init/MBPT2)
  size_t nparts = std::max<size_t>(upd.size(), (size_t)ctx->nrows);
  ctx->d.eparts = (double*)dmalloc(ctx, sizeof(double) * nparts);
  ctx->d.rparts = (double*)dmalloc(ctx, sizeof(double) * nparts);
  int mx = 0;
  for (int x = 0; x < ctx->nx; x++) mx = std::max(mx, std::max(ctx->h_x_nph[x], ctx->h_x_nhp[x]));
  ctx->max_x_dim = mx;
  ctx->ctl = (LoopCtl*)dmalloc(ctx, sizeof(LoopCtl));
  CUDA_TRY(cudaMemsetAsync(ctx->ctl, 0, sizeof(LoopCtl), s));
  ctx->small = (double*)dmalloc(ctx, sizeof(double) * 8);
  ctx->sysctl = (SysCtl*)dmalloc(ctx, sizeof(SysCtl) * nsys);
  CUDA_TRY(cudaMemsetAsync(ctx->sysctl, 0, sizeof(SysCtl) * nsys, s));
  ctx->d.sysctl = ctx->sysctl;
  // cross channels of the ph launch: S_z >= 0 (S_z < 0 ones are read at their flips), costliest first;
  // shared memory for the largest (NM = 1: rows/columns; NM = 2: those of the halves, twice)
  // CTA per channel in three size classes (larger than PH_SMALL_DIM: k_ph_big; larger than
  // PH_MID_DIM; the rest), warp per channel (at most PH_WARP_DIM)
  std::vector<int> xb, xm, xl, xw;
  std::vector<long> xcost(ctx->nx, 0);
  for (int x = 0; x < ctx->nx; x++) {
    int c = ctx->h_x_cls[x];
    if (c < 0) continue;
    long ph = ctx->h_x_nph[x], hp = ctx->h_x_nhp[x];
    int d = (int)std::max(ph, hp);
    if (c == 0) {
      d /= 2;
      xcost[x] = ph * hp * hp / 4;
    } else {
      xcost[x] = ph * hp * hp;
    }
    if (d <= PH_WARP_DIM) {
      xw.push_back(x);
      continue;
    }
    int nm = c == 0 ? 2 : 1;
    if (d > PH_SMALL_DIM) {
      ctx->ph_big_smem64 = std::max(ctx->ph_big_smem64, ph_smem_bytes(d, nm, sizeof(double)));
      ctx->ph_big_smem32 = std::max(ctx->ph_big_smem32, ph_smem_bytes(d, nm, sizeof(float)));
      xb.push_back(x);
    } else if (d > PH_MID_DIM) {
      ctx->ph_mid_smem64 = std::max(ctx->ph_mid_smem64, ph_smem_bytes(d, nm, sizeof(double)));
      ctx->ph_mid_smem32 = std::max(ctx->ph_mid_smem32, ph_smem_bytes(d, nm, sizeof(float)));
      xm.push_back(x);
    } else {
      ctx->ph_smem64 = std::max(ctx->ph_smem64, ph_smem_bytes(d, nm, sizeof(double)));
      ctx->ph_smem32 = std::max(ctx->ph_smem32, ph_smem_bytes(d, nm, sizeof(float)));
      xl.push_back(x);
    }
  }
  auto costlier = [&](int a, int b) { return xcost[a] != xcost[b] ? xcost[a] > xcost[b] : a < b; };
  std::sort(xb.begin(), xb.end(), costlier);
  std::sort(xm.begin(), xm.end(), costlier);
  std::sort(xl.begin(), xl.end(), costlier);
  std::sort(xw.begin(), xw.end(), costlier);
  ctx->n_ph_big = (int)xb.size();
  ctx->n_ph_mid = (int)xm.size();
  ctx->n_ph = (int)xl.size();
  ctx->n_ph_warp = (int)xw.size();
  // list order: big, middle, small, warp
  xl.insert(xl.end(), xw.begin(), xw.end());
  xl.insert(xl.begin(), xm.begin(), xm.end());
  xl.insert(xl.begin(), xb.begin(), xb.end());
  size_t ph_smem = std::max(std::max(ctx->ph_smem64, ctx->ph_mid_smem64), ctx->ph_big_smem64);
  ctx->ph_list = (int*)dmalloc(ctx, sizeof(int) * std::max<size_t>(1, xl.size()));
  if (!xl.empty())
    CUDA_TRY(cudaMemcpyAsync(ctx->ph_list, xl.data(), sizeof(int) * xl.size(), cudaMemcpyHostToDevice, s));
  size_t pp_smem = pp64_smem(max_nlad);
  if (ph_smem > 227 * 1024 || pp_smem > 227 * 1024)
    throw PnmError{PNM_EINVAL, "channel too large for the shared-memory tiles"};
  pnm_ph_attributes(ctx);
  for (int k = 0; k < 2; k++) {
    CUDA_TRY(cudaStreamCreateWithFlags(&ctx->side[k], cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_join[k], cudaEventDisableTiming));
  }
  CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
  smem_at_least(k_pp<double>, pp_smem);
  smem_at_least(k_pp<f2>, pp_smem);
  CUDA_TRY(cudaStreamSynchronize(s));
}

void pnm_eref_all(pnm_ctx* ctx) {
  // E_ref = sum_i h0_ii + 1/2 sum_ij <ij|v|ij>, from the HF energies:
  // sum_i eps_i = sum_i h0_ii + sum_ij <ij|v|ij>, so E_ref = 1/2 (sum_i h0_ii + sum_i eps_i).
  cudaStream_t s = ctx->stream;
  std::vector<double> ekin(ctx->nsp_total), eps(ctx->nsp_total);
  CUDA_TRY(cudaMemcpyAsync(ekin.data(), ctx->d.ekin, sizeof(double) * ctx->nsp_total,
                           cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(eps.data(), ctx->d.eps, sizeof(double) * ctx->nsp_total,
                           cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  for (auto& S : ctx->sys) {
    double a = 0, b = 0;
    for (int i = 0; i < S.N; i++) {
      a += ekin[S.sp_off + i];
      b += eps[S.sp_off + i];
    }
    S.eref = 0.5 * (a + b);
  }
}

void pnm_mbpt2_all(pnm_ctx* ctx, double* out) {
  cudaStream_t s = ctx->stream;
  int nsys = (int)ctx->sys.size();
  CUDA_TRY(cudaEventRecord(ctx->ev[0], s));
  k_mbpt2<<<ctx->nrows, 128, 0, s>>>(ctx->d, ctx->lut_off_d);
  k_reduce_rows<<<nsys, 256, 0, s>>>(ctx->d.eparts, ctx->row_lo_d, ctx->row_hi_d,
                                     ctx->d.rparts);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaEventRecord(ctx->ev[1], s));
  CUDA_TRY(cudaMemcpyAsync(out, ctx->d.rparts, sizeof(double) * nsys, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  float ms = 0;
  cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
  ctx->t_mbpt2 = ms;
}

// Third-order diagrams (Fig. goldstone, Eqs. diag3-diag5) from the MBPT2 amplitudes t0 held in
// D.t0, the pp ladder of t0 in D.rpp (channels with a V_pppp block) and the linear ph term of t0 in D.xq:
// per row (channel, ij) the partial sums over ab of
//   (4)  t0_ab^ij sum_{c<d} <ab|v|cd> t0_cd^ij,
//   (5)  t0_ab^ij sum_{k<l} t0_ab^kl <kl|v|ij>,
//   (3)  t0_ab^ij [P(ij)P(ab) sum_kc <kb|v|cj> t0_ik^ac],
// into parts[0..3) x nrows.
__global__ void __launch_bounds__(128) k_mbpt3_rows(DevState D, double* __restrict__ parts, int nrows) {
  __shared__ double sh32[32];
  int2 it = D.row_item[blockIdx.x];
  int c = it.x, ij = it.y;
  int npp = D.ch_npp[c], nh = D.ch_nhh[c];
  long base = D.ch_t_off[c], row = base + (long)ij * npp;
  const double* __restrict__ vh = D.v_hhhh + D.ch_vhh_off[c];
  const double* __restrict__ t = D.t0;
  bool has_vpp = D.ch_vpp[c] != 0;
  double e4 = 0.0, e5 = 0.0, e3 = 0.0;
  for (int ab = threadIdx.x; ab < npp; ab += blockDim.x) {
    long z = row + ab;
    // one amplitude of each spin-flip pair, counted twice (the ladder is formed on those rows)
    const int fc = D.fmap[z];
    const long f = (long)(fc > 0 ? fc : -fc) - 1;
    if (f < z) continue;
    double tz = (f == z ? 1.0 : 2.0) * t[z];
    if (has_vpp) {
      int sg;
      double rl = D.rpp[lad_index(D, c, ij, ab, sg)];
      e4 += tz * (sg > 0 ? rl : -rl);
    }
    double hh = 0.0;
    for (int kl = 0; kl < nh; kl++) hh += t[base + (long)kl * npp + ab] * vh[(long)kl * nh + ij];
    e5 += tz * hh;
    int4 q = D.qmap[z];
    double ph = 0.0;
    if (q.x >= 0) ph += D.xq[q.x];
    if (q.y >= 0) ph -= D.xq[q.y];
    if (q.z >= 0) ph -= D.xq[q.z];
    if (q.w >= 0) ph += D.xq[q.w];
    e3 += tz * ph;
  }
  e4 = block_sum(e4, sh32);
  e5 = block_sum(e5, sh32);
  e3 = block_sum(e3, sh32);
  if (threadIdx.x == 0) {
    parts[blockIdx.x] = e4;
    parts[nrows + blockIdx.x] = e5;
    parts[2 * nrows + blockIdx.x] = e3;
  }
}

// out[3 s + {0, 1, 2}] = diagrams (4), (5), (3) of system s.  Replaces the context's
// amplitudes by the MBPT2 guess.
void pnm_mbpt3_all(pnm_ctx* ctx, double* out) {
  cudaStream_t s = ctx->stream;
  pnm_need_vpp64(ctx);
  int nsys = (int)ctx->sys.size();
  if (!ctx->mbpt3_buf) ctx->mbpt3_buf = (double*)dmalloc(ctx, sizeof(double) * (3 * (size_t)ctx->nrows + 3 * nsys));
  double* parts = ctx->mbpt3_buf;
  double* res = parts + 3 * (size_t)ctx->nrows;
  CUDA_TRY(cudaEventRecord(ctx->ev[0], s));
  // amplitudes of the start in t0, read by the contraction kernels (iteration parity 0, no
  // system frozen)
  CUDA_TRY(cudaMemsetAsync(&ctx->ctl->iter, 0, sizeof(int), s));
  CUDA_TRY(cudaMemsetAsync(&ctx->ctl->skip_done, 0, sizeof(int), s));
  k_init<<<ctx->nrows, 128, 0, s>>>(ctx->d, PNM_INIT_MBPT2);
  pnm_launch_pp64(ctx, s);
  if (ctx->nx > 0) launch_ph64(ctx, s, true);  // without cross channels no Q is read
  k_mbpt3_rows<<<ctx->nrows, 128, 0, s>>>(ctx->d, parts, ctx->nrows);
  for (int k = 0; k < 3; k++)
    k_reduce_rows<<<nsys, 256, 0, s>>>(parts + (size_t)k * ctx->nrows, ctx->row_lo_d, ctx->row_hi_d,
                                       res + (size_t)k * nsys);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaEventRecord(ctx->ev[1], s));
  std::vector<double> h(3 * (size_t)nsys);
  CUDA_TRY(cudaMemcpyAsync(h.data(), res, sizeof(double) * 3 * nsys, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  for (int k = 0; k < 3; k++)
    for (int y = 0; y < nsys; y++) out[3 * y + k] = h[(size_t)k * nsys + y];
  float ms = 0;
  cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
  ctx->t_mbpt3 = ms;
}

// The MBPT2 kernels of pnm_mbpt2_all with caller-chosen device buffers for the per-row
// partial sums (nrows doubles) and the per-system results (nsys doubles).
void pnm_launch_mbpt2_into(const pnm_ctx* ctx, double* partials, double* results) {
  DevState d = ctx->d;
  d.eparts = partials;
  k_mbpt2<<<ctx->nrows, 128, 0, ctx->stream>>>(d, ctx->lut_off_d);
  k_reduce_rows<<<(int)ctx->sys.size(), 256, 0, ctx->stream>>>(partials, ctx->row_lo_d,
                                                                ctx->row_hi_d, results);
}

// The body of one update, enqueued on the context stream (FP64 path).
// per_row: partials of the per-row mixed update (items upd_items), else of the grouped update.
FinArgs fin_args(pnm_ctx* ctx, int use_cond, cudaGraphConditionalHandle h, bool per_row) {
  FinArgs f;
  f.eparts = ctx->d.eparts;
  f.rparts = ctx->d.rparts;
  f.lo = per_row ? ctx->upd_lo_d : ctx->grp_lo_d;
  f.hi = per_row ? ctx->upd_hi_d : ctx->grp_hi_d;
  f.nsys = (int)ctx->sys.size();
  f.sc = ctx->sysctl;
  f.hist = ctx->hist;
  f.hist_cap = ctx->hist_cap;
  f.use_cond = use_cond;
  f.handle = h;
  return f;
}

// The FP64 pp ladder in the ladder basis: the amplitudes gathered into it (s = sum of the
// signed members of each vector), then k_pp64 on a view of the state whose channel width is
// the basis size, whose amplitudes are s and whose V blocks are the ladder V; the result stays
// in the ladder layout (consumers read it through lad_index).
template <typename T_>
static void lad_expand(pnm_ctx* ctx, const T_* rs, int planes, long pstride, double* host_out) {
  cudaStream_t s = ctx->stream;
  if (!ctx->expand_buf) ctx->expand_buf = (double*)dmalloc(ctx, sizeof(double) * std::max<long>(ctx->nt, 1));
  if (ctx->nrows > 0)
    k_lad_expand<T_><<<ctx->nrows, 128, 0, s>>>(ctx->d, rs, planes, pstride, ctx->expand_buf);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(host_out, ctx->expand_buf, sizeof(double) * ctx->nt, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
}

void pnm_lad_expand(pnm_ctx* ctx, const float* rs, int planes, long pstride, double* host_out) {
  lad_expand(ctx, rs, planes, pstride, host_out);
}

void pnm_lad_expand(pnm_ctx* ctx, const double* rs, int planes, long pstride, double* host_out) {
  lad_expand(ctx, rs, planes, pstride, host_out);
}

void pnm_lad_expand(pnm_ctx* ctx, const f2* rs, int planes, long pstride, double* host_out) {
  lad_expand(ctx, rs, planes, pstride, host_out);
}

// rep_only: only the rows the updates compute (one of each spin-flip pair of rows); the ladder
// operator of pnm_apply_pp_ladder takes every row.
void pnm_launch_pp64(pnm_ctx* ctx, cudaStream_t s, bool rep_only, const f2* vpp_f2) {
  // the FP64 ladder V is built before any capture by the host-side callers (pnm_need_vpp64)
  if (!vpp_f2 && !ctx->d.v_pppp) throw PnmError{PNM_EINVAL, "the FP64 ladder V has not been built"};
  if (ctx->n_pp_items == 0) return;
  if (vpp_f2)
    k_lad_gather<f2><<<ctx->n_lad_rows, 128, 0, s>>>(ctx->d, ctx->ctl, ctx->lad_rows, ctx->t_pair,
                                                      reinterpret_cast<f2*>(ctx->d.s64));
  else
    k_lad_gather<double><<<ctx->n_lad_rows, 128, 0, s>>>(ctx->d, ctx->ctl, ctx->lad_rows, nullptr, ctx->d.s64);
  DevState L = ctx->d;
  L.ch_npp = ctx->d.ch_nlad;
  L.ch_t_off = ctx->d.ch_s_off;
  L.t0 = L.t1 = ctx->d.s64;
  if (vpp_f2)
    k_pp<f2><<<ctx->n_pp_items, PP64_WARPS * 32, pp64_smem(ctx->max_nlad), s>>>(L, ctx->ctl, ctx->pp_items,
                                                                                rep_only ? 1 : 0, vpp_f2);
  else
    k_pp<double><<<ctx->n_pp_items, PP64_WARPS * 32, pp64_smem(ctx->max_nlad), s>>>(L, ctx->ctl, ctx->pp_items,
                                                                                    rep_only ? 1 : 0, ctx->d.v_pppp);
}

// The ph term and the pp ladder do not depend on each other nor on the one-body sums: in a
// captured update they run on two side streams next to the stats kernels.  While kernels are
// being profiled one by one everything stays on the context stream.
bool pnm_concurrent(const pnm_ctx* ctx) {
  return !ctx->prof_live && !ctx->serial_sched[ctx->cur_mode];
}

void pnm_fork(pnm_ctx* ctx) {
  if (!pnm_concurrent(ctx)) return;
  CUDA_TRY(cudaEventRecord(ctx->ev_fork, ctx->stream));
  for (int k = 0; k < 2; k++) CUDA_TRY(cudaStreamWaitEvent(ctx->side[k], ctx->ev_fork, 0));
}

void pnm_join(pnm_ctx* ctx) {
  if (!pnm_concurrent(ctx)) return;
  for (int k = 0; k < 2; k++) {
    CUDA_TRY(cudaEventRecord(ctx->ev_join[k], ctx->side[k]));
    CUDA_TRY(cudaStreamWaitEvent(ctx->stream, ctx->ev_join[k], 0));
  }
}

// One-body intermediates and <kl|chi|ij> (shared by both precision modes, FP64).
// One-body sums, chi_hh and the one-body terms: FP64 (mixed = false) or from the FP32
// copies of the mixed-precision iteration.
void pnm_enqueue_stats(pnm_ctx* ctx, bool mixed, bool pair) {
  cudaStream_t s = ctx->stream;
  DevState& D = ctx->d;
  unsigned nb = (unsigned)(ctx->nrows + ctx->n_ab_items);
  unsigned nd = (unsigned)((ctx->nsp_total * 32 + 255) / 256);
  prof_begin(ctx, mixed ? KID_TSTATS32 : KID_TSTATS);
  if (mixed) k_tstats<float><<<nb, 128, 0, s>>>(D, ctx->ctl, ctx->nrows, ctx->ab_items);
  else if (pair)
    k_tstats<double, true><<<nb, 128, 0, s>>>(D, ctx->ctl, ctx->nrows, ctx->ab_items, ctx->t_pair,
                                             ctx->vpphh_f2);
  else k_tstats<double><<<nb, 128, 0, s>>>(D, ctx->ctl, ctx->nrows, ctx->ab_items);
  prof_end(ctx);
  prof_begin(ctx, mixed ? KID_DCHI32 : KID_DCHI);
  if (mixed) k_dchi<float><<<nd, 256, 0, s>>>(D, ctx->nsp_total);
  else k_dchi<double><<<nd, 256, 0, s>>>(D, ctx->nsp_total);
  prof_end(ctx);
}

// One FP64 update.  terms (PNM_TERMS_*): the full Eq. (ccd3), or a truncation whose
// intermediates were fixed by pnm_prepare_terms (one-body terms zero, chi_kl^ij = <kl|v|ij>
// or zero, the ph term zero unless the linear ph term is launched here).
// pair: the ph and pp contractions with FP32-pair arithmetic (full Eq. ccd3 only).
static void enqueue_body_fp64(pnm_ctx* ctx, int use_cond, cudaGraphConditionalHandle h, int terms, bool pair) {
  cudaStream_t s_ph = pnm_concurrent(ctx) ? ctx->side[0] : ctx->stream;
  cudaStream_t s_pp = pnm_concurrent(ctx) ? ctx->side[1] : ctx->stream;
  bool ph_on = terms == PNM_TERMS_FULL || terms == PNM_TERMS_LINEAR;
  if (pair) pnm_split_cur(ctx, ctx->stream);  // before the fork: both branches read it
  pnm_fork(ctx);
  if (ctx->nx > 0 && ph_on) {
    prof_begin(ctx, pair ? KID_PH_F2 : KID_PH64);
    if (pair) launch_ph_f2(ctx, ctx->t_pair, ctx->xw_f2, ctx->xv1_f2, s_ph);
    else launch_ph64(ctx, s_ph, terms == PNM_TERMS_LINEAR);
    prof_end(ctx);
  }
  if (ctx->n_pp_items > 0) {
    prof_begin(ctx, pair ? KID_PP_F2 : KID_PP64);
    pnm_launch_pp64(ctx, s_pp, true, pair ? ctx->vpp_f2 : nullptr);
    prof_end(ctx);
  }
  if (terms == PNM_TERMS_FULL) pnm_enqueue_stats(ctx, false, pair);
  pnm_join(ctx);
  prof_begin(ctx, KID_UPDATE);
  launch_update64(ctx, use_cond, h, pair);
  prof_end(ctx);
}

const char* const pnm_kernel_names[PNM_NKERNELS] = {
    "k_tstats", "k_dchi", "k_ph64", "k_pp64", "k_update", "k_finalize(unused)",
    "k_pp_tc", "k_ph32", "k_tstats32", "k_update_mix", "k_pack", "k_dchi32", "k_ph_f2", "k_pp_f2"};

void prof_begin(pnm_ctx* ctx, int kid) {
  if (!ctx->prof_live) return;
  size_t k = ctx->prof_pending.size();
  if (k >= ctx->prof_ev.size()) {
    cudaEvent_t a, b;
    CUDA_TRY(cudaEventCreate(&a));
    CUDA_TRY(cudaEventCreate(&b));
    ctx->prof_ev.push_back({a, b});
  }
  ctx->prof_pending.push_back(kid);
  CUDA_TRY(cudaEventRecord(ctx->prof_ev[k].first, ctx->stream));
}

void prof_end(pnm_ctx* ctx) {
  if (!ctx->prof_live) return;
  CUDA_TRY(cudaEventRecord(ctx->prof_ev[ctx->prof_pending.size() - 1].second, ctx->stream));
}

void prof_collect(pnm_ctx* ctx) {
  for (size_t k = 0; k < ctx->prof_pending.size(); k++) {
    float ms = 0;
    CUDA_TRY(cudaEventSynchronize(ctx->prof_ev[k].second));
    CUDA_TRY(cudaEventElapsedTime(&ms, ctx->prof_ev[k].first, ctx->prof_ev[k].second));
    ctx->prof_ms[ctx->prof_pending[k]] += ms;
    ctx->prof_n[ctx->prof_pending[k]] += 1;
  }
  ctx->prof_pending.clear();
}

// mode = precision | (terms << 4) | (pair << 8); truncations (terms != 0) are FP64 only; pair
// selects the FP32-pair contractions for an FP64 update (the refinement sweeps).
void pnm_enqueue_body(pnm_ctx* ctx, int mode, int use_cond, cudaGraphConditionalHandle h) {
  int prec = mode & 15, terms = (mode >> 4) & 15;
  bool pair = ((mode >> 8) & 1) != 0;
  ctx->cur_mode = prec == PNM_PREC_FP64 ? (pair ? 2 : 0) : 1;
  if (prec == PNM_PREC_FP64) enqueue_body_fp64(ctx, use_cond, h, terms, pair);
  else pnm_enqueue_body_mixed(ctx, use_cond, h);
}

// FP32-pair copies of the ladder-basis V_pppp, V_pphh, W and <kb|v|cj> (once per context).
void pnm_prepare_f2(pnm_ctx* ctx) {
  if (ctx->t_pair) return;
  cudaStream_t s = ctx->stream;
  pnm_need_vpp_f2(ctx);
  ctx->t_pair = ctx_alloc<f2>(ctx, ctx->nt);
  ctx->xw_f2 = ctx_alloc<f2>(ctx, ctx->nxt);
  ctx->xv1_f2 = ctx_alloc<f2>(ctx, ctx->nxc);
  ctx->vpphh_f2 = ctx_alloc<f2>(ctx, ctx->nt);
  pnm_split_f2(ctx->d.v_pphh, ctx->vpphh_f2, ctx->nt, s);
  pnm_split_f2(ctx->d.x_w, ctx->xw_f2, ctx->nxt, s);
  pnm_split_f2(ctx->d.x_v1, ctx->xv1_f2, ctx->nxc, s);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(s));
}

// Fixed intermediates of a truncated iteration: no one-body terms, chi_kl^ij = <kl|v|ij>
// (hh ladder with the bare interaction) or zero (no hh ladder), and no ph term unless the
// linear one is recomputed every step.
void pnm_prepare_terms(pnm_ctx* ctx, int terms) {
  if (terms == PNM_TERMS_FULL) return;
  cudaStream_t s = ctx->stream;
  CUDA_TRY(cudaMemsetAsync(ctx->d.dchi, 0, sizeof(double) * ctx->nsp_total, s));
  if (terms == PNM_TERMS_PP) CUDA_TRY(cudaMemsetAsync(ctx->d.chi_hh, 0, sizeof(double) * ctx->nvhh, s));
  else CUDA_TRY(cudaMemcpyAsync(ctx->d.chi_hh, ctx->d.v_hhhh, sizeof(double) * ctx->nvhh,
                                cudaMemcpyDeviceToDevice, s));
  if (terms != PNM_TERMS_LINEAR && ctx->nxt > 0)
    CUDA_TRY(cudaMemsetAsync(ctx->d.xq, 0, sizeof(double) * ctx->nxt, s));
}

// Kernel nodes of a captured update: the ph term at the lowest priority, every other kernel at
// the highest, so that the shorter branches (pp ladder, one-body sums) are dispatched ahead of
// the many ph CTAs and run beside them instead of after them.
static bool is_ph_kernel(const void* f) {
  return f == (const void*)k_ph<double, PH_THREADS, 2> || f == (const void*)k_ph<float, PH_THREADS, ph_tile<float>()> ||
         f == (const void*)k_ph<f2, PH_THREADS, 2> || f == (const void*)k_ph_big<double, 2> ||
         f == (const void*)k_ph_big<float, ph_tile<float>()> || f == (const void*)k_ph_big<f2, 2>;
}

void pnm_set_node_priorities(cudaGraph_t body) {
  int least = 0, greatest = 0;
  CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  size_t n = 0;
  CUDA_TRY(cudaGraphGetNodes(body, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  if (n) CUDA_TRY(cudaGraphGetNodes(body, nodes.data(), &n));
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    CUDA_TRY(cudaGraphNodeGetType(nd, &t));
    if (t != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams kp = {};
    CUDA_TRY(cudaGraphKernelNodeGetParams(nd, &kp));
    cudaKernelNodeAttrValue v = {};
    v.priority = is_ph_kernel(kp.func) ? least : greatest;
    CUDA_TRY(cudaGraphKernelNodeSetAttribute(nd, cudaKernelNodeAttributePriority, &v));
  }
}

// Build (once per mode) a graph whose single node is a WHILE conditional looping the body.
static cudaGraphExec_t graph_for(pnm_ctx* ctx, int mode) {
  auto f = ctx->graphs.find(mode);
  if (f != ctx->graphs.end()) return f->second;
  const auto w0 = std::chrono::steady_clock::now();
  cudaGraph_t g;
  CUDA_TRY(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CUDA_TRY(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  CUDA_TRY(cudaStreamBeginCaptureToGraph(ctx->stream, body, nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal));
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
  cudaGraphExec_t ge;
  CUDA_TRY(cudaGraphInstantiate(&ge, g, cudaGraphInstantiateFlagUseNodePriority));
  ctx->graphs[mode] = ge;
  ctx->graph_defs[mode] = g;
  ctx->t_graph_host += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w0).count();
  return ge;
}

// Runs updates until every system meets its tolerance or the cap is hit.  Returns the
// loop status (1 converged, PNM_ENOTCONV, PNM_EDIVERGED).
int pnm_run_loop(pnm_ctx* ctx, int mode, int max_iter, int min_iter, int host_loop, double alpha, int* iter_out) {
  cudaStream_t s = ctx->stream;
  LoopCtl hc{};
  // keep iteration parity: ctl->iter is reset by k_start; only the limits, alpha and mode
  // are set here
  CUDA_TRY(cudaMemcpyAsync(&ctx->ctl->max_iter, &max_iter, sizeof(int), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(&ctx->ctl->min_iter, &min_iter, sizeof(int), cudaMemcpyHostToDevice, s));
  static const int kOne = 1, kZero = 0;
  CUDA_TRY(cudaMemcpyAsync(&ctx->ctl->alpha, &alpha, sizeof(double), cudaMemcpyHostToDevice, s));
  static const int kMode[2] = {0, 1};
  CUDA_TRY(cudaMemcpyAsync(&ctx->ctl->mode, &kMode[(mode & 15) == PNM_PREC_FP64 ? 0 : 1], sizeof(int),
                           cudaMemcpyHostToDevice, s));
  if (max_iter <= 0) return PNM_ENOTCONV;
  CUDA_TRY(cudaMemcpyAsync(&ctx->ctl->skip_done, &kOne, sizeof(int), cudaMemcpyHostToDevice, s));
  if (!host_loop) {
    cudaGraphExec_t ge = graph_for(ctx, mode);
    CUDA_TRY(cudaGraphLaunch(ge, s));
  } else {
    ctx->prof_live = ctx->prof_on;
    for (;;) {
      pnm_enqueue_body(ctx, mode, 0, 0);
      CUDA_TRY(cudaGetLastError());
      CUDA_TRY(cudaMemcpyAsync(&hc, ctx->ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaStreamSynchronize(s));
      if (ctx->prof_live) prof_collect(ctx);
      if (hc.status != 0) break;
    }
    ctx->prof_live = false;
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(&ctx->ctl->skip_done, &kZero, sizeof(int), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(&hc, ctx->ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (iter_out) *iter_out = hc.iter;
  return hc.status;
}

// Initial amplitudes and their energy; resets iteration counters.
void pnm_start(pnm_ctx* ctx, int init, const std::vector<double>& tol) {
  cudaStream_t s = ctx->stream;
  int nsys = (int)ctx->sys.size();
  std::vector<SysCtl> hs(nsys);
  for (int k = 0; k < nsys; k++) {
    hs[k] = SysCtl{};
    hs[k].tol = tol[k];
  }
  CUDA_TRY(cudaMemcpyAsync(ctx->sysctl, hs.data(), sizeof(SysCtl) * nsys, cudaMemcpyHostToDevice, s));
  if (init == PNM_INIT_KEEP) pnm_flip_symmetrise(ctx, ctx->d.t0, s);
  k_init<<<ctx->nrows, 128, 0, s>>>(ctx->d, init);
  k_start<<<1, 256, 0, s>>>(ctx->d.eparts, ctx->row_lo_d, ctx->row_hi_d, nsys, ctx->sysctl,
                            ctx->ctl, ctx->hist, ctx->hist_cap);
  CUDA_TRY(cudaGetLastError());
}

// Reopen the convergence test of every system for a further phase (refinement), keeping
// amplitudes, energies and iteration counts.
__global__ void k_reopen(SysCtl* sc, int nsys, LoopCtl* ctl) {
  for (int s = 0; s < nsys; s++) {
    sc[s].done = 0;
    sc[s].grow = 0;
  }
  ctl->status = 0;
}

void pnm_reopen(pnm_ctx* ctx) {
  k_reopen<<<1, 1, 0, ctx->stream>>>(ctx->sysctl, (int)ctx->sys.size(), ctx->ctl);
  CUDA_TRY(cudaGetLastError());
}

// Make t0 hold the latest amplitudes (the loop leaves them in t[iter & 1]).
void pnm_settle_amplitudes(pnm_ctx* ctx) {
  int it = 0;
  CUDA_TRY(cudaMemcpyAsync(&it, &ctx->ctl->iter, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (it & 1) {
    CUDA_TRY(cudaMemcpyAsync(ctx->d.t0, ctx->d.t1, sizeof(double) * ctx->nt,
                             cudaMemcpyDeviceToDevice, ctx->stream));
    int zero = 0;
    CUDA_TRY(cudaMemcpyAsync(&ctx->ctl->iter, &zero, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  }
  ctx->last_iters_host = it;
}

// ------------------------------------------------- device-side steps of a whole-solve graph
// Start of a solve: every system's control block cleared with its tolerance; kernels do not
// skip converged systems until the loop begins.
__global__ void k_solve_begin(SysCtl* __restrict__ sc, const double* __restrict__ tol, int nsys,
                              LoopCtl* __restrict__ ctl) {
  for (int k = threadIdx.x; k < nsys; k += blockDim.x) {
    SysCtl z = {};
    z.tol = tol[k];
    sc[k] = z;
  }
  if (threadIdx.x == 0) ctl->skip_done = 0;
}

// Parameters of the first iteration loop (what pnm_run_loop sets from the host).
__global__ void k_loop_begin(LoopCtl* __restrict__ ctl, const SolveParams* __restrict__ par, int mode) {
  ctl->max_iter = par->max_iter;
  ctl->min_iter = 0;
  ctl->alpha = par->alpha;
  ctl->mode = mode;
  ctl->skip_done = 1;
}

// After the mixed loop: if it converged, reopen every system for exactly refine_sweeps FP64
// updates and then the FP64 test (within max_iter more) and run the refinement loop; else
// skip it (the loop status stays the mixed loop's).
__global__ void k_refine_gate(LoopCtl* __restrict__ ctl, SysCtl* __restrict__ sc, int nsys,
                              const SolveParams* __restrict__ par, cudaGraphConditionalHandle h) {
  const bool go = ctl->status == 1;
  if (go) {
    for (int k = 0; k < nsys; k++) {
      sc[k].done = 0;
      sc[k].grow = 0;
    }
    const int it0 = ctl->iter;
    ctl->status = 0;
    ctl->max_iter = it0 + par->refine_sweeps + par->max_iter;
    ctl->min_iter = it0 + par->refine_sweeps;
    ctl->mode = 0;
  }
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void k_loop_end(LoopCtl* __restrict__ ctl) { ctl->skip_done = 0; }

// t0 = the latest amplitudes (the loop leaves them in t[iter & 1]); the iteration parity is
// reset by k_settle_reset once every block has copied.
__global__ void k_settle_copy(DevState D, const LoopCtl* __restrict__ ctl, long n) {
  if (!(ctl->iter & 1)) return;
  for (long z = (long)blockIdx.x * blockDim.x + threadIdx.x; z < n; z += (long)gridDim.x * blockDim.x)
    D.t0[z] = D.t1[z];
}
__global__ void k_settle_reset(LoopCtl* __restrict__ ctl) {
  if (ctl->iter & 1) ctl->iter = 0;
}

// The spin flips of the current FP64 amplitudes, the buffer chosen on the device.
__global__ void k_flip_copy_cur(DevState D, const LoopCtl* __restrict__ ctl, long n) {
  long z = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= n) return;
  double* t = (ctl->iter & 1) ? D.t1 : D.t0;
  int cd = D.fmap[z];
  long f = (long)(cd > 0 ? cd : -cd) - 1;
  if (f > z) t[f] = cd > 0 ? t[z] : -t[z];
}

void pnm_solve_begin(pnm_ctx* ctx) {
  k_solve_begin<<<1, 256, 0, ctx->stream>>>(ctx->sysctl, ctx->d_tol, (int)ctx->sys.size(), ctx->ctl);
  CUDA_TRY(cudaGetLastError());
}

// Initial amplitudes and their energy (the device-side pnm_start: control blocks from
// k_solve_begin).
void pnm_start_device(pnm_ctx* ctx, int init) {
  cudaStream_t s = ctx->stream;
  if (init == PNM_INIT_KEEP) pnm_flip_symmetrise(ctx, ctx->d.t0, s);
  k_init<<<ctx->nrows, 128, 0, s>>>(ctx->d, init);
  k_start<<<1, 256, 0, s>>>(ctx->d.eparts, ctx->row_lo_d, ctx->row_hi_d, (int)ctx->sys.size(), ctx->sysctl,
                            ctx->ctl, ctx->hist, ctx->hist_cap);
  CUDA_TRY(cudaGetLastError());
}

void pnm_loop_begin(pnm_ctx* ctx, int mode) {
  k_loop_begin<<<1, 1, 0, ctx->stream>>>(ctx->ctl, ctx->d_par, (mode & 15) == PNM_PREC_FP64 ? 0 : 1);
  CUDA_TRY(cudaGetLastError());
}

void pnm_refine_gate(pnm_ctx* ctx, cudaGraphConditionalHandle h) {
  k_refine_gate<<<1, 1, 0, ctx->stream>>>(ctx->ctl, ctx->sysctl, (int)ctx->sys.size(), ctx->d_par, h);
  CUDA_TRY(cudaGetLastError());
}

void pnm_loop_end_settle(pnm_ctx* ctx) {
  cudaStream_t s = ctx->stream;
  k_loop_end<<<1, 1, 0, s>>>(ctx->ctl);
  if (ctx->nt > 0) {
    const long blocks = std::min<long>((ctx->nt + 255) / 256, 4096);
    k_settle_copy<<<(unsigned)blocks, 256, 0, s>>>(ctx->d, ctx->ctl, ctx->nt);
  }
  k_settle_reset<<<1, 1, 0, s>>>(ctx->ctl);
  CUDA_TRY(cudaGetLastError());
}

void pnm_flip_copy_device(pnm_ctx* ctx) {
  if (ctx->nt > 0)
    k_flip_copy_cur<<<(unsigned)((ctx->nt + 255) / 256), 256, 0, ctx->stream>>>(ctx->d, ctx->ctl, ctx->nt);
  CUDA_TRY(cudaGetLastError());
}

// Schedule tuning: time a few updates with the ph term and the pp ladder on side streams
// (concurrent with the one-body kernels) and a few with everything on one stream; keep the
// faster for this precision mode.  The held amplitudes are saved and restored.
static std::mutex g_sched_mu;
static std::map<std::string, bool> g_sched_cache;  // (shape key, mode) -> one stream

void pnm_tune_schedule(pnm_ctx* ctx, int mode, double alpha) {
  const bool pair = ((mode >> 8) & 1) != 0;
  int m = (mode & 15) == PNM_PREC_FP64 ? (pair ? 2 : 0) : 1;
  if (ctx->sched_tuned[m]) return;
  if (m == 0) pnm_need_vpp64(ctx);
  const std::string key = pnm_shape_key(ctx) + (m == 1 ? "|mixed" : m == 2 ? "|pair" : "|fp64");
  {
    std::lock_guard<std::mutex> lock(g_sched_mu);
    auto f = g_sched_cache.find(key);
    if (f != g_sched_cache.end()) {
      ctx->serial_sched[m] = f->second;
      ctx->sched_tuned[m] = true;
      return;
    }
  }
  cudaStream_t s = ctx->stream;
  double* save = (double*)dmalloc(ctx, sizeof(double) * std::max<long>(ctx->nt, 1));
  CUDA_TRY(cudaMemcpyAsync(save, ctx->d.t0, sizeof(double) * ctx->nt, cudaMemcpyDeviceToDevice, s));
  std::vector<double> never(ctx->sys.size(), 0.0);
  int big = 1 << 30;
  CUDA_TRY(cudaMemcpyAsync(&ctx->ctl->max_iter, &big, sizeof(int), cudaMemcpyHostToDevice, s));
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_serial = 0;
  for (int serial = 0; serial < 2; serial++) {
    ctx->serial_sched[m] = serial != 0;
    CUDA_TRY(cudaMemcpyAsync(ctx->d.t0, save, sizeof(double) * ctx->nt, cudaMemcpyDeviceToDevice, s));
    pnm_start(ctx, PNM_INIT_KEEP, never);
    if (m == 1) pnm_mixed_pack_initial(ctx, alpha);
    pnm_enqueue_body(ctx, mode, 0, 0);
    CUDA_TRY(cudaEventRecord(e0, s));
    for (int k = 0; k < 4; k++) pnm_enqueue_body(ctx, mode, 0, 0);
    CUDA_TRY(cudaEventRecord(e1, s));
    CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0;
    CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) {
      best = ms;
      best_serial = serial;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->serial_sched[m] = best_serial != 0;
  ctx->sched_tuned[m] = true;
  {
    std::lock_guard<std::mutex> lock(g_sched_mu);
    g_sched_cache[key] = ctx->serial_sched[m];
  }
  CUDA_TRY(cudaMemcpyAsync(ctx->d.t0, save, sizeof(double) * ctx->nt, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(s));
}
