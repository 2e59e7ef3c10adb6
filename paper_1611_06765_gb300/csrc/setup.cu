// setup.cu -- GPU construction of the basis, the channel tables, the index maps and the
// antisymmetrized Minnesota blocks of a pnmcc context.
//
//   basis     Sec. "Single-particle basis for infinite matter": k = 2 pi n / L, L^3 = N/rho,
//             closed shells; state order of the shell loop in Sec. "Developing a CCD code"
//             (shell, then n_x, n_y, n_z ascending, then s = -1 before +1).
//   channels  Sec. "Developing a CCD code": direct channels T (quantum numbers added) and
//             cross channels X (subtracted).  One warp per channel key walks the rows in
//             ascending state order; in a row every partner is unique for a given key, so a
//             ballot/popc prefix gives each pair its lexicographic position with no sort.
//   blocks    Sec. "Two-body interaction" (Minnesota in momentum space) and the particle-hole
//             character blocks t_pphh, v_pphh, v_pppp, v_hhhh, v_hpph of the channel mapping.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include <type_traits>

#include "pnm_context.cuh"

namespace {

__device__ __forceinline__ int cube_index(int x, int y, int z, int r) {
  if (x < -r || x > r || y < -r || y > r || z < -r || z > r) return -1;
  int w = 2 * r + 1;
  return ((x + r) * w + (y + r)) * w + (z + r);
}

// Charge label of a state (the .w of its char4): the spin s = +-1 in systems of neutrons only
// (species 1); s + 4t (t = +1 neutron, -1 proton) in systems with protons (species 2: protons
// only, 3: both), so that sums and differences of two labels decode uniquely into (S_z, T_z).
// A channel key's charge slot is (S_z + 2)/2 of 3 (neutrons only) or 3 (S_z + 2)/2 +
// (T_z + 2)/2 of 9.
__device__ __forceinline__ int charge_slot(int wsum, int species) {
  if (species == 1) return (wsum + 2) >> 1;
  int tsum = wsum >= 6 ? 2 : (wsum <= -6 ? -2 : 0);
  int ssum = wsum - 4 * tsum;
  return 3 * ((ssum + 2) >> 1) + ((tsum + 2) >> 1);
}

__device__ __forceinline__ int charge_sum(int slot, int species) {
  if (species == 1) return 2 * slot - 2;
  return (2 * (slot / 3) - 2) + 4 * (2 * (slot % 3) - 2);
}

__device__ __forceinline__ int charge_slots(int species) { return species == 1 ? 3 : 9; }

// State index of (n, w) in a system, or -1.  A lattice point holds 2 states (one species) or
// 4 (s = -1 then +1; within a spin the proton before the neutron).
__device__ __forceinline__ int lookup_state(const int* __restrict__ idx3, int r, int x, int y,
                                            int z, int w, int species) {
  int c = cube_index(x, y, z, r);
  if (c < 0) return -1;
  int sp, slot;
  if (species == 1) {
    if (w != -1 && w != 1) return -1;
    return idx3[2 * c + ((w + 1) >> 1)];
  }
  int t = (w == 3 || w == 5) ? 1 : ((w == -3 || w == -5) ? -1 : 0);
  if (t == 0 || !(species & (t > 0 ? 1 : 2))) return -1;
  sp = w - 4 * t;
  slot = species == 3 ? 2 * ((sp + 1) >> 1) + ((t + 1) >> 1) : (sp + 1) >> 1;
  return idx3[(species == 3 ? 4 : 2) * c + slot];
}

__device__ __forceinline__ void decode_key(int K, int m, int M, int species, int& Px, int& Py,
                                           int& Pz, int& W) {
  int nq = charge_slots(species);
  W = charge_sum(K % nq, species);
  int rest = K / nq;
  Pz = rest % M - m;
  rest /= M;
  Py = rest % M - m;
  Px = rest / M - m;
}

__device__ __forceinline__ int encode_key(int Px, int Py, int Pz, int W, int m, int M, int species) {
  return (((Px + m) * M + (Py + m)) * M + (Pz + m)) * charge_slots(species) + charge_slot(W, species);
}

// Spin s = +-1 of a state's charge label, and the state with the same momentum and species
// and the opposite spin (the global spin flip), or -1.
__device__ __forceinline__ int spin_of(int w, int species) {
  return species == 1 ? w : w - 4 * (w > 0 ? 1 : -1);
}

__device__ __forceinline__ int flip_state(const char4* __restrict__ nv, const int* __restrict__ idx3,
                                          int r, int p, int species) {
  char4 s = nv[p];
  return lookup_state(idx3, r, s.x, s.y, s.z, s.w - 2 * spin_of(s.w, species), species);
}

// ---------------------------------------------------------------------------- basis
// Cube points c = ((x+r)w + (y+r))w + (z+r) are in (n_x, n_y, n_z) lexicographic order, so a
// point's slot in the shell-ordered list is (points in lower shells) + (points of the same
// shell with a smaller cube index).  k_basis_count: one CTA counts the shells (shared-memory
// atomics) and writes the shell starts; k_basis_place: one thread per cube point counts the
// same-shell points before it and writes the two spin states.
__global__ void k_basis_count(int n2max, int r, int g, int* __restrict__ start, int* __restrict__ nsp_out) {
  extern __shared__ int cnt[];  // [n2max + 1]
  int w = 2 * r + 1, ncube = w * w * w;
  for (int k = threadIdx.x; k <= n2max; k += blockDim.x) cnt[k] = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < ncube; c += blockDim.x) {
    int x = c / (w * w) - r, y = (c / w) % w - r, z = c % w - r;
    int n2 = dot3(x, y, z);
    if (n2 <= n2max) atomicAdd(&cnt[n2], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int k = 0; k <= n2max; k++) {
      start[k] = acc;
      acc += cnt[k];
    }
    *nsp_out = g * acc;
  }
}

__global__ void k_basis_place(int n2max, int r, int species, const int* __restrict__ start,
                              char4* __restrict__ nvec, int* __restrict__ idx3) {
  int w = 2 * r + 1, ncube = w * w * w;
  int g = species == 3 ? 4 : 2;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncube) return;
  int x = c / (w * w) - r, y = (c / w) % w - r, z = c % w - r;
  int n2 = dot3(x, y, z);
  if (n2 > n2max) {
    for (int j = 0; j < g; j++) idx3[g * c + j] = -1;
    return;
  }
  // same-shell points before (x, y, z) in lexicographic order
  int rank = 0;
  for (int x2 = -r; x2 <= x; x2++) {
    int ylim = x2 < x ? r : y;
    for (int y2 = -r; y2 <= ylim; y2++) {
      int zlim = (x2 < x || y2 < y) ? r : z - 1;
      int rest = n2 - x2 * x2 - y2 * y2;
      for (int z2 = -r; z2 <= zlim; z2++) rank += (z2 * z2 == rest);
    }
  }
  int slot = start[n2] + rank;
  int j = 0;
  for (int sp = -1; sp <= 1; sp += 2)
    for (int t = -1; t <= 1; t += 2) {
      if (!(species & (t > 0 ? 1 : 2))) continue;
      int lab = species == 1 ? sp : sp + 4 * t;
      nvec[g * slot + j] = make_char4((char)x, (char)y, (char)z, (char)lab);
      idx3[g * c + j] = g * slot + j;
      j++;
    }
}

// hlut[m] = 1/2 sum_{a=R,S} (V_a / L^3)(pi/kappa_a)^{3/2} exp(-(2 pi/L)^2 m / (4 kappa_a)),
// the half of Vt that the antisymmetrized element adds twice (exact scaling by 1/2).
__global__ void k_lut(double* __restrict__ hlut, int len, double L, double VR, double kR,
                      double VS, double kS) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= len) return;
  double L3 = L * L * L;
  double q2 = (2.0 * PNM_PI / L) * (2.0 * PNM_PI / L) * (double)m;
  double vt = VR / L3 * pow(PNM_PI / kR, 1.5) * exp(-q2 / (4.0 * kR)) +
              VS / L3 * pow(PNM_PI / kS, 1.5) * exp(-q2 / (4.0 * kS));
  hlut[m] = 0.5 * vt;
}

// With protons the three Gaussians carry different spin-isospin weights: hlut3[3m + a] =
// 1/2 (V_a / L^3)(pi/kappa_a)^{3/2} exp(-(2 pi/L)^2 m / (4 kappa_a)) for a = R, T, S.
__global__ void k_lut3(double* __restrict__ hlut3, int len, double L, double VR, double kR,
                       double VT, double kT, double VS, double kS) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= len) return;
  double L3 = L * L * L;
  double q2 = (2.0 * PNM_PI / L) * (2.0 * PNM_PI / L) * (double)m;
  hlut3[3 * m] = 0.5 * (VR / L3 * pow(PNM_PI / kR, 1.5) * exp(-q2 / (4.0 * kR)));
  hlut3[3 * m + 1] = 0.5 * (VT / L3 * pow(PNM_PI / kT, 1.5) * exp(-q2 / (4.0 * kT)));
  hlut3[3 * m + 2] = 0.5 * (VS / L3 * pow(PNM_PI / kS, 1.5) * exp(-q2 / (4.0 * kS)));
}

// ------------------------------------------------------------------ twisted boundaries
// Sec. "Twist-averaged boundary conditions": k = (2 pi n + theta)/L, so the kinetic energy is
// hbar^2/2m (2 pi/L)^2 |n + phi|^2 with phi = theta/(2 pi).  The three axis terms are added
// smallest first and every step is rounded on its own (no fused multiply-add), so that states
// related by a permutation of axes with equal twist components get bit-identical values; with
// phi = 0 the result is the integer n^2.
__device__ __forceinline__ double twisted_n2(char4 sp, double px, double py, double pz) {
  double a = __dadd_rn((double)sp.x, px), b = __dadd_rn((double)sp.y, py);
  double c = __dadd_rn((double)sp.z, pz);
  a = __dmul_rn(a, a);
  b = __dmul_rn(b, b);
  c = __dmul_rn(c, c);
  double lo = fmin(a, b), hi = fmax(a, b);
  double x0 = fmin(lo, c), mid = fmax(lo, c);
  double x1 = fmin(mid, hi), x2 = fmax(mid, hi);
  return __dadd_rn(__dadd_rn(x0, x1), x2);
}

__global__ void k_twist_keys(const char4* __restrict__ nvec, int nsp, double px, double py,
                             double pz, double* __restrict__ key) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nsp) key[p] = twisted_n2(nvec[p], px, py, pz);
}

// Stable reorder by key ("order states by energy and fill holes"): a state's new slot is the
// number of states with a smaller key, or an equal key and a smaller shell-order index.
// Keys are staged through shared memory in tiles of the block size.
constexpr int TWIST_THREADS = 256;
__global__ void __launch_bounds__(TWIST_THREADS)
k_twist_rank(const double* __restrict__ key, int nsp, const char4* __restrict__ nvec_in,
             char4* __restrict__ nvec_out, double* __restrict__ key_out, int* __restrict__ perm) {
  __shared__ double sk[TWIST_THREADS];
  int p = blockIdx.x * TWIST_THREADS + threadIdx.x;
  double kp = p < nsp ? key[p] : 0.0;
  int rank = 0;
  for (int q0 = 0; q0 < nsp; q0 += TWIST_THREADS) {
    int q = q0 + threadIdx.x;
    sk[threadIdx.x] = q < nsp ? key[q] : 0.0;
    __syncthreads();
    int lim = min(TWIST_THREADS, nsp - q0);
    if (p < nsp)
      for (int u = 0; u < lim; u++) {
        double kq = sk[u];
        rank += (kq < kp) || (kq == kp && q0 + u < p);
      }
    __syncthreads();
  }
  if (p < nsp) {
    nvec_out[rank] = nvec_in[p];
    key_out[rank] = kp;
    perm[p] = rank;
  }
}

// Cube point -> state index map follows the reorder.
__global__ void k_twist_idx3(int* __restrict__ idx3, int n, const int* __restrict__ perm) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n && idx3[c] >= 0) idx3[c] = perm[idx3[c]];
}

// eps_p = h0_pp + sum_i <pi|v|pi>  (holes are the first N states of the system).
__global__ void k_eps(const char4* __restrict__ nvec, const double* __restrict__ lut, int nsp,
                      int N, double L, double hbar2_2m, double px, double py, double pz,
                      double* __restrict__ ekin, double* __restrict__ eps,
                      int* __restrict__ sp_sys, int* __restrict__ sp_hole, int sys) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nsp) return;
  char4 sp = nvec[p];
  double k0 = 2.0 * PNM_PI / L;
  double ek = hbar2_2m * k0 * k0 * twisted_n2(sp, px, py, pz);
  double acc = 0.0;
  for (int i = 0; i < N; i++) {
    char4 si = nvec[i];
    acc += v_minnesota_as(sp, si, sp, si, lut);
  }
  ekin[p] = ek;
  eps[p] = ek + acc;
  sp_sys[p] = sys;
  sp_hole[p] = p < N;
}

// ---------------------------------------------------------------------- channel counts
// One thread per ordered pair (p, q) of a system's states.  Direct keys (total momentum and
// charge label sum): restricted pairs p < q of one class, counted in cnt_hh (both holes,
// index < N) or cnt_pp (both particles).  Cross keys (n_p - n_q and the label difference):
// cnt_ph for p a particle and q a hole, cnt_hp for p a hole and q a particle.  Sums and
// differences of two states' momenta lie in [-m, m] (m = 2r), and of two labels decode
// uniquely (charge_slot), so every pair has a key.
__global__ void k_count_pairs(const char4* __restrict__ nvec, int m, int M, int species, int N, int nsp,
                              int* __restrict__ cnt_hh, int* __restrict__ cnt_pp, int* __restrict__ cnt_ph,
                              int* __restrict__ cnt_hp) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)nsp * nsp) return;
  const int p = (int)(e / nsp), q = (int)(e - (long)p * nsp);
  const char4 a = nvec[p], b = nvec[q];
  const bool hole_p = p < N, hole_q = q < N;
  if (p < q && hole_p == hole_q)
    atomicAdd((hole_p ? cnt_hh : cnt_pp) + encode_key(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w, m, M, species), 1);
  if (hole_p != hole_q)
    atomicAdd((hole_q ? cnt_ph : cnt_hp) + encode_key(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w, m, M, species), 1);
}

// ------------------------------------------------------------------------ channel fill
// One warp per direct channel.  Writes pairs (global state indices) in lexicographic order
// and the pair -> position tables used by the index maps.
__global__ void k_fill_direct(const char4* __restrict__ nvec, const int* __restrict__ idx3,
                              int r, int m, int M, int species, int N, int nsp, int sp_off, int nch_sys,
                              const int* __restrict__ key, const int* __restrict__ hh_off,
                              const int* __restrict__ pp_off, int2* __restrict__ hh_pair,
                              int2* __restrict__ pp_pair, int* __restrict__ pos_hh,
                              int* __restrict__ pos_pp) {
  int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (c >= nch_sys) return;
  int Px, Py, Pz, Sz;
  decode_key(key[c], m, M, species, Px, Py, Pz, Sz);
  int np = nsp - N;
  int nh_fill = 0, np_fill = 0;
  unsigned lt = (1u << lane) - 1u;
  for (int p0 = 0; p0 < nsp; p0 += 32) {
    int p = p0 + lane;
    int q = -1;
    bool vh = false, vp = false;
    if (p < nsp) {
      char4 s = nvec[p];
      q = lookup_state(idx3, r, Px - s.x, Py - s.y, Pz - s.z, Sz - s.w, species);
      bool v = (q > p) && ((p < N) == (q < N));
      vh = v && p < N;
      vp = v && p >= N;
    }
    unsigned bh = __ballot_sync(0xffffffffu, vh);
    unsigned bp = __ballot_sync(0xffffffffu, vp);
    if (vh) {
      int pos = nh_fill + __popc(bh & lt);
      hh_pair[hh_off[c] + pos] = make_int2(p + sp_off, q + sp_off);
      pos_hh[p * N + q] = pos;
    }
    if (vp) {
      int pos = np_fill + __popc(bp & lt);
      pp_pair[pp_off[c] + pos] = make_int2(p + sp_off, q + sp_off);
      pos_pp[(size_t)(p - N) * np + (q - N)] = pos;
    }
    nh_fill += __popc(bh);
    np_fill += __popc(bp);
  }
}

// One warp per cross channel: rows (a,i) and columns (k,c) in lexicographic order.
__global__ void k_fill_cross(const char4* __restrict__ nvec, const int* __restrict__ idx3,
                             int r, int m, int M, int species, int N, int nsp, int sp_off, int nx_sys,
                             const int* __restrict__ key, const int* __restrict__ ph_off,
                             const int* __restrict__ hp_off, int2* __restrict__ ph_pair,
                             int2* __restrict__ hp_pair, int* __restrict__ phpos,
                             int* __restrict__ phch, int* __restrict__ hppos) {
  int x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (x >= nx_sys) return;
  int Dx, Dy, Dz, Ds;
  decode_key(key[x], m, M, species, Dx, Dy, Dz, Ds);
  int np = nsp - N;
  int f_ph = 0, f_hp = 0;
  unsigned lt = (1u << lane) - 1u;
  for (int p0 = 0; p0 < nsp; p0 += 32) {
    int p = p0 + lane;
    int q = -1;
    bool vph = false, vhp = false;
    if (p < nsp) {
      char4 s = nvec[p];
      q = lookup_state(idx3, r, s.x - Dx, s.y - Dy, s.z - Dz, s.w - Ds, species);
      vph = (q >= 0) && p >= N && q < N;
      vhp = (q >= 0) && p < N && q >= N;
    }
    unsigned b1 = __ballot_sync(0xffffffffu, vph);
    unsigned b2 = __ballot_sync(0xffffffffu, vhp);
    if (vph) {
      int pos = f_ph + __popc(b1 & lt);
      ph_pair[ph_off[x] + pos] = make_int2(p + sp_off, q + sp_off);
      phpos[(size_t)(p - N) * N + q] = pos;
      phch[(size_t)(p - N) * N + q] = x;
    }
    if (vhp) {
      int pos = f_hp + __popc(b2 & lt);
      hp_pair[hp_off[x] + pos] = make_int2(p + sp_off, q + sp_off);
      hppos[(size_t)p * np + (q - N)] = pos;
    }
    f_ph += __popc(b1);
    f_hp += __popc(b2);
  }
}

// ------------------------------------------------------------------------- index maps
// Position code of t_{h1 h2}^{p1 p2} (system-local states) in the restricted direct blocks:
// sign * (t index + 1), 0 where it vanishes (p1 = p2 or h1 = h2) or its channel is not held.
__device__ __forceinline__ int t_code(int p1, int p2, int h1, int h2, const char4* __restrict__ nv, int N,
                                      int np, int m, int M, int species, const int* __restrict__ key2ch,
                                      int ch0, const long* __restrict__ ch_t_off,
                                      const int* __restrict__ ch_npp, const int* __restrict__ pos_hh,
                                      const int* __restrict__ pos_pp) {
  if (p1 == p2 || h1 == h2) return 0;
  int sgn = 1;
  if (p1 > p2) { int z = p1; p1 = p2; p2 = z; sgn = -sgn; }
  if (h1 > h2) { int z = h1; h1 = h2; h2 = z; sgn = -sgn; }
  char4 s1 = nv[p1], s2 = nv[p2];
  int ch = key2ch[encode_key(s1.x + s2.x, s1.y + s2.y, s1.z + s2.z, s1.w + s2.w, m, M, species)];
  if (ch < 0) return 0;
  int g = ch0 + ch;
  long idx = ch_t_off[g] + (long)pos_hh[h1 * N + h2] * ch_npp[g] + pos_pp[(size_t)(p1 - N) * np + (p2 - N)];
  return sgn * (int)(idx + 1);
}

// T_x[(a,i)][(k,c)] = t_ik^ac, read from the restricted direct block with its sign.
// Encoded as sign * (t index + 1); 0 where the element vanishes (a = c or i = k).
__global__ void k_xmap(int x0, const int* __restrict__ x_nph, const int* __restrict__ x_nhp,
                       const long* __restrict__ x_t_off, const int* __restrict__ x_ph_off,
                       const int* __restrict__ x_hp_off, const int2* __restrict__ ph_pair,
                       const int2* __restrict__ hp_pair, const char4* __restrict__ nvec,
                       int sp_off, int N, int nsp, int m, int M, int species,
                       const int* __restrict__ key2ch, int ch0, const long* __restrict__ ch_t_off,
                       const int* __restrict__ ch_npp, const int* __restrict__ pos_hh,
                       const int* __restrict__ pos_pp, int* __restrict__ xmap) {
  int x = x0 + blockIdx.x;
  int nph = x_nph[x], nhp = x_nhp[x];
  long base = x_t_off[x];
  for (int e = threadIdx.x; e < nph * nhp; e += blockDim.x) {
    int rr = e / nhp, ss = e % nhp;
    int2 ai = ph_pair[x_ph_off[x] + rr], kc = hp_pair[x_hp_off[x] + ss];
    int a = ai.x - sp_off, i = ai.y - sp_off, k = kc.x - sp_off, c = kc.y - sp_off;
    xmap[base + e] = t_code(a, c, i, k, nvec + sp_off, N, nsp - N, m, M, species, key2ch, ch0, ch_t_off,
                            ch_npp, pos_hh, pos_pp);
  }
}

// For every restricted t element (ij, ab) of a row: the positions of
// Q_ij^ab, Q_ji^ab, Q_ij^ba, Q_ji^ba with Q_ij^ab = Q_x[(a,i)][(j,b)].
// Position of Q_x[(p,h)][(h2,p2)], or -1.  The ph kernels form Q (and read T) only in the
// cross channels with S_z >= 0 and, in those with S_z = 0, only in the rows of a spin-up
// particle; every other position is replaced by that of its spin flip
// Q_F(x)[(Fp,Fh)][(Fh2,Fp2)], which holds the same value for flip-symmetric amplitudes.
__device__ __forceinline__ int qpos(int p, int h, int h2, int p2, int N, int np,
                                    const int* __restrict__ phch, const int* __restrict__ phpos,
                                    const int* __restrict__ hppos, int x0,
                                    const long* __restrict__ x_t_off,
                                    const int* __restrict__ x_nhp, const int* __restrict__ x_cls,
                                    const char4* __restrict__ nv, const int* __restrict__ idx3, int r,
                                    int species) {
  size_t u = (size_t)(p - N) * N + h;
  int x = phch[u];
  if (x < 0) return -1;
  int g = x0 + x;
  if (x_cls[g] < 0 || (x_cls[g] == 0 && spin_of(nv[p].w, species) < 0)) {
    p = flip_state(nv, idx3, r, p, species);
    h = flip_state(nv, idx3, r, h, species);
    h2 = flip_state(nv, idx3, r, h2, species);
    p2 = flip_state(nv, idx3, r, p2, species);
    u = (size_t)(p - N) * N + h;
    g = x0 + phch[u];
  }
  return (int)(x_t_off[g] + (long)phpos[u] * x_nhp[g] + hppos[(size_t)h2 * np + (p2 - N)]);
}

__global__ void k_qmap(int row0, const int2* __restrict__ row_item,
                       const int* __restrict__ ch_hh_off, const int* __restrict__ ch_pp_off,
                       const int* __restrict__ ch_npp, const long* __restrict__ ch_t_off,
                       const int2* __restrict__ hh_pair, const int2* __restrict__ pp_pair,
                       int sp_off, int N, int nsp, const int* __restrict__ phch,
                       const int* __restrict__ phpos, const int* __restrict__ hppos, int x0,
                       const long* __restrict__ x_t_off, const int* __restrict__ x_nhp,
                       const int* __restrict__ x_cls, const char4* __restrict__ nvec,
                       const int* __restrict__ idx3, int r, int species, int4* __restrict__ qmap) {
  int2 it = row_item[row0 + blockIdx.x];
  int c = it.x, ij = it.y;
  int np = nsp - N;
  int2 h = hh_pair[ch_hh_off[c] + ij];
  int i = h.x - sp_off, j = h.y - sp_off;
  int npp = ch_npp[c];
  long base = ch_t_off[c] + (long)ij * npp;
  const char4* nv = nvec + sp_off;
  for (int ab = threadIdx.x; ab < npp; ab += blockDim.x) {
    int2 pb = pp_pair[ch_pp_off[c] + ab];
    int a = pb.x - sp_off, b = pb.y - sp_off;
    int4 q;
    q.x = qpos(a, i, j, b, N, np, phch, phpos, hppos, x0, x_t_off, x_nhp, x_cls, nv, idx3, r, species);
    q.y = qpos(a, j, i, b, N, np, phch, phpos, hppos, x0, x_t_off, x_nhp, x_cls, nv, idx3, r, species);
    q.z = qpos(b, i, j, a, N, np, phch, phpos, hppos, x0, x_t_off, x_nhp, x_cls, nv, idx3, r, species);
    q.w = qpos(b, j, i, a, N, np, phch, phpos, hppos, x0, x_t_off, x_nhp, x_cls, nv, idx3, r, species);
    qmap[base + ab] = q;
  }
}

// ------------------------------------------------------------------------ spin flip
// The global spin flip F (every state to the one of opposite spin) leaves H and the
// spin-saturated reference unchanged, so the amplitudes of the solution obey
// t(F i, F j; F a, F b) = t(i, j; a, b) and every cross-channel matrix M of the ph term
// (T, W, <kb|v|cj>, Q) obeys M_F(x)[F r][F c] = M_x[r][c].  For every cross channel of a
// system it records:
//   x_cls   +1 for S_z = s_a - s_i > 0 (formed in full), 0 for S_z = 0 (F maps the channel
//           onto itself; formed on its spin-up rows), -1 for S_z < 0 (not formed: the update
//           reads the flipped channel F(x) instead, see qpos);
//   x_fcol  per column (k,c) the column of (F k, F c) in F(x);
//   x_rrow / x_rcol (S_z = 0)  the rows (a,i) and columns (k,c) with spin-up a and k, in order
//           (half of each: the other half are their flips).
// Sets *err when the rows or columns of a channel do not map onto one channel F(x) (a
// reference that is not spin saturated).
// One warp per channel; the spin-up rows and columns are compacted in order with ballots.
__global__ void k_xflip(int x0, int nxs, const int* __restrict__ x_nph, const int* __restrict__ x_nhp,
                        const int* __restrict__ x_ph_off, const int* __restrict__ x_hp_off,
                        const int2* __restrict__ ph_pair, const int2* __restrict__ hp_pair,
                        const char4* __restrict__ nvec, const int* __restrict__ idx3, int r, int species,
                        int sp_off, int N, int nsp, const int* __restrict__ phpos,
                        const int* __restrict__ phch, const int* __restrict__ hppos, int* __restrict__ x_cls,
                        int* __restrict__ x_fcol,
                        int* __restrict__ x_rrow, int* __restrict__ x_rcol, int* __restrict__ err) {
  const int xl = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (xl >= nxs) return;  // warp-uniform
  const unsigned lt = (1u << lane) - 1u;
  const int x = x0 + xl;
  const int nph = x_nph[x], nhp = x_nhp[x], po = x_ph_off[x], ho = x_hp_off[x];
  const char4* nv = nvec + sp_off;
  const int np = nsp - N;
  bool bad = nph <= 0 || nhp <= 0;
  int sz = 0, mir = -1, nr = 0, nc = 0;
  if (!bad) {
    int2 p0 = ph_pair[po];
    sz = spin_of(nv[p0.x - sp_off].w, species) - spin_of(nv[p0.y - sp_off].w, species);
  }
  for (int k0 = 0; k0 < nph && !bad; k0 += 32) {
    const int k = k0 + lane;
    bool lbad = false, up = false;
    int ch = -1;
    if (k < nph) {
      int2 ai = ph_pair[po + k];
      int a = ai.x - sp_off, i = ai.y - sp_off;
      int fa = flip_state(nv, idx3, r, a, species), fi = flip_state(nv, idx3, r, i, species);
      if (fa < N || fi < 0 || fi >= N) {
        lbad = true;
      } else {
        size_t u = (size_t)(fa - N) * N + fi;
        ch = phch[u];
        if (ch < 0) lbad = true;
        up = sz == 0 && spin_of(nv[a].w, species) > 0;
      }
    }
    if (mir < 0) mir = __shfl_sync(0xffffffffu, ch, 0);
    bad = __any_sync(0xffffffffu, lbad || (k < nph && ch != mir));
    unsigned bu = __ballot_sync(0xffffffffu, up);
    if (up) x_rrow[po + nr + __popc(bu & lt)] = k;
    nr += __popc(bu);
  }
  for (int k0 = 0; k0 < nhp && !bad; k0 += 32) {
    const int k = k0 + lane;
    bool lbad = false, up = false;
    if (k < nhp) {
      int2 hc = hp_pair[ho + k];
      int h = hc.x - sp_off, p = hc.y - sp_off;
      int fh = flip_state(nv, idx3, r, h, species), fp = flip_state(nv, idx3, r, p, species);
      if (fh < 0 || fh >= N || fp < N) {
        lbad = true;
      } else {
        x_fcol[ho + k] = hppos[(size_t)fh * np + (fp - N)];
        up = sz == 0 && spin_of(nv[h].w, species) > 0;
      }
    }
    bad = __any_sync(0xffffffffu, lbad);
    unsigned bu = __ballot_sync(0xffffffffu, up);
    if (up) x_rcol[ho + nc + __popc(bu & lt)] = k;
    nc += __popc(bu);
  }
  if (lane != 0) return;
  if (!bad && sz == 0 && (2 * nr != nph || 2 * nc != nhp || mir != xl)) bad = true;
  if (!bad && sz != 0 && mir == xl) bad = true;
  x_cls[x] = sz > 0 ? 1 : (sz == 0 ? 0 : -1);
  if (bad) atomicExch(err, 1);
}

// Per amplitude: the position code of its spin-flipped amplitude (sign * (index + 1)); one
// CTA per (channel, ij) row.
__global__ void k_fmap(int row0, const int2* __restrict__ row_item, const int* __restrict__ ch_hh_off,
                       const int* __restrict__ ch_pp_off, const int* __restrict__ ch_npp,
                       const long* __restrict__ ch_t_off, const int2* __restrict__ hh_pair,
                       const int2* __restrict__ pp_pair, const char4* __restrict__ nvec,
                       const int* __restrict__ idx3, int r, int species, int sp_off, int N, int nsp, int m,
                       int M, const int* __restrict__ key2ch, int ch0, const int* __restrict__ pos_hh,
                       const int* __restrict__ pos_pp, int* __restrict__ fmap, int* __restrict__ err) {
  int2 it = row_item[row0 + blockIdx.x];
  int c = it.x, ij = it.y;
  const char4* nv = nvec + sp_off;
  int2 h = hh_pair[ch_hh_off[c] + ij];
  int fi = flip_state(nv, idx3, r, h.x - sp_off, species), fj = flip_state(nv, idx3, r, h.y - sp_off, species);
  int npp = ch_npp[c];
  long base = ch_t_off[c] + (long)ij * npp;
  for (int ab = threadIdx.x; ab < npp; ab += blockDim.x) {
    int2 pb = pp_pair[ch_pp_off[c] + ab];
    int fa = flip_state(nv, idx3, r, pb.x - sp_off, species), fb = flip_state(nv, idx3, r, pb.y - sp_off, species);
    int code = 0;
    if (fi >= 0 && fi < N && fj >= 0 && fj < N && fa >= N && fb >= N)
      code = t_code(fa, fb, fi, fj, nv, N, nsp - N, m, M, species, key2ch, ch0, ch_t_off, ch_npp, pos_hh,
                    pos_pp);
    if (code == 0) atomicExch(err, 1);
    fmap[base + ab] = code;
  }
}

// Pairs containing each state (for the one-body intermediates): count then fill.
// One warp per state p of the system; partners d of the same class.
__global__ void k_occ(int fill, const char4* __restrict__ nvec, int sp_off, int N, int nsp,
                      int m, int M, int species, const int* __restrict__ key2ch, int ch0,
                      const int* __restrict__ ch_hh_off, const int* __restrict__ ch_pp_off,
                      const int* __restrict__ pos_hh, const int* __restrict__ pos_pp,
                      int* __restrict__ occ_cnt, const int* __restrict__ occ_off,
                      int* __restrict__ occ_idx) {
  int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (p >= nsp) return;
  int np = nsp - N;
  bool hole = p < N;
  int lo = hole ? 0 : N, hi = hole ? N : nsp;
  char4 sp = nvec[sp_off + p];
  int n = 0;
  unsigned lt = (1u << lane) - 1u;
  for (int d0 = lo; d0 < hi; d0 += 32) {
    int d = d0 + lane;
    int gidx = -1;
    if (d < hi && d != p) {
      char4 sd = nvec[sp_off + d];
      int K = encode_key(sp.x + sd.x, sp.y + sd.y, sp.z + sd.z, sp.w + sd.w, m, M, species);
      int ch = key2ch[K];
      if (ch >= 0) {
        int p1 = min(p, d), p2 = max(p, d);
        int g = ch0 + ch;
        gidx = hole ? ch_hh_off[g] + pos_hh[p1 * N + p2]
                    : ch_pp_off[g] + pos_pp[(size_t)(p1 - N) * np + (p2 - N)];
      }
    }
    unsigned b = __ballot_sync(0xffffffffu, gidx >= 0);
    if (fill && gidx >= 0) occ_idx[occ_off[sp_off + p] + n + __popc(b & lt)] = gidx;
    n += __popc(b);
  }
  if (!fill && lane == 0) occ_cnt[p] = n;
}

// -------------------------------------------------------------------------- V blocks
__global__ void k_v_pphh(int row0, const int2* __restrict__ row_item,
                         const int* __restrict__ ch_hh_off, const int* __restrict__ ch_pp_off,
                         const int* __restrict__ ch_npp, const long* __restrict__ ch_t_off,
                         const int2* __restrict__ hh_pair, const int2* __restrict__ pp_pair,
                         const char4* __restrict__ nvec, const double* __restrict__ lut,
                         double* __restrict__ v_pphh) {
  int2 it = row_item[row0 + blockIdx.x];
  int c = it.x, ij = it.y;
  int2 h = hh_pair[ch_hh_off[c] + ij];
  char4 si = nvec[h.x], sj = nvec[h.y];
  int npp = ch_npp[c];
  long base = ch_t_off[c] + (long)ij * npp;
  for (int ab = threadIdx.x; ab < npp; ab += blockDim.x) {
    int2 pb = pp_pair[ch_pp_off[c] + ab];
    v_pphh[base + ab] = v_minnesota_as(nvec[pb.x], nvec[pb.y], si, sj, lut);
  }
}

// Denominators eps_ij^ab = e_i + e_j - e_a - e_b (HF energies) and their reciprocals.
__global__ void k_den(int row0, const int2* __restrict__ row_item, const int* __restrict__ ch_hh_off,
                      const int* __restrict__ ch_pp_off, const int* __restrict__ ch_npp,
                      const long* __restrict__ ch_t_off, const int2* __restrict__ hh_pair,
                      const int2* __restrict__ pp_pair, const double* __restrict__ eps,
                      double* __restrict__ den, double* __restrict__ inv_den) {
  int2 it = row_item[row0 + blockIdx.x];
  int c = it.x, ij = it.y;
  int2 h = hh_pair[ch_hh_off[c] + ij];
  double eij = eps[h.x] + eps[h.y];
  int npp = ch_npp[c];
  long base = ch_t_off[c] + (long)ij * npp;
  for (int ab = threadIdx.x; ab < npp; ab += blockDim.x) {
    int2 pb = pp_pair[ch_pp_off[c] + ab];
    double d = eij - eps[pb.x] - eps[pb.y];
    den[base + ab] = d;
    inv_den[base + ab] = 1.0 / d;
  }
}

// ---------------------------------------------------------------------- ladder basis
// For two neutrons <ab|v|cd> acts only on the spin singlet: with each pp pair of an S_z = 0
// channel written with its spin-up particle first (sign e = -1 when the stored order is the
// other one), the element e_x e_z <x|v|z> depends on the spatial pair of z only through the
// two Gaussians of n_u - n_u' and n_u - n_d', so it is the same for z and its partner z'
// (spatial labels of the two spins exchanged).  The pp ladder R_x = sum_z <x|v|z> t_z is then
// R_x = e_x sum_c W(c(x), c) s_c with one vector per partner couple, s_c = e_z t_z + e_z' t_z'
// and W(c, c') = e e' <rep c|v|rep c'>: a quarter of the elements and of the products.  Other
// channels (systems with protons) keep one vector per pair.
// One CTA (256 threads) per channel with a V_pppp block; dynamic shared memory holds three
// ints per pair: partner position, sign e, rank of a representative.
constexpr int LAD_THREADS = 256;
__global__ void __launch_bounds__(LAD_THREADS) k_ladder_basis(
    const int* __restrict__ chans, int species, const int* __restrict__ ch_pp_off,
    const int* __restrict__ ch_npp, const int2* __restrict__ pp_pair, const char4* __restrict__ nvec,
    int N, int nsp, int r, const int* __restrict__ idx3, const int* __restrict__ pos_pp,
    int* __restrict__ lad_map, int2* __restrict__ lad_mem, int* __restrict__ ch_nlad) {
  extern __shared__ int lsm[];
  __shared__ int warp_tot[LAD_THREADS / 32];
  __shared__ int base_sh;
  int c = chans[blockIdx.x];
  int off = ch_pp_off[c], npp = ch_npp[c];
  if (species != 1) {  // no reduction: one vector per pair
    for (int x = threadIdx.x; x < npp; x += blockDim.x) {
      lad_map[off + x] = x + 1;
      lad_mem[off + x] = make_int2(x + 1, 0);
    }
    if (threadIdx.x == 0) ch_nlad[c] = npp;
    return;
  }
  int* part = lsm;
  int* sgn = lsm + npp;
  int* rnk = lsm + 2 * npp;
  int np = nsp - N;
  for (int x = threadIdx.x; x < npp; x += blockDim.x) {
    int2 pr = pp_pair[off + x];
    char4 sa = nvec[pr.x], sb = nvec[pr.y];
    bool a_up = sa.w > 0;
    char4 su = a_up ? sa : sb, sd = a_up ? sb : sa;
    sgn[x] = a_up ? 1 : -1;
    int u2 = lookup_state(idx3, r, sd.x, sd.y, sd.z, 1, 1);   // spin up at the down momentum
    int d2 = lookup_state(idx3, r, su.x, su.y, su.z, -1, 1);  // spin down at the up momentum
    int p1 = min(u2, d2), p2 = max(u2, d2);
    part[x] = (p1 < N) ? x : pos_pp[(size_t)(p1 - N) * np + (p2 - N)];
  }
  if (threadIdx.x == 0) base_sh = 0;
  __syncthreads();
  // rank of each representative (partner position >= own position) in pair order
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int x0 = 0; x0 < npp; x0 += blockDim.x) {
    int x = x0 + threadIdx.x;
    bool rep = x < npp && part[x] >= x;
    unsigned bal = __ballot_sync(0xffffffffu, rep);
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    int before = base_sh;
    for (int w = 0; w < warp; w++) before += warp_tot[w];
    if (rep) rnk[x] = before + __popc(bal & ((1u << lane) - 1u));
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < LAD_THREADS / 32; w++) tot += warp_tot[w];
      base_sh += tot;
    }
    __syncthreads();
  }
  for (int x = threadIdx.x; x < npp; x += blockDim.x) {
    int px = part[x];
    int rk = px >= x ? rnk[x] : rnk[px];
    lad_map[off + x] = (rk + 1) * sgn[x];
    if (px >= x) lad_mem[off + rk] = make_int2((x + 1) * sgn[x], px != x ? (px + 1) * sgn[px] : 0);
  }
  if (threadIdx.x == 0) ch_nlad[c] = base_sh;
}

// W(c, c') = e e' <rep c|v|rep c'> for VLAD_ROWS rows of one channel per CTA; the channel's
// representative pair states, their signs and the LUT are staged in shared memory.
constexpr int VLAD_ROWS = 16;
// Out: double (the FP64 ladder V) or f2 (its FP32-pair copy, the element split once).
template <typename Out>
__global__ void __launch_bounds__(256) k_v_ladder(const int2* __restrict__ items, const int* __restrict__ ch_pp_off,
                                                  const int* __restrict__ ch_nlad, const long* __restrict__ ch_vl_off,
                                                  const int2* __restrict__ lad_mem, const int2* __restrict__ pp_pair,
                                                  const char4* __restrict__ nvec, const double* __restrict__ lut,
                                                  int lut_elems, Out* __restrict__ v_lad) {
  extern __shared__ __align__(16) unsigned char vsm[];
  double* slut = reinterpret_cast<double*>(vsm);
  int2 it = items[blockIdx.x];
  int c = it.x, r0 = it.y;
  int nl = ch_nlad[c], off = ch_pp_off[c];
  char4* sa = reinterpret_cast<char4*>(slut + lut_elems);
  char4* sb = sa + nl;
  int* sg = reinterpret_cast<int*>(sb + nl);
  for (int m = threadIdx.x; m < lut_elems; m += blockDim.x) slut[m] = lut[m];
  for (int q = threadIdx.x; q < nl; q += blockDim.x) {
    int m = lad_mem[off + q].x;
    int pos = (m > 0 ? m : -m) - 1;
    int2 pr = pp_pair[off + pos];
    sa[q] = nvec[pr.x];
    sb[q] = nvec[pr.y];
    sg[q] = m > 0 ? 1 : -1;
  }
  __syncthreads();
  int r1 = min(r0 + VLAD_ROWS, nl);
  for (int row = r0; row < r1; row++) {
    char4 sc = sa[row], sd = sb[row];
    int g = sg[row];
    Out* out = v_lad + ch_vl_off[c] + (long)row * nl;
    for (int q = threadIdx.x; q < nl; q += blockDim.x) {
      double v = v_minnesota_as(sa[q], sb[q], sc, sd, slut);
      v = g * sg[q] > 0 ? v : __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ull);
      if constexpr (std::is_same<Out, f2>::value) out[q] = Arith<f2>::from_double(v);
      else out[q] = v;
    }
  }
}

__global__ void k_v_hhhh(int c0, const int* __restrict__ ch_hh_off,
                         const int* __restrict__ ch_nhh, const long* __restrict__ ch_vhh_off,
                         const int2* __restrict__ hh_pair, const char4* __restrict__ nvec,
                         const double* __restrict__ lut, double* __restrict__ v_hhhh) {
  int c = c0 + blockIdx.x;
  int nh = ch_nhh[c];
  for (int e = threadIdx.x; e < nh * nh; e += blockDim.x) {
    int kl = e / nh, ij = e % nh;
    int2 a = hh_pair[ch_hh_off[c] + kl], b = hh_pair[ch_hh_off[c] + ij];
    v_hhhh[ch_vhh_off[c] + e] = v_minnesota_as(nvec[a.x], nvec[a.y], nvec[b.x], nvec[b.y], lut);
  }
}

// V1_x[(k,c)][(j,b)] = <kb|v|cj>,  W_x[(k,c)][(e,l)] = <kl|v|ce> (stored as W_x^T).
__global__ void k_v_cross(int x0, const int* __restrict__ x_nph, const int* __restrict__ x_nhp,
                          const long* __restrict__ x_c_off, const long* __restrict__ x_w_off,
                          const int* __restrict__ x_ph_off, const int* __restrict__ x_hp_off,
                          const int2* __restrict__ ph_pair, const int2* __restrict__ hp_pair,
                          const char4* __restrict__ nvec, const double* __restrict__ lut,
                          double* __restrict__ x_v1, double* __restrict__ x_w) {
  int x = x0 + blockIdx.x;
  int nph = x_nph[x], nhp = x_nhp[x];
  for (int e = threadIdx.x; e < nhp * nhp; e += blockDim.x) {
    int2 kc = hp_pair[x_hp_off[x] + e / nhp], jb = hp_pair[x_hp_off[x] + e % nhp];
    x_v1[x_c_off[x] + e] = v_minnesota_as(nvec[kc.x], nvec[jb.y], nvec[kc.y], nvec[jb.x], lut);
  }
  // stored transposed, W^T[(e,l)][(k,c)], so the ph kernel stages it with coalesced loads
  for (int e = threadIdx.x; e < nph * nhp; e += blockDim.x) {
    int2 el = ph_pair[x_ph_off[x] + e / nhp], kc = hp_pair[x_hp_off[x] + e % nhp];
    x_w[x_w_off[x] + e] = v_minnesota_as(nvec[kc.x], nvec[el.y], nvec[kc.y], nvec[el.x], lut);
  }
}

template <typename T>
T* dalloc(size_t n, std::vector<void*>& owned, cudaStream_t s) {
  void* p = pnm_pool_alloc(s, std::max<size_t>(n, 1) * sizeof(T));
  owned.push_back(p);
  return (T*)p;
}

template <typename T>
void h2d(T* d, const std::vector<T>& h, cudaStream_t s) {
  if (!h.empty()) CUDA_TRY(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
}

template <typename T>
std::vector<T> d2h(const T* d, size_t n, cudaStream_t s) {
  std::vector<T> h(n);
  if (n) {
    CUDA_TRY(cudaMemcpyAsync(h.data(), d, n * sizeof(T), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  return h;
}

int isqrt_floor(int x) {
  int r = (int)std::floor(std::sqrt((double)x));
  while (r * r > x) r--;
  while ((r + 1) * (r + 1) <= x) r++;
  return r;
}

}  // namespace

// Per-system scratch that lives only during setup.
struct SysScratch {
  cudaStream_t stream = nullptr;  // allocations and their release are ordered on it
  int* idx3 = nullptr;
  int *key2ch = nullptr, *key2x = nullptr;
  int *pos_hh = nullptr, *pos_pp = nullptr, *phpos = nullptr, *phch = nullptr, *hppos = nullptr;
  std::vector<int> dkeys, dnhh, dnpp, xkeys, xnph, xnhp;
  std::vector<void*> owned;
  ~SysScratch() {
    for (void* p : owned) pnm_pool_free(stream, p);
  }
};

// The ladder-basis V_pppp of every system into out64 (FP64) or out2 (FP32 pairs).
void pnm_ladder_v(pnm_ctx* ctx, double* out64, f2* out2) {
  cudaStream_t s = ctx->stream;
  DevState& D = ctx->d;
  const int nsys = (int)ctx->sys.size();
  if (out64) smem_at_least(k_v_ladder<double>, ctx->vl_smem);
  if (out2) smem_at_least(k_v_ladder<f2>, ctx->vl_smem);
  for (int k = 0; k < nsys; k++) {
    const int lo = ctx->vl_sys[k], hi = ctx->vl_sys[k + 1];
    if (hi <= lo) continue;
    const SysInfo& S = ctx->sys[k];
    const int lut_elems = S.lut_len * (S.species == 1 ? 1 : 3);
    if (out64)
      k_v_ladder<double><<<(unsigned)(hi - lo), 256, ctx->vl_smem, s>>>(
          ctx->vl_items + lo, D.ch_pp_off, D.ch_nlad, D.ch_vpp_off, D.lad_mem, D.pp_pair, D.nvec,
          D.lut + S.lut_off, lut_elems, out64);
    if (out2)
      k_v_ladder<f2><<<(unsigned)(hi - lo), 256, ctx->vl_smem, s>>>(
          ctx->vl_items + lo, D.ch_pp_off, D.ch_nlad, D.ch_vpp_off, D.lad_mem, D.pp_pair, D.nvec,
          D.lut + S.lut_off, lut_elems, out2);
  }
  CUDA_TRY(cudaGetLastError());
}

// The FP64 ladder V (the FP64 pp ladder and operator): built once, on first use.
void pnm_need_vpp64(pnm_ctx* ctx) {
  if (ctx->d.v_pppp) return;
  ctx->d.v_pppp = ctx_alloc<double>(ctx, std::max<long>(ctx->nvpp, 1));
  pnm_ladder_v(ctx, ctx->d.v_pppp, nullptr);
}

// The FP32-pair ladder V (the refinement sweeps' pp ladder, and the source of the tensor-core
// ladder's BF16 tiles, whose split starts from the same FP32 rounding): built once.
void pnm_need_vpp_f2(pnm_ctx* ctx) {
  if (ctx->vpp_f2) return;
  ctx->vpp_f2 = ctx_alloc<f2>(ctx, std::max<long>(ctx->nvpp, 1));
  pnm_ladder_v(ctx, nullptr, ctx->vpp_f2);
}

void pnm_build(pnm_ctx* ctx, int nsys, const int* Ns, const int* Zs, const double* rhos,
               const int* n2maxs, const double* thetas, const pnm_minnesota& P) {
  cudaStream_t s = ctx->stream;
  DevState& D = ctx->d;
  std::vector<SysInfo>& sys = ctx->sys;
  sys.resize(nsys);
  std::vector<SysScratch> scr(nsys);
  for (auto& x : scr) x.stream = s;
  ctx->hbar2_2m = P.hbar2_2m;

  // ---- basis per system (into scratch), closed-shell check on the host
  std::vector<std::vector<char4>> hvec(nsys);
  int nsp_total = 0, lut_total = 0;
  for (int k = 0; k < nsys; k++) {
    SysInfo& S = sys[k];
    int Nn = Ns[k], Z = Zs ? Zs[k] : 0;
    if (Nn < 0 || Z < 0 || (Nn > 0 && Z > 0 && Nn != Z))
      throw PnmError{PNM_EINVAL, "system " + std::to_string(k) +
                                     ": neutrons only, protons only, or equal numbers of both"};
    S.N = Nn + Z;
    S.Z = Z;
    S.species = (Nn > 0 ? 1 : 0) | (Z > 0 ? 2 : 0);
    S.rho = rhos[k];
    S.n2max = n2maxs[k];
    if (S.N <= 0 || !(S.rho > 0.0) || S.n2max < 0 || S.n2max > 400)
      throw PnmError{PNM_EINVAL, "invalid N, rho or n2max"};
    S.r = isqrt_floor(S.n2max);
    S.m = 2 * S.r;
    S.M = 2 * S.m + 1;
    S.nkeys = S.M * S.M * S.M * (S.species == 1 ? 3 : 9);
    int g = S.species == 3 ? 4 : 2;  // states per lattice point
    S.L = std::cbrt((double)S.N / S.rho);
    bool twisted = false;
    for (int a = 0; a < 3; a++) {
      double th = thetas ? thetas[3 * k + a] : 0.0;
      if (!std::isfinite(th)) throw PnmError{PNM_EINVAL, "twist angle is not finite"};
      S.phi[a] = th / (2.0 * PNM_PI);
      twisted = twisted || S.phi[a] != 0.0;
    }
    int w = 2 * S.r + 1, ncube = w * w * w;
    char4* tvec = dalloc<char4>((size_t)g * ncube, scr[k].owned, s);
    scr[k].idx3 = dalloc<int>((size_t)g * ncube, scr[k].owned, s);
    int* dnsp = dalloc<int>(1, scr[k].owned, s);
    int* shell_start = dalloc<int>(S.n2max + 1, scr[k].owned, s);
    k_basis_count<<<1, 512, (S.n2max + 1) * sizeof(int), s>>>(S.n2max, S.r, g, shell_start, dnsp);
    k_basis_place<<<(ncube + 127) / 128, 128, 0, s>>>(S.n2max, S.r, S.species, shell_start, tvec,
                                                      scr[k].idx3);
    CUDA_TRY(cudaGetLastError());
    S.nsp = d2h(dnsp, 1, s)[0];
    if (S.N >= S.nsp) throw PnmError{PNM_EINVAL, "no particle states: n2max too small for N"};
    if (!twisted) {
      hvec[k] = d2h(tvec, S.nsp, s);
      auto sh = [&](const char4& c) { return c.x * c.x + c.y * c.y + c.z * c.z; };
      if (sh(hvec[k][S.N - 1]) == sh(hvec[k][S.N]))
        throw PnmError{PNM_EINVAL, "N = " + std::to_string(S.N) + " does not close a shell"};
    } else {
      double* key = dalloc<double>(S.nsp, scr[k].owned, s);
      double* skey = dalloc<double>(S.nsp, scr[k].owned, s);
      int* perm = dalloc<int>(S.nsp, scr[k].owned, s);
      char4* tv2 = dalloc<char4>(S.nsp, scr[k].owned, s);
      int nb = (S.nsp + TWIST_THREADS - 1) / TWIST_THREADS;
      k_twist_keys<<<nb, TWIST_THREADS, 0, s>>>(tvec, S.nsp, S.phi[0], S.phi[1], S.phi[2], key);
      k_twist_rank<<<nb, TWIST_THREADS, 0, s>>>(key, S.nsp, tvec, tv2, skey, perm);
      k_twist_idx3<<<(g * ncube + 255) / 256, 256, 0, s>>>(scr[k].idx3, g * ncube, perm);
      CUDA_TRY(cudaGetLastError());
      hvec[k] = d2h(tv2, S.nsp, s);
      std::vector<double> hk = d2h(skey, S.nsp, s);
      if (!(hk[S.N - 1] < hk[S.N]))
        throw PnmError{PNM_EINVAL, "system " + std::to_string(k) + ": N = " + std::to_string(S.N) +
                                       " leaves no gap at this twist (degenerate Fermi level)"};
    }
    S.sp_off = nsp_total;
    nsp_total += S.nsp;
    S.lut_off = lut_total;
    S.lut_len = 4 * S.n2max + 1;
    lut_total += S.lut_len * (S.species == 1 ? 1 : 3);  // interleaved R, T, S halves with protons
  }
  ctx->nsp_total = nsp_total;
  D.nvec = dalloc<char4>(nsp_total, ctx->owned, s);
  D.eps = dalloc<double>(nsp_total, ctx->owned, s);
  D.ekin = dalloc<double>(nsp_total, ctx->owned, s);
  D.sp_sys = dalloc<int>(nsp_total, ctx->owned, s);
  D.sp_hole = dalloc<int>(nsp_total, ctx->owned, s);
  D.lut = dalloc<double>(lut_total, ctx->owned, s);
  D.dchi = dalloc<double>(nsp_total, ctx->owned, s);
  for (int k = 0; k < nsys; k++) {
    SysInfo& S = sys[k];
    h2d(D.nvec + S.sp_off, hvec[k], s);
    if (S.species == 1)
      k_lut<<<(S.lut_len + 127) / 128, 128, 0, s>>>(D.lut + S.lut_off, S.lut_len, S.L, P.VR, P.kR,
                                                   P.VS, P.kS);
    else
      k_lut3<<<(S.lut_len + 127) / 128, 128, 0, s>>>(D.lut + S.lut_off, S.lut_len, S.L, P.VR, P.kR,
                                                    P.VT, P.kT, P.VS, P.kS);
    k_eps<<<(S.nsp + 127) / 128, 128, 0, s>>>(D.nvec + S.sp_off, D.lut + S.lut_off, S.nsp, S.N,
                                             S.L, P.hbar2_2m, S.phi[0], S.phi[1], S.phi[2],
                                             D.ekin + S.sp_off,
                                             D.eps + S.sp_off, D.sp_sys + S.sp_off,
                                             D.sp_hole + S.sp_off, k);
    CUDA_TRY(cudaGetLastError());
  }

  // ---- channel counts (GPU, every system, one copy back) and selection (host: keys with
  // both classes, ascending)
  std::vector<long> key_off(nsys + 1, 0);
  for (int k = 0; k < nsys; k++) key_off[k + 1] = key_off[k] + sys[k].nkeys;
  int* dcnt = dalloc<int>(4 * key_off[nsys], scr[0].owned, s);
  CUDA_TRY(cudaMemsetAsync(dcnt, 0, sizeof(int) * 4 * key_off[nsys], s));
  for (int k = 0; k < nsys; k++) {
    const SysInfo& S = sys[k];
    int* c = dcnt + 4 * key_off[k];
    const long npairs = (long)S.nsp * S.nsp;
    k_count_pairs<<<(unsigned)((npairs + 255) / 256), 256, 0, s>>>(D.nvec + S.sp_off, S.m, S.M, S.species, S.N,
                                                                  S.nsp, c, c + S.nkeys, c + 2 * S.nkeys,
                                                                  c + 3 * S.nkeys);
  }
  CUDA_TRY(cudaGetLastError());
  const std::vector<int> hcnt = d2h(dcnt, 4 * key_off[nsys], s);
  for (int k = 0; k < nsys; k++) {
    SysInfo& S = sys[k];
    const int* hh = hcnt.data() + 4 * key_off[k];
    const int* pp = hh + S.nkeys;
    const int* ph = hh + 2 * S.nkeys;
    const int* hp = hh + 3 * S.nkeys;
    std::vector<int> key2ch(S.nkeys, -1), key2x(S.nkeys, -1);
    for (int K = 0; K < S.nkeys; K++) {
      if (hh[K] > 0 && pp[K] > 0) {
        key2ch[K] = (int)scr[k].dkeys.size();
        scr[k].dkeys.push_back(K);
        scr[k].dnhh.push_back(hh[K]);
        scr[k].dnpp.push_back(pp[K]);
      }
      if (ph[K] > 0 && hp[K] > 0) {
        key2x[K] = (int)scr[k].xkeys.size();
        scr[k].xkeys.push_back(K);
        scr[k].xnph.push_back(ph[K]);
        scr[k].xnhp.push_back(hp[K]);
      }
    }
    scr[k].key2ch = dalloc<int>(S.nkeys, scr[k].owned, s);
    scr[k].key2x = dalloc<int>(S.nkeys, scr[k].owned, s);
    h2d(scr[k].key2ch, key2ch, s);
    h2d(scr[k].key2x, key2x, s);
  }

  // ---- channel metadata and offsets (host prefix sums over channels)
  std::vector<int> h_ch_sys, h_key, h_nhh, h_npp, h_hh_off, h_pp_off, h_vpp;
  std::vector<long> h_t_off, h_vpp_off, h_vhh_off;
  std::vector<int2> h_rows;
  std::vector<std::vector<int>> h_lad_chans(nsys);  // per system: channels with a V_pppp block
  std::vector<int> h_x_nph, h_x_nhp, h_x_ph_off, h_x_hp_off;
  std::vector<long> h_x_t_off, h_x_c_off, h_x_w_off;
  long t_acc = 0, vhh_acc = 0, xt_acc = 0, xc_acc = 0;
  int hh_acc = 0, pp_acc = 0, ph_acc = 0, hp_acc = 0;
  for (int k = 0; k < nsys; k++) {
    SysInfo& S = sys[k];
    SysScratch& X = scr[k];
    S.ch_begin = (int)h_key.size();
    S.t_begin = t_acc;
    S.row_begin = (int)h_rows.size();
    for (size_t c = 0; c < X.dkeys.size(); c++) {
      int g = (int)h_key.size();
      int K = X.dkeys[c];
      h_ch_sys.push_back(k);
      h_key.push_back(K);
      h_nhh.push_back(X.dnhh[c]);
      h_npp.push_back(X.dnpp[c]);
      h_hh_off.push_back(hh_acc);
      h_pp_off.push_back(pp_acc);
      h_t_off.push_back(t_acc);
      h_vhh_off.push_back(vhh_acc);
      // <ab|v|cd> vanishes for identical-nucleon pairs of equal spin (|S_z| = |T_z| = 2); in
      // neutron-only systems that leaves S_z = 0
      int slot = sys[k].species == 1 ? K % 3 : K % 9;
      bool has_vpp = sys[k].species == 1 ? slot == 1 : !(slot / 3 != 1 && slot % 3 != 1);
      h_vpp.push_back(has_vpp ? 1 : 0);
      if (has_vpp) h_lad_chans[k].push_back(g);
      for (int ij = 0; ij < X.dnhh[c]; ij++) h_rows.push_back(make_int2(g, ij));
      hh_acc += X.dnhh[c];
      pp_acc += X.dnpp[c];
      t_acc += (long)X.dnhh[c] * X.dnpp[c];
      vhh_acc += (long)X.dnhh[c] * X.dnhh[c];
    }
    S.ch_end = (int)h_key.size();
    S.t_end = t_acc;
    S.row_end = (int)h_rows.size();
    S.x_begin = (int)h_x_nph.size();
    for (size_t x = 0; x < X.xkeys.size(); x++) {
      h_x_nph.push_back(X.xnph[x]);
      h_x_nhp.push_back(X.xnhp[x]);
      h_x_ph_off.push_back(ph_acc);
      h_x_hp_off.push_back(hp_acc);
      h_x_t_off.push_back(xt_acc);
      h_x_c_off.push_back(xc_acc);
      h_x_w_off.push_back(xt_acc);  // W_x has n_hp x n_ph entries, as many as T_x
      ph_acc += X.xnph[x];
      hp_acc += X.xnhp[x];
      xt_acc += (long)X.xnph[x] * X.xnhp[x];
      xc_acc += (long)X.xnhp[x] * X.xnhp[x];
    }
    S.x_end = (int)h_x_nph.size();
  }
  if (t_acc >= (1L << 31) - 2 || xt_acc >= (1L << 31) - 2)
    throw PnmError{PNM_EINVAL, "problem too large for 32-bit element maps"};
  ctx->nch = (int)h_key.size();
  ctx->nx = (int)h_x_nph.size();
  ctx->nt = t_acc;
  ctx->nvhh = vhh_acc;
  ctx->nxt = xt_acc;
  ctx->nxc = xc_acc;
  ctx->nrows = (int)h_rows.size();
  ctx->n_hh_pairs = hh_acc;
  ctx->n_pp_pairs = pp_acc;
  ctx->h_ch_sys = h_ch_sys;
  ctx->h_key = h_key;
  ctx->h_nhh = h_nhh;
  ctx->h_npp = h_npp;
  ctx->h_t_off = h_t_off;
  ctx->h_vpp = h_vpp;
  ctx->h_rows = h_rows;
  ctx->h_x_nph = h_x_nph;
  ctx->h_x_nhp = h_x_nhp;
  ctx->h_x_t_off = h_x_t_off;
  ctx->h_x_ph_off = h_x_ph_off;
  ctx->h_x_hp_off = h_x_hp_off;
  ctx->h_hh_off = h_hh_off;
  ctx->h_pp_off = h_pp_off;

  int C = ctx->nch, NX = ctx->nx;
  D.ch_sys = dalloc<int>(C, ctx->owned, s);
  D.ch_key = dalloc<int>(C, ctx->owned, s);
  D.ch_nhh = dalloc<int>(C, ctx->owned, s);
  D.ch_npp = dalloc<int>(C, ctx->owned, s);
  D.ch_hh_off = dalloc<int>(C, ctx->owned, s);
  D.ch_pp_off = dalloc<int>(C, ctx->owned, s);
  D.ch_vpp = dalloc<int>(C, ctx->owned, s);
  D.ch_t_off = dalloc<long>(C, ctx->owned, s);
  D.ch_vpp_off = dalloc<long>(C, ctx->owned, s);  // ladder V blocks, set once the basis is known
  D.ch_nlad = dalloc<int>(C, ctx->owned, s);
  D.ch_s_off = dalloc<long>(C, ctx->owned, s);
  D.ch_vhh_off = dalloc<long>(C, ctx->owned, s);
  D.row_item = dalloc<int2>(ctx->nrows, ctx->owned, s);
  D.x_nph = dalloc<int>(NX, ctx->owned, s);
  D.x_sys = dalloc<int>(NX, ctx->owned, s);
  D.x_nhp = dalloc<int>(NX, ctx->owned, s);
  D.x_ph_off = dalloc<int>(NX, ctx->owned, s);
  D.x_hp_off = dalloc<int>(NX, ctx->owned, s);
  D.x_t_off = dalloc<long>(NX, ctx->owned, s);
  D.x_c_off = dalloc<long>(NX, ctx->owned, s);
  D.x_w_off = dalloc<long>(NX, ctx->owned, s);
  h2d(D.ch_sys, h_ch_sys, s);
  {
    std::vector<int> h_x_sys(NX);
    for (int k = 0; k < nsys; k++)
      for (int x = ctx->sys[k].x_begin; x < ctx->sys[k].x_end; x++) h_x_sys[x] = k;
    h2d(D.x_sys, h_x_sys, s);
  }
  h2d(D.ch_key, h_key, s);
  h2d(D.ch_nhh, h_nhh, s);
  h2d(D.ch_npp, h_npp, s);
  h2d(D.ch_hh_off, h_hh_off, s);
  h2d(D.ch_pp_off, h_pp_off, s);
  h2d(D.ch_vpp, h_vpp, s);
  h2d(D.ch_t_off, h_t_off, s);
  h2d(D.ch_vhh_off, h_vhh_off, s);
  h2d(D.row_item, h_rows, s);
  h2d(D.x_nph, h_x_nph, s);
  h2d(D.x_nhp, h_x_nhp, s);
  h2d(D.x_ph_off, h_x_ph_off, s);
  h2d(D.x_hp_off, h_x_hp_off, s);
  h2d(D.x_t_off, h_x_t_off, s);
  h2d(D.x_c_off, h_x_c_off, s);
  h2d(D.x_w_off, h_x_w_off, s);

  D.hh_pair = dalloc<int2>(hh_acc, ctx->owned, s);
  D.pp_pair = dalloc<int2>(pp_acc, ctx->owned, s);
  D.ph_pair = dalloc<int2>(ph_acc, ctx->owned, s);
  D.hp_pair = dalloc<int2>(hp_acc, ctx->owned, s);
  D.x_cls = dalloc<int>(NX, ctx->owned, s);
  D.x_rrow = dalloc<int>(ph_acc, ctx->owned, s);
  D.x_fcol = dalloc<int>(hp_acc, ctx->owned, s);
  D.x_rcol = dalloc<int>(hp_acc, ctx->owned, s);
  D.fmap = dalloc<int>(t_acc, ctx->owned, s);
  int* flip_err = dalloc<int>(1, ctx->owned, s);
  CUDA_TRY(cudaMemsetAsync(flip_err, 0, sizeof(int), s));
  D.xmap = dalloc<int>(xt_acc, ctx->owned, s);
  D.qmap = dalloc<int4>(t_acc, ctx->owned, s);
  D.v_pphh = dalloc<double>(t_acc, ctx->owned, s);
  D.den = dalloc<double>(t_acc, ctx->owned, s);
  D.inv_den = dalloc<double>(t_acc, ctx->owned, s);
  D.lad_map = dalloc<int>(pp_acc, ctx->owned, s);
  D.lad_mem = dalloc<int2>(pp_acc, ctx->owned, s);
  D.v_hhhh = dalloc<double>(vhh_acc, ctx->owned, s);
  D.x_v1 = dalloc<double>(xc_acc, ctx->owned, s);
  D.x_w = dalloc<double>(xt_acc, ctx->owned, s);
  D.t0 = dalloc<double>(t_acc, ctx->owned, s);
  D.t1 = dalloc<double>(t_acc, ctx->owned, s);
  D.chi_hh = dalloc<double>(vhh_acc, ctx->owned, s);
  D.sab = dalloc<double>(pp_acc, ctx->owned, s);
  D.sij = dalloc<double>(hh_acc, ctx->owned, s);
  D.xq = dalloc<double>(xt_acc, ctx->owned, s);
  D.occ_off = dalloc<int>(nsp_total + 1, ctx->owned, s);

  // ---- pair lists, maps, V blocks per system
  std::vector<int> h_occ_off(nsp_total + 1, 0);
  int* occ_cnt = dalloc<int>(std::max(nsp_total, 1), scr[0].owned, s);
  for (int k = 0; k < nsys; k++) {
    SysInfo& S = sys[k];
    SysScratch& X = scr[k];
    int np = S.nsp - S.N;
    X.pos_hh = dalloc<int>((size_t)S.N * S.N, X.owned, s);
    X.pos_pp = dalloc<int>((size_t)np * np, X.owned, s);
    X.phpos = dalloc<int>((size_t)np * S.N, X.owned, s);
    X.phch = dalloc<int>((size_t)np * S.N, X.owned, s);
    X.hppos = dalloc<int>((size_t)S.N * np, X.owned, s);
    CUDA_TRY(cudaMemsetAsync(X.phch, 0xff, sizeof(int) * (size_t)np * S.N, s));
    int nchs = S.ch_end - S.ch_begin, nxs = S.x_end - S.x_begin;
    if (nchs > 0)
      k_fill_direct<<<(nchs * 32 + 255) / 256, 256, 0, s>>>(
          D.nvec + S.sp_off, X.idx3, S.r, S.m, S.M, S.species, S.N, S.nsp, S.sp_off, nchs,
          D.ch_key + S.ch_begin, D.ch_hh_off + S.ch_begin, D.ch_pp_off + S.ch_begin, D.hh_pair,
          D.pp_pair, X.pos_hh, X.pos_pp);
    if (nxs > 0) {
      int* xk = dalloc<int>(nxs, X.owned, s);
      h2d(xk, X.xkeys, s);
      k_fill_cross<<<(nxs * 32 + 255) / 256, 256, 0, s>>>(
          D.nvec + S.sp_off, X.idx3, S.r, S.m, S.M, S.species, S.N, S.nsp, S.sp_off, nxs, xk,
          D.x_ph_off + S.x_begin, D.x_hp_off + S.x_begin, D.ph_pair, D.hp_pair, X.phpos, X.phch,
          X.hppos);
      k_xmap<<<nxs, 256, 0, s>>>(S.x_begin, D.x_nph, D.x_nhp, D.x_t_off, D.x_ph_off, D.x_hp_off,
                                 D.ph_pair, D.hp_pair, D.nvec, S.sp_off, S.N, S.nsp, S.m, S.M,
                                 S.species, X.key2ch, S.ch_begin, D.ch_t_off, D.ch_npp, X.pos_hh, X.pos_pp,
                                 D.xmap);
      k_xflip<<<(nxs * 32 + 255) / 256, 256, 0, s>>>(S.x_begin, nxs, D.x_nph, D.x_nhp, D.x_ph_off, D.x_hp_off,
                                                D.ph_pair, D.hp_pair, D.nvec, X.idx3, S.r, S.species,
                                                S.sp_off, S.N, S.nsp, X.phpos, X.phch, X.hppos, D.x_cls,
                                                D.x_fcol, D.x_rrow, D.x_rcol, flip_err);
      k_v_cross<<<nxs, 256, 0, s>>>(S.x_begin, D.x_nph, D.x_nhp, D.x_c_off, D.x_w_off,
                                    D.x_ph_off, D.x_hp_off, D.ph_pair, D.hp_pair, D.nvec,
                                    D.lut + S.lut_off, D.x_v1, D.x_w);
    }
    int nrows = S.row_end - S.row_begin;
    if (nrows > 0) {
      k_qmap<<<nrows, 128, 0, s>>>(S.row_begin, D.row_item, D.ch_hh_off, D.ch_pp_off, D.ch_npp,
                                   D.ch_t_off, D.hh_pair, D.pp_pair, S.sp_off, S.N, S.nsp,
                                   X.phch, X.phpos, X.hppos, S.x_begin, D.x_t_off, D.x_nhp,
                                   D.x_cls, D.nvec, X.idx3, S.r, S.species, D.qmap);
      k_fmap<<<nrows, 128, 0, s>>>(S.row_begin, D.row_item, D.ch_hh_off, D.ch_pp_off, D.ch_npp, D.ch_t_off,
                                   D.hh_pair, D.pp_pair, D.nvec, X.idx3, S.r, S.species, S.sp_off, S.N,
                                   S.nsp, S.m, S.M, X.key2ch, S.ch_begin, X.pos_hh, X.pos_pp, D.fmap,
                                   flip_err);
      k_v_pphh<<<nrows, 128, 0, s>>>(S.row_begin, D.row_item, D.ch_hh_off, D.ch_pp_off, D.ch_npp,
                                     D.ch_t_off, D.hh_pair, D.pp_pair, D.nvec, D.lut + S.lut_off,
                                     D.v_pphh);
      k_den<<<nrows, 128, 0, s>>>(S.row_begin, D.row_item, D.ch_hh_off, D.ch_pp_off, D.ch_npp, D.ch_t_off,
                                  D.hh_pair, D.pp_pair, D.eps, D.den, D.inv_den);
    }
    if (nchs > 0)
      k_v_hhhh<<<nchs, 128, 0, s>>>(S.ch_begin, D.ch_hh_off, D.ch_nhh, D.ch_vhh_off, D.hh_pair,
                                    D.nvec, D.lut + S.lut_off, D.v_hhhh);
    CUDA_TRY(cudaGetLastError());
    // pairs containing each state (counted for every system, copied back once below)
    int ob = (S.nsp * 32 + 255) / 256;
    k_occ<<<ob, 256, 0, s>>>(0, D.nvec, S.sp_off, S.N, S.nsp, S.m, S.M, S.species, X.key2ch, S.ch_begin,
                             D.ch_hh_off, D.ch_pp_off, X.pos_hh, X.pos_pp, occ_cnt + S.sp_off, nullptr, nullptr);
  }
  {
    const std::vector<int> hc = d2h(occ_cnt, nsp_total, s);
    for (int p = 0; p < nsp_total; p++) h_occ_off[p + 1] = h_occ_off[p] + hc[p];
  }
  h2d(D.occ_off, h_occ_off, s);
  D.occ_idx = dalloc<int>(h_occ_off[nsp_total], ctx->owned, s);
  for (int k = 0; k < nsys; k++) {
    SysInfo& S = sys[k];
    SysScratch& X = scr[k];
    int ob = (S.nsp * 32 + 255) / 256;
    k_occ<<<ob, 256, 0, s>>>(1, D.nvec, S.sp_off, S.N, S.nsp, S.m, S.M, S.species, X.key2ch, S.ch_begin,
                             D.ch_hh_off, D.ch_pp_off, X.pos_hh, X.pos_pp, nullptr, D.occ_off,
                             D.occ_idx);
  }
  // ---- ladder basis of the pp ladder (pairs and the partner table of each system are ready)
  CUDA_TRY(cudaMemsetAsync(D.ch_nlad, 0, sizeof(int) * std::max(C, 1), s));
  int max_npp = 0;
  for (int c = 0; c < C; c++)
    if (h_vpp[c]) max_npp = std::max(max_npp, h_npp[c]);
  size_t lsm = 3 * sizeof(int) * (size_t)max_npp;
  if (lsm > 200 * 1024) throw PnmError{PNM_EINVAL, "channel too large for the ladder basis"};
  smem_at_least(k_ladder_basis, lsm);
  for (int k = 0; k < nsys; k++) {
    if (h_lad_chans[k].empty()) continue;
    SysInfo& S = sys[k];
    int* lc = dalloc<int>(h_lad_chans[k].size(), scr[k].owned, s);
    h2d(lc, h_lad_chans[k], s);
    k_ladder_basis<<<(unsigned)h_lad_chans[k].size(), LAD_THREADS, lsm, s>>>(
        lc, S.species, D.ch_pp_off, D.ch_npp, D.pp_pair, D.nvec, S.N, S.nsp, S.r, scr[k].idx3,
        scr[k].pos_pp, D.lad_map, D.lad_mem, D.ch_nlad);
    CUDA_TRY(cudaGetLastError());
  }
  std::vector<int> h_nlad = d2h(D.ch_nlad, C, s);
  if (d2h(flip_err, 1, s)[0]) throw PnmError{PNM_EINVAL, "spin-flip tables not closed (reference not spin saturated)"};
  ctx->h_x_cls = d2h(D.x_cls, NX, s);
  std::vector<long> h_s_off(C, 0), h_vl_off(C, -1);
  long s_acc = 0, vl_acc = 0;
  int max_nlad = 0;
  std::vector<int2> vl_items;
  for (int c = 0; c < C; c++) {
    h_s_off[c] = s_acc;
    if (!h_vpp[c]) continue;
    h_vl_off[c] = vl_acc;
    s_acc += (long)h_nhh[c] * h_nlad[c];
    vl_acc += (long)h_nlad[c] * h_nlad[c];
    max_nlad = std::max(max_nlad, h_nlad[c]);
    for (int r0 = 0; r0 < h_nlad[c]; r0 += VLAD_ROWS) vl_items.push_back(make_int2(c, r0));
  }
  ctx->h_nlad = h_nlad;
  ctx->h_s_off = h_s_off;
  ctx->h_vl_off = h_vl_off;
  ctx->ns = s_acc;
  ctx->nvpp = vl_acc;
  h2d(D.ch_s_off, h_s_off, s);
  h2d(D.ch_vpp_off, h_vl_off, s);
  D.v_pppp = nullptr;  // the ladder V is built on first use, in the representation a path needs
  D.rpp = dalloc<double>(s_acc, ctx->owned, s);
  D.s64 = dalloc<double>(s_acc, ctx->owned, s);
  // work list of the ladder V (one launch per system: the LUT differs per system), kept for
  // pnm_ladder_v
  ctx->vl_sys.assign(nsys + 1, 0);
  if (!vl_items.empty()) {
    int max_lut = 0;
    for (const SysInfo& S : sys) max_lut = std::max(max_lut, S.lut_len * (S.species == 1 ? 1 : 3));
    size_t smem = sizeof(double) * max_lut + (2 * sizeof(char4) + sizeof(int)) * (size_t)max_nlad;
    if (smem > 200 * 1024) throw PnmError{PNM_EINVAL, "channel too large for the staged ladder V"};
    ctx->vl_smem = smem;
    ctx->vl_items = dalloc<int2>(vl_items.size(), ctx->owned, s);
    h2d(ctx->vl_items, vl_items, s);
    size_t lo = 0;
    for (int k = 0; k < nsys; k++) {
      size_t hi = lo;
      while (hi < vl_items.size() && h_ch_sys[vl_items[hi].x] == k) hi++;
      ctx->vl_sys[k + 1] = (int)hi;
      lo = hi;
    }
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(s));
}
