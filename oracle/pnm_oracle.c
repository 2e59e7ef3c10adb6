/*
 * pnm_oracle.c -- plain, slow, FP64 CPU oracle for coupled-cluster doubles (CCD)
 * in pure neutron matter with the Minnesota interaction.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code, header, table or
 * constant generator with the CUDA library; neither includes nor links the other.
 *
 * What it follows (the paper is Lietz, Novario, Jansen, Hagen, Hjorth-Jensen,
 * "Computational Nuclear Physics and Post Hartree-Fock Methods", arXiv:1611.06765):
 *   basis        Sec. "Single-particle basis for infinite matter" (k = 2 pi n / L,
 *                L^3 = N/rho, eps = hbar^2 k^2/2m, closed shells, Table tab:table1) and
 *                the shell-ordered state loop of Sec. "Developing a CCD code".
 *   interaction  Sec. "Two-body interaction": Minnesota V(r) with the spin/isospin
 *                exchange form and its momentum-space Gaussian (Table tab:minnesotatab).
 *   f, E_ref     Eq. (Hnormalorder) and the E_Ref expression above it:
 *                f_pq = h0_pq + sum_i <pi|v|qi>,  E_ref = sum_i h0_ii + 1/2 sum_ij <ij|v|ij>.
 *   MBPT2        Eq. (ccdGuess) and the energy below it.
 *   CCD          Eq. (ccd3) (Jacobi form of Eq. ccd2b) written with the intermediates
 *                chi_b^c, chi_k^j, chi_kl^ij, chi_kb^cj, chi_ab^cd of Sec. "Developing a CCD
 *                code", blocked in direct (T) and cross (X) channels as in the channel
 *                mapping that follows them; energy Eq. (ccdcorr); mixing
 *                t = alpha t_new + (1-alpha) t_old; stop when |dE^(n+1) - dE^(n)| < eta.
 *   truncations  Eq. (ccd1) (pp ladder only) and Eq. (ccd2) (pp and hh ladders) of Sec.
 *                "Coupled cluster theory", and the terms of Eq. (ccd3) linear in t.
 *   MBPT3        diagrams (3), (4), (5) of Fig. goldstone, Eqs. (diag3)-(diag5).
 *   nuclear      protons and neutrons (Sec. "Infinite nuclear matter"): the full Minnesota
 *   matter       operator in the 16-dimensional two-nucleon spin-isospin space, V_T active for
 *                np pairs, channels keyed by (P, S_z, T_z).
 *
 * Readings of the paper taken here (each one is listed with its evidence in the design notes):
 *   - Minnesota signs: V_R = +200 MeV, V_T = -178 MeV, V_S = -91.85 MeV (the table prints
 *     magnitudes only).  The kappa_alpha of the table is the alpha of the Gaussian.
 *   - Single-particle energies in the denominators are the HF energies eps_p = f_pp.
 *   - The channel index of Sec. "Developing a CCD code" is not injective as printed; this
 *     file uses the mixed-radix key ((Px+m)M + (Py+m))M + (Pz+m)) * 3 + (Sz+2)/2 with
 *     m = 2 floor(sqrt(n2max)), M = 2m+1 and spins in units of hbar/2.
 *   - State order: shells ascending, then nx, ny, nz ascending, then s = -1 before +1;
 *     the first N states are holes.  Pairs inside a channel are in lexicographic order.
 *   - Twisted boundary conditions (Sec. "Twist-averaged boundary conditions"): k = (2 pi n +
 *     theta)/L, so eps_kin = hbar^2/2m (2 pi/L)^2 |n + phi|^2 with phi = theta/(2 pi) per axis
 *     (the paper's printed shift of eps_k is garbled; this is |k + theta/L|^2 written out).
 *     The model space stays n^2 <= n2max.  States are reordered by |n + phi|^2 (ties kept in
 *     the order above) and the first N are the holes, as the paper's "order states by energy
 *     and fill holes".  |n + phi|^2 is summed over the three axes in ascending order of the
 *     axis terms, so twists with equal components give bit-identical energies to states that
 *     differ by a permutation; N must leave a gap: |n + phi|^2 of state N-1 below that of N.
 *   - Direct-channel blocks of t and v are stored for restricted pairs (p<q); a sum
 *     1/2 sum_{cd} over ordered pairs of a pair-antisymmetric product equals sum_{c<d}.
 *     Cross-channel blocks use ordered pairs, as the paper's X channels do.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OM_PI 3.14159265358979323846

typedef struct {
    double VR, kR, VT, kT, VS, kS, hbar2_2m;
} om_minnesota;

typedef struct om_sys {
    int N, nsp, n2max, m, M;         /* N: particles (holes) of every species together */
    double rho, L;
    double phi[3];                   /* twist theta / (2 pi) per axis; 0 = periodic */
    om_minnesota P;
    int species;                     /* 1 neutrons, 2 protons, 3 both (nuclear matter) */
    int nq;                          /* charge slots of a channel key: 3 (S_z) or 9 (S_z, T_z) */
    int *nx, *ny, *nz, *sz, *tz;     /* sz, tz in units of 1/2: -1 or +1 (tz +1 neutron) */
    double *ekin, *eps;              /* kinetic and HF single-particle energies */
    double Ospin[3][16][16];         /* spin-isospin operators of the R, T, S terms */

    /* direct channels: those with both restricted hh and pp pairs */
    int nch;
    int *chkey, *nhh, *npp, *hh_off, *pp_off;
    int *hh_p, *hh_q, *pp_p, *pp_q;  /* restricted pairs, channel-major, lexicographic */
    size_t *t_off, nt;               /* t block per channel: npp x nhh (pp rows) */
    size_t *vpp_off, nvpp;           /* <ab|v|cd> block: npp x npp */
    size_t *vhh_off, nvhh;           /* <kl|v|ij> block: nhh x nhh */
    int *pair_ch, *pair_pos;         /* (p,q), p<q -> channel (or -1) and position */

    /* cross channels for the particle-hole term */
    int nx_ch;
    int *xkey, *nph, *nhp, *ph_off, *hp_off;
    int *ph_a, *ph_i, *hp_k, *hp_c;  /* (a,i) rows, (k,c) columns, lexicographic */
    size_t *xt_off, nxt;             /* T_d and Q_d: nph x nhp */
    size_t *xc_off, nxc;             /* V1_d and C_d: nhp x nhp */
    size_t *xw_off, nxw;             /* W_d: nhp x nph */
    int *phx_ch, *phx_pos;           /* (a,i) -> cross channel, row   (index a*N+i) */
    int *hpx_ch, *hpx_pos;           /* (k,c) -> cross channel, column (index k*nsp+c) */

    /* blocks */
    double *v_pphh, *v_pppp, *v_hhhh, *x_v1, *x_w;
    double *t;                       /* amplitudes, layout of v_pphh */
    int have_ccd_blocks;
} om_sys;

/* ------------------------------------------------------------------------ basis */

static int isqrt_floor(int x) {
    int r = (int)floor(sqrt((double)x));
    while (r * r > x) r--;
    while ((r + 1) * (r + 1) <= x) r++;
    return r;
}

/* Shell-ordered enumeration of plane-wave states with n^2 <= n2max; per momentum s = -1
 * then +1 and, within a spin, the species present (proton t = -1 before neutron t = +1). */
static int build_basis(om_sys *S) {
    int r = isqrt_floor(S->n2max);
    int cap = 4 * (2 * r + 1) * (2 * r + 1) * (2 * r + 1);
    S->nx = malloc(sizeof(int) * cap);
    S->ny = malloc(sizeof(int) * cap);
    S->nz = malloc(sizeof(int) * cap);
    S->sz = malloc(sizeof(int) * cap);
    S->tz = malloc(sizeof(int) * cap);
    int n = 0;
    for (int shell = 0; shell <= S->n2max; shell++)
        for (int x = -r; x <= r; x++)
            for (int y = -r; y <= r; y++)
                for (int z = -r; z <= r; z++)
                    for (int s = -1; s <= 1; s += 2)
                        for (int t = -1; t <= 1; t += 2)
                            if (x * x + y * y + z * z == shell &&
                                (S->species & (t > 0 ? 1 : 2))) {
                                S->nx[n] = x; S->ny[n] = y; S->nz[n] = z; S->sz[n] = s;
                                S->tz[n] = t;
                                n++;
                            }
    S->nsp = n;
    return n;
}

/* |n + phi|^2 with the three axis terms added in ascending order. */
static double twisted_n2(const om_sys *S, int p) {
    double a[3] = {(S->nx[p] + S->phi[0]) * (S->nx[p] + S->phi[0]),
                   (S->ny[p] + S->phi[1]) * (S->ny[p] + S->phi[1]),
                   (S->nz[p] + S->phi[2]) * (S->nz[p] + S->phi[2])};
    for (int i = 0; i < 3; i++)
        for (int j = i + 1; j < 3; j++)
            if (a[j] < a[i]) { double x = a[i]; a[i] = a[j]; a[j] = x; }
    return (a[0] + a[1]) + a[2];
}

typedef struct { double key; int idx; } om_rank;

static int rank_cmp(const void *x, const void *y) {
    const om_rank *a = x, *b = y;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/* Stable reorder of the shell-ordered states by |n + phi|^2; returns the sorted keys. */
static double *order_by_energy(om_sys *S) {
    size_t n = S->nsp > 0 ? (size_t)S->nsp : 1;
    om_rank *r = malloc(sizeof(om_rank) * n);
    for (int p = 0; p < (int)n; p++) { r[p].key = twisted_n2(S, p); r[p].idx = p; }
    qsort(r, n, sizeof(om_rank), rank_cmp);
    int *tmp = malloc(sizeof(int) * 5 * n);
    for (int p = 0; p < (int)n; p++) {
        int q = r[p].idx;
        tmp[5 * p] = S->nx[q]; tmp[5 * p + 1] = S->ny[q];
        tmp[5 * p + 2] = S->nz[q]; tmp[5 * p + 3] = S->sz[q]; tmp[5 * p + 4] = S->tz[q];
    }
    double *key = malloc(sizeof(double) * n);
    for (int p = 0; p < (int)n; p++) {
        S->nx[p] = tmp[5 * p]; S->ny[p] = tmp[5 * p + 1];
        S->nz[p] = tmp[5 * p + 2]; S->sz[p] = tmp[5 * p + 3]; S->tz[p] = tmp[5 * p + 4];
        key[p] = r[p].key;
    }
    free(tmp);
    free(r);
    return key;
}

/* ------------------------------------------------------------- Minnesota force */

/* Two-particle spin-isospin space: one particle's label l = 2u + w with u = (s+1)/2 and
 * w = (t+1)/2; the pair's index is 4 l1 + l2.  The exchange operators swap the spin labels
 * (P_s) or the isospin labels (P_t) of the two particles.  The operators multiplying the three
 * radial Gaussians are, from V(r) = 1/2 (V_R + 1/2(1+Ps) V_T + 1/2(1-Ps) V_S)(1 - Ps Pt):
 *   O_R = 1/2 (1 - Ps Pt),  O_T = 1/4 (1 + Ps)(1 - Ps Pt),  O_S = 1/4 (1 - Ps)(1 - Ps Pt).
 * For two neutrons P_t = 1 on every pair state, and O_T vanishes. */
#define OM_SD 16
static void matmul16(double A[OM_SD][OM_SD], double B[OM_SD][OM_SD], double C[OM_SD][OM_SD]) {
    for (int i = 0; i < OM_SD; i++)
        for (int j = 0; j < OM_SD; j++) {
            double acc = 0;
            for (int k = 0; k < OM_SD; k++) acc += A[i][k] * B[k][j];
            C[i][j] = acc;
        }
}

static void build_spin_ops(om_sys *S) {
    static double I[OM_SD][OM_SD], Ps[OM_SD][OM_SD], Pt[OM_SD][OM_SD];
    memset(I, 0, sizeof(I)); memset(Ps, 0, sizeof(Ps)); memset(Pt, 0, sizeof(Pt));
    for (int u1 = 0; u1 < 2; u1++)
        for (int w1 = 0; w1 < 2; w1++)
            for (int u2 = 0; u2 < 2; u2++)
                for (int w2 = 0; w2 < 2; w2++) {
                    int ket = 4 * (2 * u1 + w1) + (2 * u2 + w2);
                    I[ket][ket] = 1.0;
                    Ps[4 * (2 * u2 + w1) + (2 * u1 + w2)][ket] = 1.0;  /* |u2 w1, u1 w2> */
                    Pt[4 * (2 * u1 + w2) + (2 * u2 + w1)][ket] = 1.0;  /* |u1 w2, u2 w1> */
                }
    double PsPt[OM_SD][OM_SD], A[OM_SD][OM_SD], X[OM_SD][OM_SD], Y[OM_SD][OM_SD];
    matmul16(Ps, Pt, PsPt);
    for (int i = 0; i < OM_SD; i++)
        for (int j = 0; j < OM_SD; j++) A[i][j] = I[i][j] - PsPt[i][j];   /* 1 - Ps Pt */
    for (int i = 0; i < OM_SD; i++)
        for (int j = 0; j < OM_SD; j++) S->Ospin[0][i][j] = 0.5 * A[i][j];
    for (int i = 0; i < OM_SD; i++)
        for (int j = 0; j < OM_SD; j++) X[i][j] = 0.5 * (I[i][j] + Ps[i][j]);
    matmul16(X, A, Y);
    for (int i = 0; i < OM_SD; i++)
        for (int j = 0; j < OM_SD; j++) S->Ospin[1][i][j] = 0.5 * Y[i][j];
    for (int i = 0; i < OM_SD; i++)
        for (int j = 0; j < OM_SD; j++) X[i][j] = 0.5 * (I[i][j] - Ps[i][j]);
    matmul16(X, A, Y);
    for (int i = 0; i < OM_SD; i++)
        for (int j = 0; j < OM_SD; j++) S->Ospin[2][i][j] = 0.5 * Y[i][j];
}

static int label(const om_sys *S, int p) { return 2 * ((S->sz[p] + 1) / 2) + (S->tz[p] + 1) / 2; }

/* Momentum-space Gaussian: (V_a / L^3) (pi / kappa)^{3/2} exp(-q^2 / (4 kappa)). */
static double gauss_ft(const om_sys *S, double V, double kappa, double q2) {
    double L3 = S->L * S->L * S->L;
    return V / L3 * pow(OM_PI / kappa, 1.5) * exp(-q2 / (4.0 * kappa));
}

/* Direct (not antisymmetrized) element <pq|V|rs>. */
static double v_direct(const om_sys *S, int p, int q, int r, int s) {
    if (S->nx[p] + S->nx[q] != S->nx[r] + S->nx[s]) return 0.0;
    if (S->ny[p] + S->ny[q] != S->ny[r] + S->ny[s]) return 0.0;
    if (S->nz[p] + S->nz[q] != S->nz[r] + S->nz[s]) return 0.0;
    int bra = 4 * label(S, p) + label(S, q);
    int ket = 4 * label(S, r) + label(S, s);
    double oR = S->Ospin[0][bra][ket], oT = S->Ospin[1][bra][ket], oS = S->Ospin[2][bra][ket];
    if (oR == 0.0 && oT == 0.0 && oS == 0.0) return 0.0;
    /* relative-momentum transfer q = 1/2 (k_p - k_q - k_r + k_s), k = 2 pi n / L */
    double f = OM_PI / S->L;
    double qx = f * (S->nx[p] - S->nx[q] - S->nx[r] + S->nx[s]);
    double qy = f * (S->ny[p] - S->ny[q] - S->ny[r] + S->ny[s]);
    double qz = f * (S->nz[p] - S->nz[q] - S->nz[r] + S->nz[s]);
    double q2 = qx * qx + qy * qy + qz * qz;
    double v = 0.0;
    v += oR * gauss_ft(S, S->P.VR, S->P.kR, q2);
    v += oT * gauss_ft(S, S->P.VT, S->P.kT, q2);
    v += oS * gauss_ft(S, S->P.VS, S->P.kS, q2);
    return v;
}

/* Antisymmetrized element <pq|v|rs> = <pq|V|rs> - <pq|V|sr>. */
double om_v(const om_sys *S, int p, int q, int r, int s) {
    return v_direct(S, p, q, r, s) - v_direct(S, p, q, s, r);
}

/* ------------------------------------------------------------------- channels */

/* Pure neutron matter: ((Px+m)M + Py+m)M + Pz+m, times 3 plus (Sz+2)/2.  With protons the
 * charge slot is 3 (Sz+2)/2 + (Tz+2)/2 of 9. */
static int chan_key(const om_sys *S, int Px, int Py, int Pz, int Sz, int Tz) {
    int m = S->m, M = S->M;
    int slot = S->nq == 3 ? (Sz + 2) / 2 : 3 * ((Sz + 2) / 2) + (Tz + 2) / 2;
    return (((Px + m) * M + (Py + m)) * M + (Pz + m)) * S->nq + slot;
}

static int dir_key(const om_sys *S, int p, int q) {
    return chan_key(S, S->nx[p] + S->nx[q], S->ny[p] + S->ny[q], S->nz[p] + S->nz[q],
                    S->sz[p] + S->sz[q], S->tz[p] + S->tz[q]);
}

static int cross_key(const om_sys *S, int p, int q) {
    return chan_key(S, S->nx[p] - S->nx[q], S->ny[p] - S->ny[q], S->nz[p] - S->nz[q],
                    S->sz[p] - S->sz[q], S->tz[p] - S->tz[q]);
}

static void build_direct_channels(om_sys *S) {
    int N = S->N, n = S->nsp;
    int nkeys = S->M * S->M * S->M * S->nq;
    int *cnt_hh = calloc(nkeys, sizeof(int)), *cnt_pp = calloc(nkeys, sizeof(int));
    for (int i = 0; i < N; i++)
        for (int j = i + 1; j < N; j++) cnt_hh[dir_key(S, i, j)]++;
    for (int a = N; a < n; a++)
        for (int b = a + 1; b < n; b++) cnt_pp[dir_key(S, a, b)]++;
    int *key2ch = malloc(sizeof(int) * nkeys);
    S->nch = 0;
    for (int k = 0; k < nkeys; k++) {
        key2ch[k] = -1;
        if (cnt_hh[k] > 0 && cnt_pp[k] > 0) key2ch[k] = S->nch++;
    }
    int C = S->nch;
    S->chkey = malloc(sizeof(int) * C);
    S->nhh = calloc(C, sizeof(int));
    S->npp = calloc(C, sizeof(int));
    S->hh_off = malloc(sizeof(int) * (C + 1));
    S->pp_off = malloc(sizeof(int) * (C + 1));
    for (int k = 0; k < nkeys; k++)
        if (key2ch[k] >= 0) {
            S->chkey[key2ch[k]] = k;
            S->nhh[key2ch[k]] = cnt_hh[k];
            S->npp[key2ch[k]] = cnt_pp[k];
        }
    S->hh_off[0] = S->pp_off[0] = 0;
    for (int c = 0; c < C; c++) {
        S->hh_off[c + 1] = S->hh_off[c] + S->nhh[c];
        S->pp_off[c + 1] = S->pp_off[c] + S->npp[c];
    }
    S->hh_p = malloc(sizeof(int) * (S->hh_off[C] + 1));
    S->hh_q = malloc(sizeof(int) * (S->hh_off[C] + 1));
    S->pp_p = malloc(sizeof(int) * (S->pp_off[C] + 1));
    S->pp_q = malloc(sizeof(int) * (S->pp_off[C] + 1));
    S->pair_ch = malloc(sizeof(int) * (size_t)n * n);
    S->pair_pos = malloc(sizeof(int) * (size_t)n * n);
    for (size_t x = 0; x < (size_t)n * n; x++) S->pair_ch[x] = -1, S->pair_pos[x] = -1;
    int *fill = calloc(C, sizeof(int));
    for (int i = 0; i < N; i++)
        for (int j = i + 1; j < N; j++) {
            int c = key2ch[dir_key(S, i, j)];
            if (c < 0) continue;
            int pos = fill[c]++;
            S->hh_p[S->hh_off[c] + pos] = i;
            S->hh_q[S->hh_off[c] + pos] = j;
            S->pair_ch[(size_t)i * n + j] = c;
            S->pair_pos[(size_t)i * n + j] = pos;
        }
    memset(fill, 0, sizeof(int) * C);
    for (int a = N; a < n; a++)
        for (int b = a + 1; b < n; b++) {
            int c = key2ch[dir_key(S, a, b)];
            if (c < 0) continue;
            int pos = fill[c]++;
            S->pp_p[S->pp_off[c] + pos] = a;
            S->pp_q[S->pp_off[c] + pos] = b;
            S->pair_ch[(size_t)a * n + b] = c;
            S->pair_pos[(size_t)a * n + b] = pos;
        }
    S->t_off = malloc(sizeof(size_t) * (C + 1));
    S->vpp_off = malloc(sizeof(size_t) * (C + 1));
    S->vhh_off = malloc(sizeof(size_t) * (C + 1));
    S->t_off[0] = S->vpp_off[0] = S->vhh_off[0] = 0;
    for (int c = 0; c < C; c++) {
        S->t_off[c + 1] = S->t_off[c] + (size_t)S->npp[c] * S->nhh[c];
        S->vpp_off[c + 1] = S->vpp_off[c] + (size_t)S->npp[c] * S->npp[c];
        S->vhh_off[c + 1] = S->vhh_off[c] + (size_t)S->nhh[c] * S->nhh[c];
    }
    S->nt = S->t_off[C];
    S->nvpp = S->vpp_off[C];
    S->nvhh = S->vhh_off[C];
    free(fill); free(key2ch); free(cnt_hh); free(cnt_pp);
}

static void build_cross_channels(om_sys *S) {
    int N = S->N, n = S->nsp;
    int nkeys = S->M * S->M * S->M * S->nq;
    int *cnt_ph = calloc(nkeys, sizeof(int)), *cnt_hp = calloc(nkeys, sizeof(int));
    for (int a = N; a < n; a++)
        for (int i = 0; i < N; i++) cnt_ph[cross_key(S, a, i)]++;
    for (int k = 0; k < N; k++)
        for (int c = N; c < n; c++) cnt_hp[cross_key(S, k, c)]++;
    int *key2x = malloc(sizeof(int) * nkeys);
    S->nx_ch = 0;
    for (int k = 0; k < nkeys; k++) {
        key2x[k] = -1;
        if (cnt_ph[k] > 0 && cnt_hp[k] > 0) key2x[k] = S->nx_ch++;
    }
    int X = S->nx_ch;
    S->xkey = malloc(sizeof(int) * X);
    S->nph = calloc(X, sizeof(int));
    S->nhp = calloc(X, sizeof(int));
    S->ph_off = malloc(sizeof(int) * (X + 1));
    S->hp_off = malloc(sizeof(int) * (X + 1));
    for (int k = 0; k < nkeys; k++)
        if (key2x[k] >= 0) {
            S->xkey[key2x[k]] = k;
            S->nph[key2x[k]] = cnt_ph[k];
            S->nhp[key2x[k]] = cnt_hp[k];
        }
    S->ph_off[0] = S->hp_off[0] = 0;
    for (int x = 0; x < X; x++) {
        S->ph_off[x + 1] = S->ph_off[x] + S->nph[x];
        S->hp_off[x + 1] = S->hp_off[x] + S->nhp[x];
    }
    S->ph_a = malloc(sizeof(int) * (S->ph_off[X] + 1));
    S->ph_i = malloc(sizeof(int) * (S->ph_off[X] + 1));
    S->hp_k = malloc(sizeof(int) * (S->hp_off[X] + 1));
    S->hp_c = malloc(sizeof(int) * (S->hp_off[X] + 1));
    S->phx_ch = malloc(sizeof(int) * (size_t)n * N);
    S->phx_pos = malloc(sizeof(int) * (size_t)n * N);
    S->hpx_ch = malloc(sizeof(int) * (size_t)N * n);
    S->hpx_pos = malloc(sizeof(int) * (size_t)N * n);
    for (size_t z = 0; z < (size_t)n * N; z++)
        S->phx_ch[z] = S->phx_pos[z] = S->hpx_ch[z] = S->hpx_pos[z] = -1;
    int *fill = calloc(X, sizeof(int));
    for (int a = N; a < n; a++)
        for (int i = 0; i < N; i++) {
            int x = key2x[cross_key(S, a, i)];
            if (x < 0) continue;
            int pos = fill[x]++;
            S->ph_a[S->ph_off[x] + pos] = a;
            S->ph_i[S->ph_off[x] + pos] = i;
            S->phx_ch[(size_t)a * N + i] = x;
            S->phx_pos[(size_t)a * N + i] = pos;
        }
    memset(fill, 0, sizeof(int) * X);
    for (int k = 0; k < N; k++)
        for (int c = N; c < n; c++) {
            int x = key2x[cross_key(S, k, c)];
            if (x < 0) continue;
            int pos = fill[x]++;
            S->hp_k[S->hp_off[x] + pos] = k;
            S->hp_c[S->hp_off[x] + pos] = c;
            S->hpx_ch[(size_t)k * n + c] = x;
            S->hpx_pos[(size_t)k * n + c] = pos;
        }
    S->xt_off = malloc(sizeof(size_t) * (X + 1));
    S->xc_off = malloc(sizeof(size_t) * (X + 1));
    S->xw_off = malloc(sizeof(size_t) * (X + 1));
    S->xt_off[0] = S->xc_off[0] = S->xw_off[0] = 0;
    for (int x = 0; x < X; x++) {
        S->xt_off[x + 1] = S->xt_off[x] + (size_t)S->nph[x] * S->nhp[x];
        S->xc_off[x + 1] = S->xc_off[x] + (size_t)S->nhp[x] * S->nhp[x];
        S->xw_off[x + 1] = S->xw_off[x] + (size_t)S->nhp[x] * S->nph[x];
    }
    S->nxt = S->xt_off[X];
    S->nxc = S->xc_off[X];
    S->nxw = S->xw_off[X];
    free(fill); free(key2x); free(cnt_ph); free(cnt_hp);
}

/* ------------------------------------------------------------ create/destroy */

void om_destroy(om_sys *S) {
    if (!S) return;
    void *ptrs[] = {S->nx, S->ny, S->nz, S->sz, S->tz, S->ekin, S->eps, S->chkey, S->nhh, S->npp,
                    S->hh_off, S->pp_off, S->hh_p, S->hh_q, S->pp_p, S->pp_q, S->t_off,
                    S->vpp_off, S->vhh_off, S->pair_ch, S->pair_pos, S->xkey, S->nph, S->nhp,
                    S->ph_off, S->hp_off, S->ph_a, S->ph_i, S->hp_k, S->hp_c, S->xt_off,
                    S->xc_off, S->xw_off, S->phx_ch, S->phx_pos, S->hpx_ch, S->hpx_pos,
                    S->v_pphh, S->v_pppp, S->v_hhhh, S->x_v1, S->x_w, S->t};
    for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); k++) free(ptrs[k]);
    free(S);
}

/* Error codes: 0 ok, -1 invalid argument (not a closed shell, no particle states, or an
 * unsupported composition).  Nn neutrons and Z protons: Z = 0 pure neutron matter, Nn = 0
 * pure proton matter, Nn = Z symmetric nuclear matter (Sec. "Infinite nuclear matter": the
 * channel index then carries T_z); rho is the total density (Nn + Z) / L^3.
 * theta3: twist angles (radians) per axis, NULL for periodic boundary conditions. */
om_sys *om_create_matter(int Nn, int Z, double rho, int n2max, const double *params7,
                         const double *theta3, int *err) {
    *err = -1;
    int N = Nn + Z;
    if (Nn < 0 || Z < 0 || N <= 0 || rho <= 0.0 || n2max < 0) return NULL;
    if (Nn > 0 && Z > 0 && Nn != Z) return NULL;
    om_sys *S = calloc(1, sizeof(om_sys));
    S->N = N; S->rho = rho; S->n2max = n2max;
    S->species = (Nn > 0 ? 1 : 0) | (Z > 0 ? 2 : 0);
    S->nq = S->species == 1 ? 3 : 9;
    S->P.VR = params7[0]; S->P.kR = params7[1];
    S->P.VT = params7[2]; S->P.kT = params7[3];
    S->P.VS = params7[4]; S->P.kS = params7[5];
    S->P.hbar2_2m = params7[6];
    for (int a = 0; a < 3; a++) S->phi[a] = theta3 ? theta3[a] / (2.0 * OM_PI) : 0.0;
    S->m = 2 * isqrt_floor(n2max);
    S->M = 2 * S->m + 1;
    S->L = cbrt((double)N / rho);
    build_basis(S);
    int n = S->nsp;
    if (N >= n) { om_destroy(S); return NULL; }
    double *key = order_by_energy(S);
    /* closed shell: a gap in |n + phi|^2 between the last hole and the first particle */
    if (!(key[N - 1] < key[N])) { free(key); om_destroy(S); return NULL; }
    build_spin_ops(S);
    S->ekin = malloc(sizeof(double) * n);
    S->eps = malloc(sizeof(double) * n);
    double k0 = 2.0 * OM_PI / S->L;
    for (int p = 0; p < n; p++) S->ekin[p] = S->P.hbar2_2m * k0 * k0 * key[p];
    free(key);
    /* f_pp = h0_pp + sum_i <pi|v|pi> */
    for (int p = 0; p < n; p++) {
        double acc = 0.0;
        for (int i = 0; i < N; i++) acc += om_v(S, p, i, p, i);
        S->eps[p] = S->ekin[p] + acc;
    }
    build_direct_channels(S);
    build_cross_channels(S);
    *err = 0;
    return S;
}

om_sys *om_create_twisted(int N, double rho, int n2max, const double *params7,
                          const double *theta3, int *err) {
    return om_create_matter(N, 0, rho, n2max, params7, theta3, err);
}

om_sys *om_create(int N, double rho, int n2max, const double *params7, int *err) {
    return om_create_twisted(N, rho, n2max, params7, NULL, err);
}

/* ------------------------------------------------------------------ accessors */

int om_nsp(const om_sys *S) { return S->nsp; }
double om_L(const om_sys *S) { return S->L; }
int om_nchan(const om_sys *S) { return S->nch; }
int om_nxchan(const om_sys *S) { return S->nx_ch; }
size_t om_nt(const om_sys *S) { return S->nt; }

void om_states(const om_sys *S, int *out4) {
    for (int p = 0; p < S->nsp; p++) {
        out4[4 * p + 0] = S->nx[p];
        out4[4 * p + 1] = S->ny[p];
        out4[4 * p + 2] = S->nz[p];
        out4[4 * p + 3] = S->sz[p];
    }
}

/* Isospin projection per state (+1 neutron, -1 proton). */
void om_isospin(const om_sys *S, int *out) {
    for (int p = 0; p < S->nsp; p++) out[p] = S->tz[p];
}

void om_energies(const om_sys *S, double *ekin, double *eps) {
    for (int p = 0; p < S->nsp; p++) {
        if (ekin) ekin[p] = S->ekin[p];
        if (eps) eps[p] = S->eps[p];
    }
}

/* Direct channel tables: keys[nch], nhh[nch], npp[nch]; pairs (hh then pp), each pair
 * as two ints, channel-major.  Any pointer may be NULL. */
void om_channel_tables(const om_sys *S, int *keys, int *nhh, int *npp, int *hh_pairs,
                       int *pp_pairs) {
    for (int c = 0; c < S->nch; c++) {
        if (keys) keys[c] = S->chkey[c];
        if (nhh) nhh[c] = S->nhh[c];
        if (npp) npp[c] = S->npp[c];
    }
    if (hh_pairs)
        for (int x = 0; x < S->hh_off[S->nch]; x++) {
            hh_pairs[2 * x] = S->hh_p[x];
            hh_pairs[2 * x + 1] = S->hh_q[x];
        }
    if (pp_pairs)
        for (int x = 0; x < S->pp_off[S->nch]; x++) {
            pp_pairs[2 * x] = S->pp_p[x];
            pp_pairs[2 * x + 1] = S->pp_q[x];
        }
}

/* Cross channel tables: keys, nph, nhp; ph pairs (a,i) and hp pairs (k,c). */
void om_cross_tables(const om_sys *S, int *keys, int *nph, int *nhp, int *ph_pairs,
                     int *hp_pairs) {
    for (int x = 0; x < S->nx_ch; x++) {
        if (keys) keys[x] = S->xkey[x];
        if (nph) nph[x] = S->nph[x];
        if (nhp) nhp[x] = S->nhp[x];
    }
    if (ph_pairs)
        for (int z = 0; z < S->ph_off[S->nx_ch]; z++) {
            ph_pairs[2 * z] = S->ph_a[z];
            ph_pairs[2 * z + 1] = S->ph_i[z];
        }
    if (hp_pairs)
        for (int z = 0; z < S->hp_off[S->nx_ch]; z++) {
            hp_pairs[2 * z] = S->hp_k[z];
            hp_pairs[2 * z + 1] = S->hp_c[z];
        }
}

/* ------------------------------------------------------------- E_ref, MBPT2 */

/* E_ref = sum_i h0_ii + 1/2 sum_ij <ij|v|ij>. */
double om_eref(const om_sys *S) {
    double e = 0.0;
    for (int i = 0; i < S->N; i++) e += S->ekin[i];
    double pot = 0.0;
    for (int i = 0; i < S->N; i++)
        for (int j = 0; j < S->N; j++) pot += om_v(S, i, j, i, j);
    return e + 0.5 * pot;
}

/* Delta E_MBPT2 = 1/4 sum_{ijab} <ij|v|ab><ab|v|ij> / (e_i + e_j - e_a - e_b), summed
 * channel by channel over restricted pairs (each restricted term stands for four
 * ordered ones, which cancels the 1/4). */
double om_mbpt2(const om_sys *S) {
    double total = 0.0;
#pragma omp parallel for schedule(dynamic) reduction(+ : total)
    for (int c = 0; c < S->nch; c++) {
        for (int x = 0; x < S->npp[c]; x++) {
            int a = S->pp_p[S->pp_off[c] + x], b = S->pp_q[S->pp_off[c] + x];
            for (int y = 0; y < S->nhh[c]; y++) {
                int i = S->hh_p[S->hh_off[c] + y], j = S->hh_q[S->hh_off[c] + y];
                double vabij = om_v(S, a, b, i, j), vijab = om_v(S, i, j, a, b);
                double D = S->eps[i] + S->eps[j] - S->eps[a] - S->eps[b];
                total += vijab * vabij / D;
            }
        }
    }
    return total;
}

/* ------------------------------------------------------------------ CCD blocks */

static void build_ccd_blocks(om_sys *S) {
    if (S->have_ccd_blocks) return;
    S->v_pphh = malloc(sizeof(double) * (S->nt + 1));
    S->v_pppp = malloc(sizeof(double) * (S->nvpp + 1));
    S->v_hhhh = malloc(sizeof(double) * (S->nvhh + 1));
    S->t = calloc(S->nt + 1, sizeof(double));
#pragma omp parallel for schedule(dynamic)
    for (int c = 0; c < S->nch; c++) {
        int np = S->npp[c], nh = S->nhh[c];
        const int *pa = S->pp_p + S->pp_off[c], *pb = S->pp_q + S->pp_off[c];
        const int *hi = S->hh_p + S->hh_off[c], *hj = S->hh_q + S->hh_off[c];
        double *vt = S->v_pphh + S->t_off[c];
        double *vp = S->v_pppp + S->vpp_off[c];
        double *vh = S->v_hhhh + S->vhh_off[c];
        for (int x = 0; x < np; x++)
            for (int y = 0; y < nh; y++) vt[(size_t)x * nh + y] = om_v(S, pa[x], pb[x], hi[y], hj[y]);
        for (int x = 0; x < np; x++)
            for (int y = 0; y < np; y++) vp[(size_t)x * np + y] = om_v(S, pa[x], pb[x], pa[y], pb[y]);
        for (int x = 0; x < nh; x++)
            for (int y = 0; y < nh; y++) vh[(size_t)x * nh + y] = om_v(S, hi[x], hj[x], hi[y], hj[y]);
    }
    S->x_v1 = malloc(sizeof(double) * (S->nxc + 1));
    S->x_w = malloc(sizeof(double) * (S->nxw + 1));
#pragma omp parallel for schedule(dynamic)
    for (int x = 0; x < S->nx_ch; x++) {
        int nph = S->nph[x], nhp = S->nhp[x];
        const int *hk = S->hp_k + S->hp_off[x], *hc = S->hp_c + S->hp_off[x];
        const int *pa = S->ph_a + S->ph_off[x], *pi = S->ph_i + S->ph_off[x];
        double *v1 = S->x_v1 + S->xc_off[x], *w = S->x_w + S->xw_off[x];
        /* V1[(k,c)][(j,b)] = <kb|v|cj> */
        for (int r = 0; r < nhp; r++)
            for (int s = 0; s < nhp; s++) {
                int k = hk[r], c = hc[r], j = hk[s], b = hc[s];
                v1[(size_t)r * nhp + s] = om_v(S, k, b, c, j);
            }
        /* W[(k,c)][(e,l)] = <kl|v|ce> */
        for (int r = 0; r < nhp; r++)
            for (int s = 0; s < nph; s++) {
                int k = hk[r], c = hc[r], e = pa[s], l = pi[s];
                w[(size_t)r * nph + s] = om_v(S, k, l, c, e);
            }
    }
    S->have_ccd_blocks = 1;
}

/* t_{ij}^{ab} from restricted storage, with the antisymmetry t = -t(i<->j) = -t(a<->b). */
static double t_get(const om_sys *S, const double *t, int a, int b, int i, int j) {
    if (a == b || i == j) return 0.0;
    double sgn = 1.0;
    if (a > b) { int z = a; a = b; b = z; sgn = -sgn; }
    if (i > j) { int z = i; i = j; j = z; sgn = -sgn; }
    int n = S->nsp;
    int c = S->pair_ch[(size_t)a * n + b];
    if (c < 0 || S->pair_ch[(size_t)i * n + j] != c) return 0.0;
    int x = S->pair_pos[(size_t)a * n + b], y = S->pair_pos[(size_t)i * n + j];
    return sgn * t[S->t_off[c] + (size_t)x * S->nhh[c] + y];
}

double om_t_get(const om_sys *S, int a, int b, int i, int j) {
    return t_get(S, S->t, a, b, i, j);
}

void om_t_gather(const om_sys *S, long n, const int *abij, double *out) {
    for (long z = 0; z < n; z++)
        out[z] = t_get(S, S->t, abij[4 * z], abij[4 * z + 1], abij[4 * z + 2], abij[4 * z + 3]);
}

/* Restricted amplitudes in the oracle's own layout, with their (a,b,i,j) labels. */
void om_t_dump(const om_sys *S, int *abij, double *t) {
    size_t z = 0;
    for (int c = 0; c < S->nch; c++)
        for (int x = 0; x < S->npp[c]; x++)
            for (int y = 0; y < S->nhh[c]; y++, z++) {
                if (abij) {
                    abij[4 * z + 0] = S->pp_p[S->pp_off[c] + x];
                    abij[4 * z + 1] = S->pp_q[S->pp_off[c] + x];
                    abij[4 * z + 2] = S->hh_p[S->hh_off[c] + y];
                    abij[4 * z + 3] = S->hh_q[S->hh_off[c] + y];
                }
                if (t) t[z] = S->t[z];
            }
}

/* Delta E = 1/4 sum_{ijab} <ij|v|ab> t_ij^ab = sum over restricted pairs. */
static double ccd_energy(const om_sys *S, const double *t) {
    double e = 0.0;
    for (size_t z = 0; z < S->nt; z++) e += S->v_pphh[z] * t[z];
    return e;
}

/* Particle-hole term in cross channels (the intermediate chi_kb^cj of Sec. "Developing a
 * CCD code", in the cross-coupled (a-i) channels):
 *   T[(a,i)][(k,c)] = t_ik^ac
 *   C[(k,c)][(j,b)] = <kb|v|cj> + 1/2 sum_{(e,l)} <kl|v|ce> t_lj^eb   (quad = 0: <kb|v|cj> only)
 *   Q[(a,i)][(j,b)] = sum_{(k,c)} T C = sum_kc t_ik^ac chi_kb^cj
 * absval != 0: the same with |t|, |v| everywhere (a bound for rounding-error tests). */
static void ph_cross(const om_sys *S, const double *t, double *xT, double *xC, double *xQ, int absval,
                     int quad) {
#pragma omp parallel for schedule(dynamic)
    for (int x = 0; x < S->nx_ch; x++) {
        int nph = S->nph[x], nhp = S->nhp[x];
        const int *pa = S->ph_a + S->ph_off[x], *pi = S->ph_i + S->ph_off[x];
        const int *hk = S->hp_k + S->hp_off[x], *hc = S->hp_c + S->hp_off[x];
        double *T = xT + S->xt_off[x], *Cm = xC + S->xc_off[x], *Q = xQ + S->xt_off[x];
        const double *V1 = S->x_v1 + S->xc_off[x], *W = S->x_w + S->xw_off[x];
        for (int r = 0; r < nph; r++)
            for (int s = 0; s < nhp; s++) {
                double v = t_get(S, t, pa[r], hc[s], pi[r], hk[s]);
                T[(size_t)r * nhp + s] = absval ? fabs(v) : v;
            }
        for (int r = 0; r < nhp; r++)
            for (int s = 0; s < nhp; s++) {
                double acc = 0.0;
                for (int u = 0; u < nph; u++) {
                    double w = W[(size_t)r * nph + u];
                    acc += (absval ? fabs(w) : w) * T[(size_t)u * nhp + s];
                }
                double v1 = V1[(size_t)r * nhp + s];
                Cm[(size_t)r * nhp + s] = (absval ? fabs(v1) : v1) + (quad ? 0.5 * acc : 0.0);
            }
        for (int r = 0; r < nph; r++)
            for (int s = 0; s < nhp; s++) {
                double acc = 0.0;
                for (int u = 0; u < nhp; u++) acc += T[(size_t)r * nhp + u] * Cm[(size_t)u * nhp + s];
                Q[(size_t)r * nhp + s] = acc;
            }
    }
}

/* P(ij)P(ab) Q: Q_ij^ab - Q_ji^ab - Q_ij^ba + Q_ji^ba with Q_ij^ab = Q[(a,i)][(j,b)]
 * (absval != 0: all four with + signs). */
static double ph_combine(const om_sys *S, const double *xQ, int a, int b, int i, int j, int absval) {
    int n = S->nsp, N = S->N;
    int h1[4] = {i, j, i, j}, h2[4] = {j, i, j, i};
    int p1[4] = {a, a, b, b}, p2[4] = {b, b, a, a};
    double sg[4] = {1.0, -1.0, -1.0, 1.0};
    double out = 0.0;
    for (int u = 0; u < 4; u++) {
        int xr = S->phx_ch[(size_t)p1[u] * N + h1[u]];
        int xc = S->hpx_ch[(size_t)h2[u] * n + p2[u]];
        if (xr < 0 || xr != xc) continue;
        int r = S->phx_pos[(size_t)p1[u] * N + h1[u]];
        int s = S->hpx_pos[(size_t)h2[u] * n + p2[u]];
        out += (absval ? 1.0 : sg[u]) * xQ[S->xt_off[xr] + (size_t)r * S->nhp[xr] + s];
    }
    return out;
}

/* Which terms of Eq. (ccd3) an iteration keeps (Sec. "Coupled cluster theory" truncations):
 *   OM_FULL    every term of Eq. (ccd3);
 *   OM_PP      Eq. (ccd1): v and the pp ladder with the bare interaction;
 *   OM_PPHH    Eq. (ccd2): v, the pp ladder and the hh ladder with the bare interaction;
 *   OM_LINEAR  every term linear in t (pp and hh ladders, the ph term with <kb|v|cj>), none of
 *              the quadratic ones.  One unmixed step of it from the MBPT2 amplitudes gives the
 *              third-order energy: E = E2 + the diagrams (3), (4), (5). */
enum { OM_FULL = 0, OM_PP = 1, OM_PPHH = 2, OM_LINEAR = 3 };

/* One Jacobi step of Eq. (ccd3) with the intermediates; writes t_new (restricted). */
static void ccd_step(const om_sys *S, const double *t, double *t_new, double *chi1,
                     double *chi_hh, double *xT, double *xC, double *xQ, int terms) {
    int n = S->nsp;
    int quad = terms == OM_FULL, hh_on = terms != OM_PP, ph_on = terms == OM_FULL || terms == OM_LINEAR;
    /* one-body intermediates.  Momentum and S_z conservation make them diagonal:
     *   chi_b = f_bb - 1/2 sum_{kld} t_kl^bd <kl|v|bd>  = f_bb - sum_d sum_{k<l} t v
     *   chi_j = f_jj + 1/2 sum_{cdl} <jl|v|cd> t_jl^cd  = f_jj + sum_l sum_{c<d} v t   */
    for (int p = 0; p < n; p++) chi1[p] = S->eps[p];
    for (int c = 0; c < S->nch && quad; c++) {
        int np = S->npp[c], nh = S->nhh[c];
        const double *tb = t + S->t_off[c], *vb = S->v_pphh + S->t_off[c];
        for (int x = 0; x < np; x++) {
            double s = 0.0;
            for (int y = 0; y < nh; y++) s += tb[(size_t)x * nh + y] * vb[(size_t)x * nh + y];
            chi1[S->pp_p[S->pp_off[c] + x]] -= s;
            chi1[S->pp_q[S->pp_off[c] + x]] -= s;
        }
        for (int y = 0; y < nh; y++) {
            double s = 0.0;
            for (int x = 0; x < np; x++) s += vb[(size_t)x * nh + y] * tb[(size_t)x * nh + y];
            chi1[S->hh_p[S->hh_off[c] + y]] += s;
            chi1[S->hh_q[S->hh_off[c] + y]] += s;
        }
    }
    /* chi_kl^ij = <kl|v|ij> + 1/2 sum_cd <kl|v|cd> t_ij^cd   (restricted cd) */
#pragma omp parallel for schedule(dynamic)
    for (int c = 0; c < S->nch; c++) {
        int np = S->npp[c], nh = S->nhh[c];
        const double *tb = t + S->t_off[c], *vb = S->v_pphh + S->t_off[c];
        const double *vh = S->v_hhhh + S->vhh_off[c];
        double *ch = chi_hh + S->vhh_off[c];
        for (int kl = 0; kl < nh; kl++)
            for (int ij = 0; ij < nh; ij++) {
                double s = vh[(size_t)kl * nh + ij];
                for (int cd = 0; cd < np && quad; cd++)
                    s += vb[(size_t)cd * nh + kl] * tb[(size_t)cd * nh + ij];
                ch[(size_t)kl * nh + ij] = s;
            }
    }
    if (ph_on) ph_cross(S, t, xT, xC, xQ, 0, quad);
    /* assemble Eq. (ccd3) with the intermediates, for restricted a<b, i<j */
#pragma omp parallel for schedule(dynamic)
    for (int c = 0; c < S->nch; c++) {
        int np = S->npp[c], nh = S->nhh[c];
        const double *tb = t + S->t_off[c], *vb = S->v_pphh + S->t_off[c];
        const double *vp = S->v_pppp + S->vpp_off[c];
        const double *ch = chi_hh + S->vhh_off[c];
        double *tn = t_new + S->t_off[c];
        for (int x = 0; x < np; x++) {
            int a = S->pp_p[S->pp_off[c] + x], b = S->pp_q[S->pp_off[c] + x];
            for (int y = 0; y < nh; y++) {
                int i = S->hh_p[S->hh_off[c] + y], j = S->hh_q[S->hh_off[c] + y];
                double tab = tb[(size_t)x * nh + y];
                double num = vb[(size_t)x * nh + y];
                /* P(ab) sum_c chi_b^c t_ij^ac - P(ij) sum_k chi_k^j t_ik^ab, without the
                 * f (= eps) parts, which form the denominator */
                num += ((chi1[a] - S->eps[a]) + (chi1[b] - S->eps[b]) - (chi1[i] - S->eps[i]) -
                        (chi1[j] - S->eps[j])) * tab;
                /* 1/2 sum_cd <ab|chi|cd> t_ij^cd */
                double pp = 0.0;
                for (int cd = 0; cd < np; cd++) pp += vp[(size_t)x * np + cd] * tb[(size_t)cd * nh + y];
                num += pp;
                /* 1/2 sum_kl t_kl^ab chi_kl^ij */
                double hh = 0.0;
                for (int kl = 0; kl < nh && hh_on; kl++) hh += tb[(size_t)x * nh + kl] * ch[(size_t)kl * nh + y];
                num += hh;
                /* P(ij)P(ab) sum_kc t_ik^ac chi_kb^cj = Q_ij^ab - Q_ji^ab - Q_ij^ba + Q_ji^ba */
                if (ph_on) num += ph_combine(S, xQ, a, b, i, j, 0);
                double D = S->eps[i] + S->eps[j] - S->eps[a] - S->eps[b];
                tn[(size_t)x * nh + y] = num / D;
            }
        }
    }
}

static double now_s(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return ts.tv_sec + 1e-9 * ts.tv_nsec;
}

/*
 * CCD iteration.  init: 0 = MBPT2 guess t = v/eps_ij^ab, 1 = zero amplitudes.
 * Stops when |dE^(n+1) - dE^(n)| < tol (total energy, MeV) or after maxit updates.
 * e_hist (nullable, length maxit+1) receives dE after 0, 1, 2, ... updates.
 * Returns the number of updates made, or -1 on a zero denominator.
 * timings (nullable, 2 doubles): setup seconds, iteration seconds.
 */
int om_ccd_terms(om_sys *S, double alpha, double tol, int maxit, int init, int terms,
                 double *dE_out, double *e_hist, double *timings) {
    if (terms < OM_FULL || terms > OM_LINEAR) return -2;
    double t0 = now_s();
    build_ccd_blocks(S);
    int n = S->nsp;
    double *t_new = malloc(sizeof(double) * (S->nt + 1));
    double *chi1 = malloc(sizeof(double) * n);
    double *chi_hh = malloc(sizeof(double) * (S->nvhh + 1));
    double *xT = malloc(sizeof(double) * (S->nxt + 1));
    double *xC = malloc(sizeof(double) * (S->nxc + 1));
    double *xQ = malloc(sizeof(double) * (S->nxt + 1));
    int bad = 0;
    for (int c = 0; c < S->nch; c++)
        for (int x = 0; x < S->npp[c]; x++)
            for (int y = 0; y < S->nhh[c]; y++) {
                int a = S->pp_p[S->pp_off[c] + x], b = S->pp_q[S->pp_off[c] + x];
                int i = S->hh_p[S->hh_off[c] + y], j = S->hh_q[S->hh_off[c] + y];
                double D = S->eps[i] + S->eps[j] - S->eps[a] - S->eps[b];
                size_t z = S->t_off[c] + (size_t)x * S->nhh[c] + y;
                if (D == 0.0) bad = 1;
                S->t[z] = (init == 0 && D != 0.0) ? S->v_pphh[z] / D : 0.0;
            }
    double t1 = now_s();
    if (bad) {
        free(t_new); free(chi1); free(chi_hh); free(xT); free(xC); free(xQ);
        return -1;
    }
    double e_old = ccd_energy(S, S->t);
    if (e_hist) e_hist[0] = e_old;
    int it = 0;
    while (it < maxit) {
        ccd_step(S, S->t, t_new, chi1, chi_hh, xT, xC, xQ, terms);
        for (size_t z = 0; z < S->nt; z++) S->t[z] = alpha * t_new[z] + (1.0 - alpha) * S->t[z];
        double e = ccd_energy(S, S->t);
        it++;
        if (e_hist) e_hist[it] = e;
        double diff = fabs(e - e_old);
        e_old = e;
        if (diff < tol) break;
    }
    double t2 = now_s();
    if (dE_out) *dE_out = e_old;
    if (timings) { timings[0] = t1 - t0; timings[1] = t2 - t1; }
    free(t_new); free(chi1); free(chi_hh); free(xT); free(xC); free(xQ);
    return it;
}

int om_ccd(om_sys *S, double alpha, double tol, int maxit, int init, double *dE_out,
           double *e_hist, double *timings) {
    return om_ccd_terms(S, alpha, tol, maxit, init, OM_FULL, dE_out, e_hist, timings);
}

/* Third-order energy diagrams of Sec. "Many-body perturbation theory" (Fig. goldstone), with
 * the MBPT2 amplitudes t0 = <ab|v|ij> / eps_ij^ab and restricted sums (a<b, i<j):
 *   out[0] = (4) = 1/8 sum <ij|v|cd><cd|v|ab><ab|v|ij> / (eps_ij^cd eps_ij^ab)
 *          = sum t0_ab^ij sum_{c<d} <ab|v|cd> t0_cd^ij                      (pp ladder)
 *   out[1] = (5) = 1/8 sum <ab|v|kl><kl|v|ij><ij|v|ab> / (eps_ij^ab eps_kl^ab)
 *          = sum t0_ab^ij sum_{k<l} t0_ab^kl <kl|v|ij>                      (hh ladder)
 *   out[2] = (3) = sum_{ijkabc} t0_ab^ij <kb|v|cj> t0_ac^ik                 (ph ring)
 *          = sum t0_ab^ij [P(ij)P(ab) sum_kc <kb|v|cj> t0_ik^ac]_restricted.
 * Eq. (diag3) is printed with <bk|v|ic> = <kb|v|ci>; read with <kb|v|cj> (i and j of that
 * factor swapped): as printed it vanishes for two particles and misses third-order
 * Rayleigh-Schroedinger perturbation theory, which the form used here reproduces.
 * Returns 0, or -1 on a zero denominator or no memory. */
int om_mbpt3(om_sys *S, double *out) {
    build_ccd_blocks(S);
    double *t0 = malloc(sizeof(double) * (S->nt + 1));
    double *xT = malloc(sizeof(double) * (S->nxt + 1));
    double *xC = malloc(sizeof(double) * (S->nxc + 1));
    double *xQ = malloc(sizeof(double) * (S->nxt + 1));
    if (!t0 || !xT || !xC || !xQ) {
        free(t0); free(xT); free(xC); free(xQ);
        return -1;
    }
    int bad = 0;
    for (int c = 0; c < S->nch; c++)
        for (int x = 0; x < S->npp[c]; x++)
            for (int y = 0; y < S->nhh[c]; y++) {
                int a = S->pp_p[S->pp_off[c] + x], b = S->pp_q[S->pp_off[c] + x];
                int i = S->hh_p[S->hh_off[c] + y], j = S->hh_q[S->hh_off[c] + y];
                double D = S->eps[i] + S->eps[j] - S->eps[a] - S->eps[b];
                size_t z = S->t_off[c] + (size_t)x * S->nhh[c] + y;
                if (D == 0.0) bad = 1;
                t0[z] = D != 0.0 ? S->v_pphh[z] / D : 0.0;
            }
    if (bad) {
        free(t0); free(xT); free(xC); free(xQ);
        return -1;
    }
    ph_cross(S, t0, xT, xC, xQ, 0, 0);
    double e4 = 0.0, e5 = 0.0, e3 = 0.0;
    for (int c = 0; c < S->nch; c++) {
        int np = S->npp[c], nh = S->nhh[c];
        const double *tb = t0 + S->t_off[c];
        const double *vp = S->v_pppp + S->vpp_off[c], *vh = S->v_hhhh + S->vhh_off[c];
        for (int x = 0; x < np; x++) {
            int a = S->pp_p[S->pp_off[c] + x], b = S->pp_q[S->pp_off[c] + x];
            for (int y = 0; y < nh; y++) {
                int i = S->hh_p[S->hh_off[c] + y], j = S->hh_q[S->hh_off[c] + y];
                double tz = tb[(size_t)x * nh + y];
                double pp = 0.0, hh = 0.0;
                for (int cd = 0; cd < np; cd++) pp += vp[(size_t)x * np + cd] * tb[(size_t)cd * nh + y];
                for (int kl = 0; kl < nh; kl++) hh += tb[(size_t)x * nh + kl] * vh[(size_t)kl * nh + y];
                e4 += tz * pp;
                e5 += tz * hh;
                e3 += tz * ph_combine(S, xQ, a, b, i, j, 0);
            }
        }
    }
    out[0] = e4;
    out[1] = e5;
    out[2] = e3;
    free(t0); free(xT); free(xC); free(xQ);
    return 0;
}

/* The P(ij)P(ab) sum_kc t_ik^ac chi_kb^cj part of Eq. (ccd3) for the restricted amplitudes t
 * (oracle layout), into out (same layout); absval != 0 gives the absolute-value bound. */
int om_ph_apply(om_sys *S, const double *t, double *out, int absval) {
    build_ccd_blocks(S);
    double *xT = malloc(sizeof(double) * (S->nxt + 1));
    double *xC = malloc(sizeof(double) * (S->nxc + 1));
    double *xQ = malloc(sizeof(double) * (S->nxt + 1));
    if (!xT || !xC || !xQ) {
        free(xT); free(xC); free(xQ);
        return -1;
    }
    ph_cross(S, t, xT, xC, xQ, absval, 1);
    for (int c = 0; c < S->nch; c++) {
        int np = S->npp[c], nh = S->nhh[c];
        for (int x = 0; x < np; x++) {
            int a = S->pp_p[S->pp_off[c] + x], b = S->pp_q[S->pp_off[c] + x];
            for (int y = 0; y < nh; y++) {
                int i = S->hh_p[S->hh_off[c] + y], j = S->hh_q[S->hh_off[c] + y];
                out[S->t_off[c] + (size_t)x * nh + y] = ph_combine(S, xQ, a, b, i, j, absval);
            }
        }
    }
    free(xT); free(xC); free(xQ);
    return 0;
}

int om_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void om_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* <ab|v|cd> block of direct channel c (restricted pairs, npp x npp row-major) and its size. */
long om_vpp_block(om_sys *S, int c, double *out) {
    if (c < 0 || c >= S->nch) return -1;
    build_ccd_blocks(S);
    long n = (long)S->npp[c] * S->npp[c];
    if (out) memcpy(out, S->v_pppp + S->vpp_off[c], sizeof(double) * n);
    return n;
}
