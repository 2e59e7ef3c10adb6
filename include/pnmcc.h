/*
 * pnmcc.h -- C ABI of the GB300 (sm_103a) coupled-cluster doubles library for pure
 * neutron matter with the Minnesota interaction.
 *
 * Method: Lietz, Novario, Jansen, Hagen, Hjorth-Jensen, "Computational Nuclear Physics
 * and Post Hartree-Fock Methods" (arXiv:1611.06765).  Each call below names the passage
 * of that paper which defines what it computes.
 *
 * Conventions for every call:
 *   - Return value: PNM_OK (0) or a negative PNM_E* code.  No C++ exception crosses the
 *     ABI.  pnm_last_error() returns a thread-local text for the last failure.
 *   - Host arrays passed in are read only during the call; host output arrays are owned by
 *     the caller and must hold the stated number of elements.  A NULL output pointer is
 *     allowed where stated and turns the call into a size query.
 *   - All device memory is owned by the context: allocated by pnm_create*, released by
 *     pnm_destroy.  Work runs on the CUDA stream given at creation (NULL = the legacy
 *     default stream) and every call that returns host data synchronises that stream.
 *   - Energies are totals in MeV (not per particle).  Momenta are integer lattice vectors
 *     n (k = 2 pi n / L); spins are in units of hbar/2 (-1 or +1).
 *   - A context holds one or more independent systems (N, rho, n2max); calls taking
 *     `sys` address one of them (0 for a single-system context).
 */
#ifndef PNMCC_H
#define PNMCC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PNM_OK 0
#define PNM_EINVAL (-1)     /* bad argument: N not a closed shell, no particle states, ... */
#define PNM_ENOMEM (-2)     /* device or host allocation failed */
#define PNM_ECUDA (-3)      /* a CUDA runtime call failed */
#define PNM_ENOTCONV (-4)   /* iteration cap reached before the energy change met the tolerance */
#define PNM_EDIVERGED (-5)  /* NaN/Inf energy or residual, or |dE| of a system at least doubling
                               (above its tolerance) over 6 consecutive updates */
#define PNM_ETIMEOUT (-6)   /* a device-side wait ran out of its budget */

typedef struct pnm_ctx pnm_ctx;

/* Minnesota interaction (Sec. "Two-body interaction", Table tab:minnesotatab):
 * V(r) = 1/2 (V_R e^{-kR r^2} + 1/2(1+Ps) V_T e^{-kT r^2} + 1/2(1-Ps) V_S e^{-kS r^2})(1 - Ps Pt).
 * V in MeV, kappa in fm^-2, hbar2_2m in MeV fm^2.  The paper prints magnitudes; the
 * attractive terms take V_T, V_S < 0. */
typedef struct {
    double VR, kR, VT, kT, VS, kS, hbar2_2m;
} pnm_minnesota;

#define PNM_PREC_FP64 0   /* every step in FP64 */
#define PNM_PREC_BF16X3 2 /* pp ladder as hi/lo BF16 products on tcgen05 (FP32 accumulate),
                             other contractions in FP32, denominators/energy/residual FP64,
                             then `refine_sweeps` FP64 iterations */
#define PNM_PREC_F32PAIR 3 /* contractions (pp ladder, ph term) with every value carried as the
                              unevaluated sum of two FP32 numbers, 48 significant bits, on the
                              FP32 pipe (exact products by fused multiply-add, two-sum
                              accumulation), results in FP64: an FP64-accurate alternative to
                              the FP64 pipe for the refinement sweeps (opts.refine_kernels) and
                              the operator calls; not a solve precision */

#define PNM_INIT_MBPT2 0  /* t = <ab|v|ij> / eps_ij^ab, Eq. (ccdGuess) */
#define PNM_INIT_ZERO 1   /* t = 0 (the first update then gives MBPT2) */
#define PNM_INIT_KEEP 2   /* start from the amplitudes currently held (pnm_set_amplitudes) */
#define PNM_INIT_MLP 3    /* learned start (pnm_mlp_set_model); falls back to MBPT2 if the
                             iteration from it does not converge */
/* Kept starts are first symmetrised under the global spin flip F (every state to the one of
 * opposite spin): t <- (t + F t)/2; the learned start is evaluated on one amplitude of each
 * flip pair and copied to the other.  F commutes with H and leaves the
 * spin-saturated reference unchanged, so the solution is flip-symmetric, and the iteration
 * works on flip-symmetric amplitudes only: the ph term is formed for S_z >= 0 cross channels
 * (S_z = 0 ones as half-size sum and difference blocks) and read at the flip elsewhere, and
 * the update computes one amplitude of each flip pair and writes both.  MBPT2 and zero starts
 * are symmetric already. */

/* Terms the iteration keeps (Sec. "Coupled cluster theory"):
 *   PNM_TERMS_FULL    Eq. (ccd3);
 *   PNM_TERMS_PP      Eq. (ccd1): <ab|v|ij>, the energy denominator and the pp ladder with the
 *                     bare interaction (the G-matrix equation at omega = eps_i + eps_j);
 *   PNM_TERMS_PPHH    Eq. (ccd2): and the hh ladder 1/2 sum_kl <kl|v|ij> t_kl^ab;
 *   PNM_TERMS_LINEAR  every term of Eq. (ccd3) linear in t (both ladders and the ph term with
 *                     <kb|v|cj>), none of the quadratic ones.
 * The truncations are linear in t; they run in FP64 (precision PNM_PREC_FP64). */
#define PNM_TERMS_FULL 0
#define PNM_TERMS_PP 1
#define PNM_TERMS_PPHH 2
#define PNM_TERMS_LINEAR 3

/* Options of the CCD iteration (Eq. ccd3 with mixing and the stopping rule of Sec.
 * "Developing a numerical project"). */
typedef struct {
    int precision;        /* PNM_PREC_* */
    double mix_alpha;     /* t = alpha t_new + (1-alpha) t_old, alpha in (0,1] */
    double tol_dE;        /* stop when |dE^(n+1) - dE^(n)| < tol_dE (total, MeV) */
    double tol_dE_per_N;  /* and/or when |dE^(n+1) - dE^(n)| / N < tol_dE_per_N (<= 0: unused) */
    int max_iter;         /* iteration cap (PNM_ENOTCONV when reached) */
    int refine_sweeps;    /* FP64 sweeps after a mixed-precision solve has converged: exactly
                             this many FP64 updates, the FP64 stopping test applied from the
                             last of them on (further FP64 updates, at most max_iter, until it
                             passes) */
    int init;             /* PNM_INIT_* */
    int host_loop;        /* 0: device-side loop in one CUDA graph; 1: host checks each iteration */
    int terms;            /* PNM_TERMS_*: the full Eq. (ccd3) or a truncation (FP64 only) */
    int refine_kernels;   /* contractions of the refinement sweeps: PNM_PREC_FP64 (FP64 pipe) or
                             PNM_PREC_F32PAIR (FP32 pairs); the update, denominators, residual
                             and energy of the sweeps are FP64 either way */
} pnm_solve_opts;

/* Fills the defaults of the small FP64 workload: FP64, alpha 0.5, tol 1e-10 MeV,
 * max_iter 500, no refinement (FP64-pipe refinement kernels when enabled), MBPT2 start,
 * device-side loop, full Eq. (ccd3). */
void pnm_default_opts(pnm_solve_opts *opts);

/* Build one system: the basis of Sec. "Single-particle basis for infinite matter" (k =
 * 2 pi n/L, L^3 = N/rho, n^2 <= n2max, shell order of the state loop in Sec. "Developing a
 * CCD code", first N states are holes), its direct (P, S_z) and cross channels, the
 * antisymmetrized Minnesota blocks and the HF energies eps_p = f_pp (Eq. Hnormalorder).
 * Runs on the GPU.  PNM_EINVAL if N does not close a shell or leaves no particle state.
 * stream: a cudaStream_t (NULL = legacy default stream).  *out receives the context. */
int pnm_create(int N, double rho, int n2max, const pnm_minnesota *params, void *stream,
               pnm_ctx **out);

/* Build n independent systems in one context; their channels are grouped so every
 * iteration kernel covers all systems in one launch.  Arrays have n entries. */
int pnm_create_batch(int n, const int *N, const double *rho, const int *n2max,
                     const pnm_minnesota *params, void *stream, pnm_ctx **out);

/* Twisted boundary conditions (Sec. "Twist-averaged boundary conditions"): as
 * pnm_create_batch, with system k's single-particle momenta k = (2 pi n + theta_k)/L.
 * theta: 3n doubles (radians, x y z per system), NULL for periodic boundaries; host memory,
 * read during the call.  The model space stays n^2 <= n2max; the states are reordered by
 * |n + theta/2pi|^2 (equal values keep the shell order) and the lowest N are the holes.  The
 * three axis terms of |n + theta/2pi|^2 are rounded one by one and added smallest first, so
 * twists with equal components give equal energies to states that differ by a permutation.
 * PNM_EINVAL (message naming the system) if a twist leaves no gap between state N-1 and
 * state N (a degenerate Fermi level: the reference is not unique), or a twist is not finite. */
int pnm_create_twisted(int n, const int *N, const double *rho, const int *n2max,
                       const double *theta, const pnm_minnesota *params, void *stream,
                       pnm_ctx **out);

/* Nuclear matter (Sec. "Infinite nuclear matter"): as pnm_create_twisted, with system k made
 * of N[k] neutrons and Z[k] protons: Z = 0 pure neutron matter, N = 0 pure proton matter,
 * N = Z symmetric nuclear matter (other compositions: PNM_EINVAL).  rho[k] is the total density
 * (N + Z) / L^3 and n2max[k] the lattice bound; Z = NULL means no protons anywhere.  With
 * protons every momentum carries four states (s = -1 then +1, within a spin the proton before
 * the neutron; t = +1 neutron, -1 proton), the full Minnesota operator acts (the V_T term
 * couples np pairs), and channel keys carry T_z: slot 3 (S_z + 2)/2 + (T_z + 2)/2 of 9 in
 * place of (S_z + 2)/2 of 3.  pnm_basis then reports the fourth component of a state as
 * s + 4t.  theta: as pnm_create_twisted (NULL: periodic).  Arrays have n entries, host
 * memory read during the call. */
int pnm_create_matter(int n, const int *N, const int *Z, const double *rho, const int *n2max,
                      const double *theta, const pnm_minnesota *params, void *stream,
                      pnm_ctx **out);

/* Product Gauss-Legendre twist mesh of the twist-averaging loop (Sec. "Twist-averaged
 * boundary conditions"): nx, ny, nz nodes (1..64) on [0, pi] per axis, points in x-major
 * order (m = (i ny + j) nz + k).  theta: 3 nx ny nz doubles (radians); weight: nx ny nz
 * doubles, w_x w_y w_z / pi^3 with w the Gauss-Legendre weights on [0, pi], so they sum to 1
 * and the twist average of E is sum_m weight[m] E(theta_m).  Host memory owned by the caller;
 * pure host computation.  Equal node counts on two axes put mesh points on the planes
 * theta_x = theta_y (and so on), where the Fermi level can be degenerate; distinct counts
 * with at most one odd count avoid equal components altogether.  PNM_EINVAL on bad sizes. */
int pnm_twist_mesh(int nx, int ny, int nz, double *theta, double *weight);

/* Release the context and all its device memory.  NULL is accepted. */
int pnm_destroy(pnm_ctx *ctx);

/* Number of systems held by the context. */
int pnm_num_systems(const pnm_ctx *ctx, int *n);

/* Single-particle basis of system `sys`: sizes, and (nullable) n_x, n_y, n_z, s per state
 * (4 int8 per state, state-major) and the HF energies (n_sp doubles). */
int pnm_basis(const pnm_ctx *ctx, int sys, int *n_sp, int *n_holes, int8_t *nxyzs,
              double *eps_hf);

/* Channel tables of system `sys` as built on the GPU.
 * kind 0: direct channels (P = n_p + n_q, S_z = s_p + s_q) holding restricted hh pairs
 *         i<j and pp pairs a<b (both non-empty); per channel keys[c], sizes[2c] = n_hh,
 *         sizes[2c+1] = n_pp; pairs = all hh pairs then all pp pairs, 2 ints each,
 *         channel-major, lexicographic inside a channel.
 * kind 1: cross channels (n_p - n_q, s_p - s_q) with ordered ph rows (a,i) and hp columns
 *         (k,c); sizes[2x] = n_ph, sizes[2x+1] = n_hp; pairs = all (a,i) then all (k,c).
 * key = (((Px+m)*M + (Py+m))*M + (Pz+m))*3 + (Sz+2)/2, m = 2 floor(sqrt(n2max)), M = 2m+1.
 * Sec. "Developing a CCD code" (direct T and cross X channels).  Any output may be NULL;
 * *n_chan and *n_pairs (total pair count) are always written. */
int pnm_channels(const pnm_ctx *ctx, int sys, int kind, int *n_chan, int *n_pairs,
                 int32_t *keys, int32_t *sizes, int32_t *pairs);

/* Antisymmetrized <pq|v|rs> of system `sys` (MeV), evaluated by the same device code
 * that fills the blocks.  Sec. "Two-body interaction". */
int pnm_v_element(const pnm_ctx *ctx, int sys, int p, int q, int r, int s, double *out);

/* Reference energy E_ref = sum_i h0_ii + 1/2 sum_ij <ij|v|ij> (Sec. "Normal-ordered
 * Hamiltonian", the E_Ref expression).  One value per system (e_ref[n_systems]). */
int pnm_eref(const pnm_ctx *ctx, double *e_ref);

/* Second-order correlation energy, Eq. (ccdGuess) and the energy below it, computed as a
 * fused pass over the direct channels.  One value per system. */
int pnm_mbpt2(pnm_ctx *ctx, double *dE);

/* Size of the basis in which the pp ladder of each direct channel of system `sys` is computed
 * (0 for channels without a pp-pp interaction block).  For neutron pairs of S_z = 0 the
 * interaction acts only on the spin singlet: pairs whose spatial labels differ by the exchange
 * of the two spins share one basis vector (with the sign of their stored order), so the basis
 * has about half as many vectors as the channel has pairs and the ladder's V block and products
 * shrink to about a quarter; elsewhere one vector per pair.  *n_chan receives the number of
 * direct channels; nlad (nullable, host) one int per channel in pnm_channels order. */
int pnm_ladder_sizes(const pnm_ctx *ctx, int sys, int *n_chan, int32_t *nlad);

/* Third-order correlation energy (Sec. "Many-body perturbation theory", Fig. goldstone):
 * e3[3 s + 0] = diagram (4), the pp ladder (Eq. diag4); e3[3 s + 1] = diagram (5), the hh
 * ladder (Eq. diag5); e3[3 s + 2] = diagram (3), the particle-hole ring (Eq. diag3, read with
 * <kb|v|cj> where the paper prints <bk|v|ic>; that reading is the third order of
 * Rayleigh-Schroedinger perturbation theory with HF energies).  Their sum is the MBPT3
 * correction; diagrams with HF insertions vanish in this basis.  Computed on the GPU in FP64
 * from the MBPT2 amplitudes t0 = <ab|v|ij>/eps_ij^ab: one pp-ladder launch, one linear ph
 * launch and a fused row pass with the hh ladder and the three dot products.  e3: host,
 * 3 n_systems doubles.  The context's amplitudes afterwards hold the MBPT2 guess. */
int pnm_mbpt3(pnm_ctx *ctx, double *e3);

/* The same second-order energy as pnm_mbpt2, for callers that must not allocate device
 * memory at the time of the call: loops whose device-memory budget is fixed when they start
 * (a later allocation could fail or stall them), or hosts whose device allocator belongs to
 * another framework that forbids side allocations.  This call allocates nothing (no
 * cudaMalloc, cudaFree or allocating library routine).  Its scratch is a file-scope device
 * array of (65536 + 64) doubles, about 513 KB, which every GPU that loads this library holds
 * until the process exits.  Limits: at most 65536 (channel, hole-pair) rows and 64 systems
 * per context, else PNM_EINVAL with a message.  The first call on a device looks up the
 * array's device address for that device (done once per device and kept for the life of its
 * primary context); make that first call before any stream capture.  All calls on a device
 * share the one array: every slot used is rewritten by each call, so nothing carries over,
 * but calls that overlap on the GPU (from several host threads or streams) race on it.  dE
 * receives one value per system (host memory); the call copies it back and synchronises the
 * context stream.  The paper has no counterpart: this is the library's own calling
 * convention. */
int pnm_mbpt2_noalloc(const pnm_ctx *ctx, double *dE);

/* Solve the CCD equations (Eq. ccd3 in the intermediate form of Sec. "Developing a CCD
 * code", energy Eq. ccdcorr).  Per system outputs (nullable): dE (correlation energy),
 * iters (updates made), resid (2-norm of the last residual over restricted amplitudes).
 * Returns PNM_ENOTCONV / PNM_EDIVERGED as described above; outputs are still written. */
int pnm_ccd_solve(pnm_ctx *ctx, const pnm_solve_opts *opts, double *dE, int *iters,
                  double *resid);

/* Energy after each update of the last solve: hist[0] is the start, hist[k] after k
 * updates.  *n receives the number of entries (<= cap) for system `sys`. */
int pnm_energy_history(const pnm_ctx *ctx, int sys, double *hist, int cap, int *n);

/* Number of restricted amplitudes (a<b, i<j, both pairs in one direct channel) of
 * system `sys`, and (nullable) their labels a, b, i, j in the library's order. */
int pnm_amplitude_labels(const pnm_ctx *ctx, int sys, size_t *n, int32_t *abij);

/* Copy restricted amplitudes (FP64, library order) of system `sys` to / from the host.
 * n must equal the count of pnm_amplitude_labels.  Checkpoint and training-data path. */
int pnm_get_amplitudes(const pnm_ctx *ctx, int sys, double *t, size_t n);
int pnm_set_amplitudes(pnm_ctx *ctx, int sys, const double *t, size_t n);

/* Checkpoint header of one system: what fixes its amplitude layout.  twist = theta / 2 pi per
 * axis (0 for periodic boundaries); channel_hash = FNV-1a (64 bit) over the system's direct
 * channels in pnm_channels order: per channel its key, n_hh and n_pp, then every hole and
 * particle pair (state indices within the system). */
typedef struct {
  int32_t N, Z, n2max, reserved;
  double rho;
  double twist[3];
  int64_t n_amplitudes;
  uint64_t channel_hash;
} pnm_checkpoint_header;
int pnm_checkpoint_header_of(const pnm_ctx *ctx, int sys, pnm_checkpoint_header *h);

/* Checkpoint / resume (not in the paper): write the held amplitudes of every system (those
 * pnm_get_amplitudes reads: after a solve the converged ones) to `path`, with their headers;
 * read them back into a context built for the same systems.  File: the 8 bytes "PNMCKPT1",
 * int32 number of systems, int32 0, the headers, then each system's amplitudes (FP64, library
 * order), host byte order.  pnm_checkpoint_load returns PNM_EINVAL, leaving the context's
 * amplitudes unchanged, when the file cannot be read, is truncated or any header differs from
 * the context's (bit for bit); a solve with init = PNM_INIT_KEEP resumes from the loaded
 * amplitudes. */
int pnm_checkpoint_save(const pnm_ctx *ctx, const char *path);
int pnm_checkpoint_load(pnm_ctx *ctx, const char *path);

/* The particle-particle ladder alone, as an operator on amplitudes:
 * r_ij^ab = 1/2 sum_cd <ab|v|cd> t_ij^cd = sum_{c<d} <ab|v|cd> t_ij^cd (the pp-ladder term of
 * Eq. ccd3, with <ab|chi|cd> = <ab|v|cd> of Sec. "Developing a CCD code"), evaluated by the
 * FP64 kernel, the FP32-pair kernel (PNM_PREC_F32PAIR) or the BF16x3 tensor-core kernel
 * (precision).  t and r hold n restricted
 * amplitudes of system `sys` in library order; r is 0 on channels whose V block vanishes
 * (S_z != 0 for neutrons).  Resets the solver's iteration state. */
int pnm_apply_pp_ladder(pnm_ctx *ctx, int sys, int precision, const double *t, double *r,
                        size_t n);

/* The particle-hole term alone, as an operator on amplitudes: r_ij^ab =
 * P(ij)P(ab) sum_kc t_ik^ac chi_kb^cj with chi_kb^cj = <kb|v|cj> + 1/2 sum_dl <kl|v|cd> t_lj^db
 * (the linear ph term and the quadratic ph term of Eq. ccd3 through the intermediate of Sec.
 * "Developing a CCD code"), computed in the cross-coupled channels (n_a - n_i, s_a - s_i):
 * FP64 kernels, FP32-pair kernels (PNM_PREC_F32PAIR), or the mixed-precision ones (FP32
 * operands and products).  t and r hold n restricted
 * amplitudes of system `sys` in library order; r is the term of the flip-symmetric part
 * (t + F t)/2 of t (see PNM_INIT_KEEP).  Resets the solver's iteration state. */
int pnm_apply_ph_term(pnm_ctx *ctx, int sys, int precision, const double *t, double *r, size_t n);

/* Device time (ms, CUDA events) of the last pnm_create*, pnm_mbpt2 and pnm_ccd_solve:
 * ms[0] setup, ms[1] mbpt2, ms[2] solve (total), ms[3] mixed phase, ms[4] refinement;
 * ms[5] = 1 if the last solve with init = PNM_INIT_MLP fell back to the MBPT2 start, else 0;
 * ms[6] host wall time (ms) that the last pnm_ccd_solve spent on the context's one-time
 * preparation (FP32 and FP32-pair copies, schedule tuning, capture and instantiation of the
 * iteration graphs); about 0 when all of it was done by an earlier solve of the context.
 * The first min(n, 7) entries are written. */
int pnm_get_timings(const pnm_ctx *ctx, double *ms, int n);

/* ---------------------------------------------------------------- learned warm start
 * Not in the paper: a network predicts the converged amplitudes so the Jacobi iteration of
 * Eq. (ccd3) starts closer to its fixed point than the MBPT2 guess of Eq. (ccdGuess); the
 * iteration itself still decides the result.  Network: 32 features -> 128 -> 128 -> 128
 * (GELU) -> 1, weights and layer inputs rounded to BF16, FP32 accumulation;
 *   t_start = t_MBPT2 + sigma_sys * y_scale * net(features),
 * sigma_sys = RMS of the system's MBPT2 amplitudes.  Features per restricted amplitude:
 * k_a, k_b, k_i, k_j / k_F (12), spins (4), eps_ij^ab / eps_F, N <ab|v|ij> / eps_F,
 * t_MBPT2 / sigma_sys, rho / 0.16, k_F, N / 66, then 10 zeros.
 * Parameter blob (pnm_mlp_num_params floats): mu[32], inv_std[32], y_scale, pad[3],
 * W1[128][32], b1[128], W2[128][128], b2[128], W3[128][128], b3[128], w4[128], b4. */
typedef struct {
    int epochs;               /* passes over the training amplitudes */
    int batch;                /* samples per Adam step */
    double lr;                /* Adam learning rate (beta1 0.9, beta2 0.999, eps 1e-8) */
    unsigned long long seed;  /* shuffling */
    double lr_final;          /* learning rate of the last step: the rate follows a half cosine
                                 from lr down to lr_final over all steps (<= 0 or == lr: constant) */
} pnm_mlp_opts;

/* Number of floats in a parameter blob. */
int pnm_mlp_num_params(int *n);

/* Initial parameters (host): unit feature normalisation, He-normal weights, zero biases. */
int pnm_mlp_init(float *blob, unsigned long long seed);

/* Features (n x 32 floats), MBPT2 amplitudes (n doubles) and sigma_sys of system `sys`
 * in library amplitude order (any output may be NULL).  Computed on the GPU once per context. */
int pnm_mlp_features(pnm_ctx *ctx, int sys, float *X, double *t_mbpt2, double *sigma);

/* Train on the amplitudes currently held by the given contexts (after converged solves):
 * target (t - t_MBPT2) / sigma_sys.  Sets the blob's normalisation header from the data,
 * then runs Adam on the GPU (the library's forward/backward kernels; weights and layer inputs
 * in BF16, the matrix products of both passes on the tcgen05 tensor cores).  blob: in =
 * initial parameters, out = trained.  loss_hist (nullable, cap entries) gets the mean loss per
 * epoch (in units of y_scale^2); *n_hist the number of epochs.  PNM_ETIMEOUT if a bounded wait
 * of the tensor-core products ran out. */
int pnm_mlp_train(pnm_ctx *const *ctxs, int nctx, const pnm_mlp_opts *opts, float *blob,
                  float *loss_hist, int cap, int *n_hist);

/* Install a trained blob in a context for solves with init = PNM_INIT_MLP. */
int pnm_mlp_set_model(pnm_ctx *ctx, const float *blob);

/* Write the learned start, the amplitudes a solve with init = PNM_INIT_MLP begins from, into
 * the context's held amplitudes (pnm_get_amplitudes reads them): t_MBPT2 + sigma_sys y_scale
 * net(features) on the rows the updates compute, their spin flips on the others.  Needs a
 * model (PNM_EINVAL otherwise); PNM_ETIMEOUT if a bounded wait of the inference kernel ran
 * out (the held amplitudes are then incomplete). */
int pnm_mlp_predict(pnm_ctx *ctx);

/* Network output for n feature rows (host arrays).  mode: PNM_MLP_TENSOR_CORES runs the
 * fused tcgen05 inference kernel (the learned start's), PNM_MLP_SIMT the training
 * forward with its matrix products on the SIMT kernels, PNM_MLP_SIMT_FP32 the same SIMT kernels with the BF16 rounding of weights and
 * layer inputs switched off (a debug mode for element-wise checks against an FP64
 * reference).  stream: NULL = legacy stream. */
#define PNM_MLP_SIMT 0
#define PNM_MLP_TENSOR_CORES 1
#define PNM_MLP_SIMT_FP32 2
int pnm_mlp_forward(const float *blob, const float *X, long n, float *Y, int mode, void *stream);

/* Mean squared error over n samples and its gradient (NPARAM floats, header entries 0)
 * from the library's GPU forward/backward kernels, for gradient checks.  fp32 = 0: the BF16
 * training mode (weights and layer inputs rounded to BF16) with the matrix products on the
 * tcgen05 tensor cores, as pnm_mlp_train runs them (operands split into BF16 hi + lo, three
 * products, FP32 accumulation); 1: the FP32 debug mode (SIMT kernels, no BF16 rounding of
 * weights or activations); 2: the BF16 mode with the SIMT products.  PNM_ETIMEOUT if a bounded
 * wait of the tensor-core kernel ran out. */
int pnm_mlp_loss_grad(const float *blob, const float *X, const float *T, int n, float *loss,
                      float *grad, int fp32, void *stream);

/* Per-kernel device time of host-driven solves (opts.host_loop = 1): while profiling is on,
 * every kernel launch of the update is bracketed by CUDA events on the context stream.
 * pnm_set_profiling also clears the counters.  pnm_kernel_stats returns, for kernel id
 * (0, 1, ... until the call returns PNM_EINVAL), its name (static string), total
 * milliseconds and launch count.
 * Not from the paper: this is the library's own instrumentation. */
int pnm_set_profiling(pnm_ctx *ctx, int on);
int pnm_kernel_stats(const pnm_ctx *ctx, int id, const char **name, double *total_ms,
                     int *launches);

/* Choices of the context's autotuners (not from the paper).  Tile autotuner of the
 * tensor-core pp ladder (run when the mixed-precision path is first prepared): number of
 * k-range splits per (channel, ab tile) item, depth of the shared-memory copy ring and the
 * measured microseconds per launch.  Schedule autotuner (run at the first solve of each
 * precision): serial_mask bit 0 / bit 1 / bit 4 set when the FP64 update / the mixed update /
 * the refinement update with FP32-pair contractions runs on one stream instead of three
 * concurrent ones; bit 2 / bit 3 / bit 5 set while that mode is not tuned yet.
 * Any output may be NULL; PNM_EINVAL (after writing serial_mask) before the first
 * mixed-precision solve. */
int pnm_get_tuning(const pnm_ctx *ctx, int *ksplit, int *stages, float *us, int *serial_mask);

/* Failure-path self test (not from the paper): a one-thread kernel waits, with the bounded
 * wait the tensor-core kernels use, on an mbarrier nothing arrives on.  Expected result:
 * PNM_ETIMEOUT after about a second, the context still usable.  Nothing traps or hangs. */
int pnm_selftest_timeout(pnm_ctx *ctx);

/* FMA-rate microbenchmark (not from the paper): the measured peak FP64 (fp64 = 1) or FP32
 * (fp64 = 0) fused multiply-add rate of the current device in TFLOP/s (2 flop per FMA),
 * the roofline denominator of the ALU-bound kernels.  Runs two short kernels on `stream`
 * (NULL: the default stream) and synchronizes.  PNM_ECUDA / PNM_ENOMEM on failure. */
int pnm_measure_fma_peak(int fp64, void *stream, double *tflops);

/* Thread-local text describing the last failure of a pnm_* call on this thread. */
const char *pnm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PNMCC_H */
