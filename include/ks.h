/*
 * ks.h — C ABI of the GB300 Kohn-Sham hot path (plane-wave DFT/TDDFT, arXiv 2106.03872).
 *
 * One periodic cubic cell of side L (bohr), an N^3 real-space grid (N = 2^a 3^b, even,
 * 8 <= N <= 128), a kinetic cutoff sphere S = {G : |G|^2/2 <= ecut}, a local potential
 * V_loc (sum of Gaussians) and separable Kleinman-Bylander projectors (Eq. 9).  The
 * operator is H = P_S (-1/2 nabla^2 + V + V_NL) P_S (Eq. 2), applied in operator form:
 * kinetic in Fourier space, potential and projectors on the real-space grid, two FFTs
 * per application (Sec. "Implementation of the KS Hamiltonian").
 *
 * Units are atomic (bohr, hartree, hbar/hartree).  No call lets a C++ exception out.
 * Every call returns a ks_status; ks_last_error() gives a thread-local message.
 *
 * Canonical layouts (host side of the boundary):
 *   - state coefficients: [nstates][nG] complex128, interleaved (re, im) doubles, G in
 *     the canonical sphere order: grid index (j_x, j_y, j_z) row-major, z fastest,
 *     with m_i = j_i for j_i < N/2 else j_i - N and G = (2 pi / L) m;
 *   - real-space fields: [N][N][N] in grid order (x, y, z), z fastest, r_j = (L/N) j;
 *   - psi(r_j) = Omega^{-1/2} sum_{G in S} c_G exp(i G.r_j),  Omega = L^3.
 * Device buffers passed in are borrowed (never freed by the library) and are used in
 * stream order on the given stream (NULL = legacy default stream).
 */
#ifndef KS_H
#define KS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ks_grid_s* ks_grid;
typedef struct ks_server_s* ks_server;

typedef enum {
  KS_OK = 0,
  KS_ERR_ARG = 1,         /* invalid argument; nothing was changed                     */
  KS_ERR_NOMEM = 2,       /* device allocation failed or the memory budget is exceeded */
  KS_ERR_NOT_POSDEF = 3,  /* Gram matrix not positive definite (dependent states)      */
  KS_ERR_DIVERGED = 4,    /* real-time norm left [1 - 0.05, 1 + 0.05] x initial, or NaN */
  KS_ERR_TIMEOUT = 5,     /* ks_serve_poll limit expired                               */
  KS_ERR_CUDA = 6,        /* a CUDA runtime call or kernel failed                      */
  KS_PENDING = 7,         /* ks_serve_poll: request not finished yet                   */
  KS_ERR_STATE = 8        /* call not valid in the handle's current state              */
} ks_status;

/* Internal arithmetic of a handle (any other value: KS_ERR_ARG).
 *   KS_FP64          complex128 states, FP64 FFTs, FP64 everything (correctness anchor).
 *   KS_MIXED_BF16X3  complex64 states and FFTs; projector and Gram/rotation GEMMs on the
 *                    tensor cores with each FP32 operand split into two bf16 terms (3
 *                    products), FP32 accumulation; the Cholesky factor and the subspace
 *                    eigensolver in FP32 with FP64 refinement (FP64 Rayleigh quotients for the
 *                    reported eigenvalues; FP64 throughout with KS_OPT_FP64_SUBSPACE); norms
 *                    and energies in FP64. */
typedef enum { KS_FP64 = 0, KS_MIXED_BF16X3 = 1 } ks_precision;

/* Cell description (all host memory, copied by ks_grid_create).
 *   pos      [natoms][3] atom positions (bohr), any real values (wrapped periodically).
 *   V_loc(r) = sum_a vloc_depth * exp(-|r - R_a - L n|^2 / (2 vloc_width^2)), n in {-1,0,1}^3.
 *   nproj    1 (s) or 4 (s, p_x, p_y, p_z) Gaussian projectors per atom on the sphere
 *            |d| < proj_rc (d the minimum-image displacement), beta_s = exp(-d^2/(2 s^2)),
 *            beta_p = d_alpha exp(-d^2/(2 s^2)), s = proj_sigma, each normalised to
 *            dV sum beta^2 = 1; V_NL psi = sum_{I,l} proj_D beta_Il <beta_Il|psi> (Eq. 9).
 *   occ      [nstates] occupations f_k (NULL: all 1), used by the density (Eq. 1) and
 *            by the norm and energy reductions. */
typedef struct {
  double L;
  int N;
  double ecut;
  int natoms;
  const double* pos;
  double vloc_depth, vloc_width;
  int nproj;
  double proj_sigma, proj_rc, proj_D;
  int nstates;
  const double* occ;
  ks_precision prec;
} ks_cell_desc;

/* Options of a handle, set with ks_set_option.
 *   KS_OPT_FP64_SUBSPACE (value 0 or 1, default 0): on a mixed-precision handle, 1 factors the
 *     Gram matrix (Cholesky of S in ks_orthonormalize, ks_block_iteration, ks_scf) and
 *     diagonalises the subspace matrix (Rayleigh-Ritz in ks_rayleigh_ritz, ks_block_iteration)
 *     in FP64 on the GPU, with FP64 subspace products, as the FP64 path does; the states, their
 *     FFTs and GEMMs stay in the handle's precision.  0 takes an FP32 factor and eigensolver
 *     (with FP64 Rayleigh quotients for the reported eigenvalues).  No effect on KS_FP64. */
enum { KS_OPT_FP64_SUBSPACE = 1 };

/* Number of plane waves in the cutoff sphere for (L, N, ecut).  Host only: needs no GPU.
 * KS_ERR_ARG if N is not an even 2^a 3^b in [8, 128] or the sphere leaves the grid's
 * Nyquist box. */
ks_status ks_count_gvectors(double L, int N, double ecut, int* nG);

/* Build a handle: sphere tables, V_loc, projector tables and every device buffer the
 * calls below need are allocated here (sized by desc->nstates).  *out is NULL on error.
 * The handle owns its device memory; states start at zero. */
ks_status ks_grid_create(const ks_cell_desc* desc, ks_grid* out);
ks_status ks_grid_destroy(ks_grid g);

/* nG, and optionally m[3*nG] (integer frequencies, canonical order); m may be NULL. */
ks_status ks_grid_gvectors(ks_grid g, int* nG, int* m);

/* Device bytes the handle holds (for admission control). */
ks_status ks_grid_device_bytes(ks_grid g, size_t* bytes);

/* V_loc on the grid, [N^3] doubles in grid order (host). */
ks_status ks_get_vloc(ks_grid g, double* v_host);

/* Sets a handle option (the KS_OPT_* values above; the paper has no counterpart: its code runs
 * in FP64 throughout).  KS_ERR_ARG for an unknown option or value.  Takes effect with the next
 * call on the handle. */
ks_status ks_set_option(ks_grid g, int option, int value);

/* Copy host states in ([nstates][nG] complex128, converted to the handle's precision)
 * or out (converted back to complex128).  Synchronous. */
ks_status ks_set_states(ks_grid g, const double* c_host);
ks_status ks_get_states(ks_grid g, double* c_host);

/* Device pointer to the handle's resident states, [nstates][nG] complex of the handle's
 * precision (double2 for KS_FP64, float2 otherwise).  Owned by the handle. */
ks_status ks_states_device(ks_grid g, void** psi_dev);

/* H psi for nstates <= desc->nstates states (Eq. 2): hpsi = P_S (T + V + V_NL) psi.
 * psi_dev, hpsi_dev: device [nstates][nG] complex of the handle's precision; must not
 * overlap.  V is the handle's current potential: V_loc at creation; V_loc + v_H + v_x of
 * the last density used by ks_scf or by a real-time step with hartree_xc (a real-time step
 * without it resets V to V_loc).  Asynchronous on stream. */
ks_status ks_apply_h(ks_grid g, const void* psi_dev, void* hpsi_dev, int nstates, void* stream);

/* Same operation end to end from host memory: psi_host / hpsi_host are
 * [nstates][nG] complex128 (host); the copies in and out are part of the call.
 * Synchronous. */
ks_status ks_apply_h_host(ks_grid g, const double* psi_host, double* hpsi_host, int nstates);

/* Density of the resident states, n(r) = sum_k f_k |psi_k(r)|^2 (Eq. 1), written to
 * n_dev [N^3] in grid order; element type double for KS_FP64, float otherwise.
 * Accumulated over states in a fixed order (deterministic). */
ks_status ks_density(ks_grid g, void* n_dev, void* stream);

/* CholQR of the resident states (Sec. "Ground-state solution", orthogonalisation):
 * S = Psi^H Psi, S = L L^H, Psi <- Psi L^{-H}.  KS_FP64 factors S in FP64; the mixed
 * paths (nstates <= 160) take one FP32 Cholesky factor and inverse, refined to first order
 * with the FP64 triangular product L1^{-1} S L1^{-H}.
 * S_host_opt (may be NULL) receives S, [nstates][nstates] complex128 row-major,
 * S_ij = sum_G conj(c_iG) c_jG.  KS_ERR_NOT_POSDEF if S is not positive definite
 * (states unchanged then).  Synchronous (reads a status word). */
ks_status ks_orthonormalize(ks_grid g, double* S_host_opt, void* stream);

/* Rayleigh-Ritz on the resident states (subspace diagonalisation): H_sub = Psi^H H Psi,
 * eigen-decomposed on the GPU (ascending), Psi <- Psi U, and the handle's H Psi buffer
 * <- (H Psi) U.  eig_host [nstates] receives the Ritz values.  The states should be
 * orthonormal.  Synchronous. */
ks_status ks_rayleigh_ritz(ks_grid g, double* eig_host, void* stream);

/* niter steepest-descent block iterations (Sec. "Ground-state solution"), each:
 * CholQR -> H Psi -> Rayleigh-Ritz -> Psi <- Psi - alpha (H Psi - Psi diag(eps)),
 * alpha = 1/(ecut + max V_loc - min V_loc + proj_D).  eig_host [nstates] receives the
 * Ritz values of the last iteration.  Synchronous. */
ks_status ks_block_iteration(ks_grid g, int niter, double* eig_host, void* stream);

/* Block iterations with a choice of preconditioner: precond 0 is ks_block_iteration; precond 1
 * is the Teter-preconditioned steepest descent (Sec. "Ground-state solution", applied in
 * Fourier space), per iteration CholQR -> H Psi -> Rayleigh-Ritz -> for each state i with
 * residual R_i = H psi_i - eps_i psi_i and T_i = sum_G |G|^2/2 |R_iG|^2 / sum_G |R_iG|^2
 * (floored at (2 pi / L)^2 / 2, the smallest nonzero plane-wave kinetic energy):
 *   psi_iG <- psi_iG - K(|G|^2 / (2 T_i)) R_iG / (T_i + max V_loc - min V_loc + proj_D),
 *   K(x) = (27 + 18x + 12x^2 + 8x^3) / (27 + 18x + 12x^2 + 8x^3 + 16x^4)
 * (states with R_i = 0 unchanged).  eig_host as for ks_block_iteration.  Synchronous. */
ks_status ks_block_iteration_pc(ks_grid g, int niter, int precond, double* eig_host, void* stream);

/* Self-consistent field (Sec. "Ground-state solution").  The resident states are
 * orthonormalised (CholQR) and their density is the first input density n_in.  Each SCF
 * iteration:
 *   V = V_loc + v_H[n_in] + v_x[n_in];  eig_iters block iterations with this V;
 *   CholQR;  n_out = density of the states;  R = n_out - n_in;  r = dV sum_j |R_j|;
 *   mixer 0 (static linear): n_in <- n_in + mix R;
 *   mixer 1 (Pulay / DIIS):  with the last `history` (1..8) pairs (n_in_i, R_i) and
 *     alpha minimising |sum_i alpha_i R_i| (dV-weighted L2) subject to sum_i alpha_i = 1,
 *     n_in <- sum_i alpha_i (n_in_i + mix R_i);
 *   mixer 2 (Broyden, the paper's default; Broyden's second method, which updates an
 *     approximate inverse Jacobian G of R(n_in)): over the last `history` pairs, oldest
 *     first, G starts at -mix I and takes each secant pair (dn, dR) of consecutive pairs as
 *     G <- G + (dn - G dR) dR^T / (dR^T dR) (dV-weighted inner products; a pair with dR = 0
 *     is skipped); n_in <- n_in - G R.  History 1 is linear mixing.
 * Stops after max_iter iterations or once r < tol.  eig_out [max_iter][nstates] (may be
 * NULL) receives each iteration's Ritz values, resid_out [max_iter] (may be NULL) its r,
 * iters_done (may be NULL) the number of iterations run.  Afterwards the states are
 * orthonormal and V is the potential of the last iteration's n_in.  KS_ERR_ARG unless
 * max_iter >= 0, eig_iters >= 1, mixer in {0, 1, 2}, 0 < mix <= 1, 1 <= history <= 8 and
 * tol >= 0; KS_ERR_DIVERGED if r is not finite.  Synchronous. */
ks_status ks_scf(ks_grid g, int max_iter, int eig_iters, int mixer, double mix, int history, double tol,
                 double* eig_out, double* resid_out, int* iters_done, void* stream);

/* nsteps real-time steps of dt (Sec. "Real-time propagation").
 *   propagator 0: ETRS (Eq. 6) with H(t+dt) from the density of the full step (Eq. 7);
 *                 the powers H(t)^k psi, k = 1..4, are shared by the exp(-i dt H) and
 *                 exp(-i dt/2 H) Taylor series (Eq. 8): 8 H applications per step.
 *   propagator 1: plain 4th-order Taylor step psi <- sum_k (-i dt H(t))^k/k! psi.
 *   hartree_xc 1: V(t) = V_loc + v_H[n(t)] + v_x[n(t)] recomputed from the density at the
 *                 start of every step (periodic Poisson in Fourier space with v_H(G=0)=0,
 *                 LDA Slater exchange); 0: V = V_loc fixed.
 * norm_out[s] = sum_k f_k ||psi_k(t_s)||^2 and energy_out[s] = E(t_s) (Eq. 5 with the
 * eigenvalue sum replaced by sum_k f_k <psi_k|H(t_s)|psi_k>), t_s the start of step s;
 * both may be NULL.  KS_ERR_DIVERGED if a norm leaves 5% of the first one.
 * Synchronous (copies norms and energies back at the end). */
ks_status ks_td_step(ks_grid g, double dt, int nsteps, int propagator, int hartree_xc,
                     double* norm_out, double* energy_out, void* stream);

/* ks_td_step that also records the dipole at the start of every step: dipole_out
 * [nsteps][3] (may be NULL) receives d(t_s) = dV sum_j (r_j - L/2) n(r_j, t_s), the first
 * moment of the density (Sec. "Validation with other codes": the observable of the kicked
 * response), r_j = (L/N) (jx, jy, jz).  With hartree_xc the density is the one the step
 * computes anyway; without it one density per step is added. */
ks_status ks_td_step_dipole(ks_grid g, double dt, int nsteps, int propagator, int hartree_xc,
                            double* norm_out, double* energy_out, double* dipole_out, void* stream);

/* Delta kick (Sec. "Validation with other codes": a time-localised field at t = 0): every
 * resident state psi_k(r) <- exp(i kappa . (r - L/2)) psi_k(r), projected back onto the
 * sphere S.  kappa[3] (host, bohr^-1, finite).  The phase is periodic only when kappa is a
 * reciprocal-lattice vector; otherwise the kick assumes states that vanish near the cell
 * boundary (a molecule in a box).  Asynchronous on stream. */
ks_status ks_kick(ks_grid g, const double* kappa, void* stream);

/* Forces on the atoms from the orbital gradients (Sec. "Forces", Eq. 11), for the resident
 * states with their occupations:
 *   F_I = -sum_k f_k [<grad psi_k| v_I |psi_k> + c.c.],
 * v_I the atom's local Gaussian (27 periodic images) and KB projectors; the overall sign is
 * that of -dE/dR_I (the paper prints the opposite).  The gradient is i G c in Fourier space;
 * local part dV sum_j v_I(r_j) sum_k f_k 2 Re(conj(grad psi_k) psi_k)(r_j), nonlocal part
 * sum_k f_k sum_l 2 D Re(conj(<beta_Il|grad psi_k>) <beta_Il|psi_k>) on the grid.  f_out
 * [natoms][3] (host, Ha/bohr); nothing is written when natoms = 0.  Synchronous. */
ks_status ks_forces(ks_grid g, double* f_out, void* stream);

/* Moves the atoms (Sec. "Real-time propagation": the ionic potential is recomputed for each
 * ionic configuration).  pos [natoms][3] (host, bohr, finite; positions outside [0, L) are
 * periodic images).  Rebuilds, for the same atoms and parameters as at creation: the
 * projector spheres |r_j - R_I| < proj_rc (minimum image) with their normalised beta values,
 * the projector block of the mixed path (FP64 DFT over each atom's box of grid points), and
 * V_loc from the separable 27-image Gaussians (in FP64 on the device).  The potential V
 * becomes the new V_loc (a following SCF or real-time step recomputes Hartree and exchange).
 * The states are kept.  No-op when natoms = 0.  KS_ERR_ARG on a non-finite position.
 * Synchronous. */
ks_status ks_set_positions(ks_grid g, const double* pos, void* stream);

/* The current positions pos [natoms][3] (host, bohr). */
ks_status ks_get_positions(ks_grid g, double* pos);

/* nsteps steps of Ehrenfest dynamics (Sec. "Real-time propagation"): the resident states
 * follow the ETRS step of ks_td_step (propagator 0, Hartree and exchange when hartree_xc)
 * and the atoms classical equations of motion under the forces of ks_forces (Eq. 11), by
 * velocity Verlet:
 *   R(t+dt) = R(t) + v(t) dt + F(t) dt^2 / (2 M);
 *   the ETRS step with H(t) at R(t) and H(t+dt) at R(t+dt) (the ions move between the two
 *   half steps, so that each half step sees the ionic potential of its own time);
 *   F(t+dt) from the new states at R(t+dt);  v(t+dt) = v(t) + (F(t) + F(t+dt)) dt / (2 M).
 * mass [natoms] (host, electron masses, > 0); vel [natoms][3] (host, bohr per atomic time
 * unit): v(0) in, v(t_nsteps) out.  pos_out [nsteps][natoms][3] (may be NULL) receives the
 * positions after each step; energy_out [nsteps] (may be NULL) the total energy at the start
 * of each step: the energy of ks_td_step plus sum_I M_I |v_I|^2 / 2.  The handle's positions
 * end at R(t_nsteps).  KS_ERR_ARG unless nsteps >= 0, dt > 0 and masses and velocities are
 * valid; KS_ERR_DIVERGED as for ks_td_step.  Synchronous. */
ks_status ks_ehrenfest(ks_grid g, double dt, int nsteps, int hartree_xc, const double* mass, double* vel,
                       double* pos_out, double* energy_out, void* stream);

/* Dipole of the resident states' density, d_out[3] (host) = dV sum_j (r_j - L/2) n(r_j).
 * Synchronous. */
ks_status ks_dipole(ks_grid g, double* d_out, void* stream);

/* ---------------------------------------------------------------------------------- */
/* Serving: continuous batching of independent calculations on one GPU.               */
/* ---------------------------------------------------------------------------------- */

/* A server owns worker threads and admits requests while the device memory they need fits in
 * mem_budget_bytes (0: 80% of the free device memory at creation).  The requests' device memory
 * comes from a slab pool the server keeps until ks_serve_destroy, so admitting and retiring
 * requests does not synchronise the device.  Real-time requests (kind 1) of mixed precision on
 * one grid geometry (same L, N, ecut) are stepped together, up to eight at a time, each H
 * application of their ETRS step one packed launch over all their states; a request's results
 * are the same alone and in such a group.  ks_serve_create starts 16 workers (each runs one
 * request's or group's quantum at a time, so long single-SM quanta do not hold the others). */
ks_status ks_serve_create(size_t mem_budget_bytes, ks_server* out);
/* Same with `workers` worker threads (1..64; 0: the default of 16). */
ks_status ks_serve_create_ex(size_t mem_budget_bytes, int workers, ks_server* out);
/* Stops the scheduler after the running requests finish; pending ones are dropped. */
ks_status ks_serve_destroy(ks_server s);

/* Queue one calculation: desc (copied; prec honoured) with initial states c0
 * ([nstates][nG] complex128 host, copied now; NULL = seeded random start orthonormalised
 * on the device), kind 0: `count` block iterations (result: Ritz values), kind 1: `count`
 * ETRS steps of dt with Hartree + exchange (result: energies per step).
 * KS_ERR_NOMEM if the request alone can never fit the budget. */
ks_status ks_serve_submit(ks_server s, const ks_cell_desc* desc, const double* c0, int kind,
                          int count, double dt, uint64_t* ticket);

/* Wait up to timeout_ms (0: do not wait) for a ticket.  KS_PENDING if still queued or
 * running after a zero wait, KS_ERR_TIMEOUT if the limit expired.  On KS_OK,
 * result_out receives nstates Ritz values (kind 0) or count energies (kind 1), c_out_opt
 * (may be NULL) the final states, latency_s_opt (may be NULL) submit-to-finish seconds;
 * the ticket is then released. */
ks_status ks_serve_poll(ks_server s, uint64_t ticket, int timeout_ms, double* result_out,
                        double* c_out_opt, double* latency_s_opt);

/* Counters of a server since its creation (no counterpart in the paper), out[0..nout-1] of:
 * worker seconds spent creating requests' engines and initial states, in ground-state quanta
 * (block iterations), in real-time steps (each group step counted once), in retiring requests;
 * then the number of request starts, ground-state quanta, real-time group steps, request-steps
 * in those groups (their ratio is the mean group size), and the bytes the server's device pool
 * holds; then the parts of the start time (engine creation, initial states, orthonormalisation
 * of real-time requests), the number of slabs the device pool obtained from the device and the
 * seconds spent obtaining them.  nout <= 14. */
ks_status ks_serve_stats(ks_server s, double* out, int nout);

/* Result sizes for a ticket: number of doubles in result_out, nstates, nG. */
ks_status ks_serve_result_info(ks_server s, uint64_t ticket, int* nresult, int* nstates, int* nG);

/* ---------------------------------------------------------------------------------- */
/* Instrumentation (no counterpart in the paper).                                      */
/* ---------------------------------------------------------------------------------- */

/* mode 1: record a CUDA event pair on the launching stream around every stage of the
 * handle's calls (H application, line FFTs, Gram, rotations, Cholesky, eigensolver, ...);
 * mode 0: stop recording; mode 2: drop the accumulated entries and spans; mode 3: also keep
 * every recorded stage as a span on a common clock (restarts the clock, drops old spans);
 * mode 4: stop keeping spans.  Spans need mode 1 as well. */
ks_status ks_profile(ks_grid g, int mode);

/* Entry idx (0-based) of the accumulated stage timings: name (NUL-terminated, truncated to
 * name_len), total milliseconds and number of timed scopes.  Waits for pending events.
 * KS_ERR_ARG once idx passes the last entry. */
ks_status ks_profile_read(ks_grid g, int idx, char* name, int name_len, double* ms, long* count);

/* Span idx (0-based, in order of completion collection) of the timeline started by mode 3:
 * stage name (NUL-terminated, truncated to name_len) and its start and end in milliseconds
 * after the first stage recorded since mode 3.  Stages on the side stream of the block
 * iteration appear beside the main stream's, so their overlap can be read off.  Waits for
 * pending events.  KS_ERR_ARG once idx passes the last span. */
ks_status ks_profile_span(ks_grid g, int idx, char* name, int name_len, double* start_ms, double* end_ms);

/* The status a call returns for the error word of the tensor-core GEMM kernels, which every
 * handle reads after its calls: flag 0 gives KS_OK; a nonzero flag (a bounded mbarrier wait in a
 * kernel expired after about 2 s; the kernel recorded it and returned) gives KS_ERR_CUDA with a
 * message in ks_last_error.  Host only: lets the expiry path be checked without a GPU. */
ks_status ks_tc_status_check(int flag);

/* The launch-shape autotuner's decisions so far, as JSON: the first H application or density of
 * each (grid, bucket of state counts) times the candidate plane kernels (team-owned line
 * transforms and CTA-wide Stockham stages) on the live data and keeps the faster one for the
 * process; the report lists, per decision, each candidate's best time in ms and the choice:
 *   [{"key": "plane N=96 states<=128", "ms": {"team": 0.69, "cta": 0.72}, "choice": "team"}, ...]
 * buf (may be NULL) receives at most cap bytes including the terminating NUL; len (may be NULL)
 * the size the whole report needs.  (The paper has no counterpart.) */
ks_status ks_autotune_report(char* buf, size_t cap, size_t* len);

/* Number of kernels this library has launched in this process so far. */
uint64_t ks_kernel_launches(void);

/* ---------------------------------------------------------------------------------- */
/* Allocation-free overlap (the paper has no counterpart).                             */
/* ---------------------------------------------------------------------------------- */

/* out[i][j] = sum_g conj(a[i][g]) b[j][g] for i < m, j < n: the overlap (Gram) matrix of two
 * device blocks, for callers that cannot allocate device memory: code whose device memory is
 * all handed to its own pool allocator, or latency-critical loops that cannot take the device
 * synchronisation a cudaMalloc/cudaFree may imply.  It needs no ks_grid and calls no cudaMalloc,
 * cudaFree or allocating library routine.
 *   a_dev [m][nG], b_dev [n][nG]: complex device arrays, double2 if fp64 != 0, else float2.
 *   out_dev [m][n]: complex128 device array written by the call (row-major).
 * Arithmetic: a split-K CUDA-core GEMM (the FP64 path's Gram kernel).  fp64 != 0: FP64
 * throughout, as ks_orthonormalize on a KS_FP64 handle.  fp64 == 0: FP32 products accumulated
 * in FP32 within each K range, the ranges summed in FP64; this is not the split-BF16
 * tensor-core kernel a mixed-precision handle's ks_orthonormalize uses, so the two agree to
 * FP32 rounding, not bit for bit.
 * The split-K partial sums live in a fixed 4 MiB device array inside the library (262,144
 * complex128 values), which every GPU that loads the library keeps until the process exits;
 * m * n above 262,144 is rejected with KS_ERR_ARG before any device work.  The array's device
 * address is looked up (cudaGetSymbolAddress) on the first call in each CUDA context, with
 * that context's device current; with lazy module loading that first call (or the library's
 * first kernel launch on the device) may also load the module and reserve the 4 MiB, with the
 * synchronisation that implies.  So make one call per device during set-up, outside
 * latency-critical regions and before any stream capture (and again after the context is
 * reset).  All calls share the array and it keeps the last call's contents; nothing in it has
 * to start at zero (every partial is written before it is read), but calls that overlap on the
 * GPU (different streams, or different host threads on one device) race on it and must be
 * serialised by the caller.  Asynchronous on stream. */
ks_status ks_overlap_noalloc(const void* a_dev, const void* b_dev, int m, int n, int nG, int fp64, void* out_dev,
                             void* stream);

/* Thread-local text of the last error of this thread (never NULL). */
const char* ks_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* KS_H */
