/*
 * tdks.h -- C ABI of the GB300 real-time TDKS propagator (libtdks.so).
 *
 * One time step of real-time, real-space TDDFT as in Noda et al., "SALMON: Scalable Ab-initio
 * Light-Matter simulator for Optics and Nanoscience" (Comput. Phys. Commun.):
 *   - Kohn-Sham orbitals on a uniform Cartesian grid (Sec. 2.1), vacuum outside the cuboid or
 *     periodic in all directions;
 *   - the Hamiltonian of Eq. (TDKS) (isolated) or Eq. (TDKS_solid) (Bloch orbitals in the velocity
 *     gauge), with a local pseudopotential and Kleinman-Bylander separable projectors (Sec. 3.1)
 *     whose phase follows the vector potential (Sec. 4.1);
 *   - a truncated (4th order) Taylor expansion of exp(-iH dt) and a predictor-corrector step for
 *     the density-dependent potential (Program summary);
 *   - the density of Eq. (rho), the Hartree potential of Eq. (TDKS), adiabatic LDA exchange
 *     (Sec. 3.1), the dipole of Sec. 3.1 and the current of Eq. (macro_current).
 *
 * Discrete model (fixed by this library where the paper is silent):
 *   H_q = -1/2 sum_a D2_a - i sum_a q_a D1_a + |q|^2/2 + V_loc + V_H + V_x + V_NL^q,  q = k + A/c,
 *   D2, D1: 8th-order central differences (4 neighbours per side per axis: 25-point Laplacian),
 *   V_NL^q u = sum_{atom, p} E_p beta_p(r) e^{-i q.d} sum_r' beta_p(r') e^{i q.d'} u(r') dV,
 *   d = r - R_atom (nearest image).  Projectors are s, px, py, pz:
 *   beta = N {1, dx, dy, dz} exp(-d^2/(2 w^2)) (1 - d^2/rc^2)^2 for |d| < rc, each grid-normalised
 *   to sum beta^2 dV = 1.  Orbitals are normalised to sum |u|^2 dV = 1, occupation 2, k-weight w_k.
 *   Units: Hartree atomic units.
 *
 * Memory and threading contract:
 *   - Orbitals are DEVICE arrays owned by the caller, contiguous, layout [nk][norb][nz][ny][nx],
 *     complex interleaved (re, im): double2 for TDKS_F64, float2 for TDKS_F32.
 *   - The library owns its internal device workspaces (potentials, projector tables, FFT buffers),
 *     allocated in tdks_init and released in tdks_destroy.
 *   - Every call is enqueued on the CUDA stream given to tdks_init and returns without waiting,
 *     except calls that return host values (tdks_observables, tdks_read_step_observables,
 *     tdks_check), which synchronise that stream (tdks_copy_step_observables is their
 *     asynchronous counterpart).
 *   - A context is not thread-safe; use one context per host thread.
 *   - Errors are returned as tdks_status codes; tdks_last_error() gives a message (thread-local).
 *     No call throws across the ABI.
 */
#ifndef TDKS_H_
#define TDKS_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TDKS_ABI_VERSION 4

typedef struct tdks_ctx tdks_ctx;

typedef enum {
  TDKS_OK = 0,
  TDKS_EINVAL = 1,        /* invalid argument (null pointer, bad size, inconsistent grid/cell) */
  TDKS_ENOMEM = 2,        /* device or host allocation failed */
  TDKS_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
  TDKS_ETIMEOUT = 4,      /* a device-side wait of a tile kernel gave up (see tdks_set_wait_test) */
  TDKS_ENONFINITE = 5,    /* the norm monitor found a NaN/Inf orbital */
  TDKS_EUNSUPPORTED = 6   /* a valid request this build does not implement (e.g. grid too large) */
} tdks_status;

enum { TDKS_F64 = 0, TDKS_F32 = 1 };
enum { TDKS_FIELD_NONE = 0, TDKS_FIELD_STEP = 1, TDKS_FIELD_PULSE = 2, TDKS_FIELD_TABLE = 3 };

/* Uniform grid (Sec. 2.1).  n = points per axis (x, y, z); h = spacing (bohr).
 * periodic = 1: periodic cuboid of side L = n h; coordinates r_j = j h.
 * periodic = 0: vacuum outside the box (orbitals zero outside); coordinates r_j = (j-(n-1)/2) h. */
typedef struct { int n[3]; double h[3]; int periodic; } tdks_grid;

/* Cell of a periodic grid; must equal n*h per axis within 1e-9 relative.  Ignored if isolated. */
typedef struct { double L[3]; } tdks_cell;

/* Pseudo-atom: local part V(r) = -Z erf(|r-R|/sigma)/|r-R| (Sec. 3.1 local pseudopotential), and
 * `proj` = index of its projector set in the tdks_projector array, or -1 for none. */
typedef struct { double R[3]; double Z; double sigma; int proj; } tdks_atom;

/* Kleinman-Bylander s + p projector set (Sec. 3.1): energies E_s (s) and E_p (px, py, pz),
 * cutoff radius r_cut and Gaussian width `width` of the shape given above. */
typedef struct { double E_s, E_p, r_cut, width; } tdks_projector;

/* precision: TDKS_F64 (orbitals, stencil and all reductions in FP64) or TDKS_F32 (FP32 complex
 * orbitals and stencil; density, current, dipole, norms and the Poisson solve stay in FP64).
 * hartree: include V_H (1) or leave it out (0).
 * xc: adiabatic LDA of Sec. 3.1 -- 0 none, 1 Slater exchange, 2 exchange plus the Perdew-Zunger
 *     correlation of the electron gas (eps_c = g / (1 + b1 sqrt(rs) + b2 rs) for rs >= 1, else
 *     A ln rs + B + C rs ln rs + D rs, with g = -0.1423, b1 = 1.0529, b2 = 0.3334, A = 0.0311,
 *     B = -0.048, C = 0.0020, D = -0.0116; V_c = eps_c - (rs/3) d eps_c / d rs).  hartree = xc = 0
 *     gives linear propagation.  3: the Tran-Blaha modified Becke-Johnson exchange potential (Sec.
 *     4.1 names it beside the LDA) plus the correlation of 2; see tdks_set_mbj.  xc = 3 needs
 *     ncell <= 1 and keeps one more orbital array on the device (the predictor's orbitals).
 * pc: predictor-corrector on (1) or a single Taylor step with V(t) (0).
 * ncell: number of independent copies of the system propagated together (0 or 1: one).  With
 * ncell > 1 (periodic grids only) orbitals are [ncell][nk][norb][nz][ny][nx] and every cell has its
 * own density and potential; this is the batch of microscopic cells of the multiscale mode.
 * obs_at_start: 0 (default) tdks_step leaves the observables of the propagated state, J(t+dt) and
 * dipole(t+dt), which costs one extra derivative pass over every orbital after the last Taylor
 * stage; 1 it leaves those of the input state, J(t) and dipole(t), which the first Taylor stage
 * forms from the derivative sums it computes anyway (no extra pass; the values of the final state
 * then come from tdks_observables or the next step).  The multiscale step (tdks_ms_step) always
 * uses the end-of-step current, which the Maxwell update needs.
 * norb_offset, norb_total: the orbital range of this context when the orbitals of every k-point are
 * split over several contexts (orbital parallelism, Sec. 3.2: the paper distributes the orbitals over
 * processes and sums the density over them).  The context holds orbitals norb_offset .. norb_offset +
 * norb - 1 of norb_total per k-point.  norb_total = 0 means norb (the whole set; norb_offset must then
 * be 0).  A context with norb < norb_total holds a shard: H u, Taylor steps, the kick and
 * tdks_observables act on its own orbitals (its observables are the shard's partial sums, which the
 * caller adds over the shards), while the calls that form the density-dependent potential from the
 * orbitals (tdks_update_potential, tdks_step, tdks_ms_step, tdks_ground_state) return
 * TDKS_EUNSUPPORTED: this build has no exchange of densities between shards. */
typedef struct {
  int precision; int hartree; int xc; int pc; int ncell; int obs_at_start;
  int norb_offset; int norb_total;
} tdks_options;

/* Validate options for a grid with nk k-points and norb orbitals per k-point without creating a
 * context (host only, no GPU needed); tdks_init applies the same checks.  TDKS_OK, or TDKS_EINVAL /
 * TDKS_EUNSUPPORTED with a message (tdks_last_error). */
tdks_status tdks_check_options(const tdks_grid* grid, int nk, int norb, const tdks_options* opts);

/* Observables returned to the host. */
typedef struct {
  double J[3];        /* macroscopic current density, Eq. (macro_current) (periodic only; else 0) */
  double dipole[3];   /* d = -int r (rho - rho0) dr (Sec. 3.1)                                  */
  double norm_min;    /* min over orbitals of sum |u|^2 dV                                       */
  double norm_max;    /* max over orbitals                                                       */
  double e_band;      /* sum_k w_k sum_n 2 <u|T_q + V_loc + V_NL^q|u>                           */
  double n_elec;      /* int rho dr                                                              */
  double residual;    /* tdks_step: ||V_Hxc(t+dt) - V~||_2 / ||V_Hxc(t+dt)||_2 of the predicted V~   */
  double fallbacks;   /* tdks_step: predicted steps rejected so far (redone with the plain PC)       */
} tdks_obs;

/* Create a context: builds the projector tables (host), the local potential (device), the
 * FFT plans and buffers.  kpts = [nk][3] Bloch vectors (bohr^-1), kw = [nk] weights (sum 1).
 * norb = orbitals per k-point.  stream = cudaStream_t (NULL = legacy default stream).
 * Errors: TDKS_EINVAL for bad sizes or a projector sphere wider than half the periodic cell;
 * TDKS_EUNSUPPORTED for grids beyond this build's limits; TDKS_ENOMEM; TDKS_ECUDA. */
tdks_status tdks_init(const tdks_grid* grid, const tdks_cell* cell,
                      const tdks_atom* atoms, int natom,
                      const tdks_projector* projectors, int nproj,
                      const double* kpts, const double* kw, int nk, int norb,
                      const tdks_options* opts, void* stream, tdks_ctx** out);

/* Spatially uniform field as A'(t) = A(t)/c.  kind = TDKS_FIELD_NONE: A' = 0.
 * TDKS_FIELD_STEP: A'(t) = A0 for t > 0 (impulsive kick in the velocity gauge, Eq. impulsive_A).
 * TDKS_FIELD_PULSE: A'(t) = A0 cos^2[pi (t - T/2)/T] sin[-omega (t - T/2) - 2 pi cep], 0 < t < T
 * (Eq. pulse with a real amplitude A0 already divided by c).  Isolated systems ignore the field.
 * (TDKS_FIELD_TABLE is set with tdks_set_field_table.) */
tdks_status tdks_set_field(tdks_ctx* ctx, int kind, const double A0[3], double omega,
                           double T, double cep);

/* Pump-probe fields (Sec. 3.1: two successive pulses of the Eq. (pulse) form with a time delay):
 * adds A'(t) += A0 cos^2[pi (t' - T/2)/T] sin[-omega (t' - T/2) - 2 pi cep] for 0 < t' = t - t_delay < T
 * to a field set with kind TDKS_FIELD_PULSE (whose own pulse has delay 0); at most 8 pulses.
 * Errors: EINVAL if the field is not of kind PULSE, A0 is NULL, T <= 0, t_delay is not finite or
 * 8 pulses are set. */
tdks_status tdks_add_pulse(tdks_ctx* ctx, const double A0[3], double omega, double T, double cep,
                           double t_delay);

/* A field given by a numerical table (Sec. 3.1), as samples of A'(t) = A(t)/c: Ap[3 i + a] is
 * component a at t0 + i dt_table, i < nt; A' is linear between samples and equal to the first /
 * last sample before / after the table (an E(t) table becomes one of A' = -int E dt).  The table is
 * copied; it replaces the current field (kind TDKS_FIELD_TABLE).  Errors: EINVAL for a NULL table,
 * nt outside 1..2^26, dt_table <= 0 or a non-finite value. */
tdks_status tdks_set_field_table(tdks_ctx* ctx, const double* Ap, int nt, double t0, double dt_table);

/* Ground state (the static Kohn-Sham problem solved before the time evolution; the paper's ground-
 * state step uses Gram-Schmidt orthonormalisation): the lowest norb states of every k-point at A' = 0,
 * self-consistent in V_Hxc, for the context's synthetic pseudo-atoms.  Chebyshev-filtered subspace
 * iteration on a block of nb = norb + max(4, norb/4) states per k-point: each iteration filters the
 * block with the Chebyshev polynomial of the given degree that damps the spectrum between the block's
 * highest Ritz value and an upper bound of H (the FD kinetic symbol, the largest potential and a
 * Gershgorin bound of the projectors), orthonormalises it (Cholesky: the Gram-Schmidt of the set),
 * takes the Rayleigh-Ritz rotation (norb x norb problems on the host), puts the lowest norb Ritz vectors
 * into u, and mixes the potential linearly, V_in <- V_in + mix (V_Hxc[rho(u)] - V_in).
 * It stops when the residual sqrt(sum_occupied ||H u - e u||^2 / (nk norb)) and the potential misfit
 * ||V_Hxc[rho] - V_in|| / ||V_Hxc[rho]|| are both below tol, or after max_iter iterations.
 * u: caller's orbitals [nk][norb][nz][ny][nx] (the start; overwritten by the occupied Ritz vectors,
 * orthonormal).  Afterwards V_Hxc(t) and rho0 are those of the ground state.  degree <= 0 picks 10.
 * out[3] (nullable): iterations, final residual, band energy sum_k w_k sum_n 2 e_kn.  Allocates its
 * work blocks and a context of nb orbitals per k-point for the duration of the call; synchronises every
 * iteration.  Errors: EUNSUPPORTED for ncell > 1, norb > 64 or an orbital shard; EINVAL for bad
 * arguments or linearly dependent orbitals; ENOMEM. */
tdks_status tdks_ground_state(tdks_ctx* ctx, void* u, int max_iter, double tol, double degree, double mix,
                              double* out);

/* Number density of excited electron-hole pairs (Sec. 4.2 example; the paper gives no formula):
 * n_eh = (1 / Omega) sum_k w_k 2 (norb - sum_{m,n} |<phi_km|psi_kn> dV|^2), the occupied weight that has
 * left the ground-state subspace spanned by u_gs (e.g. from tdks_ground_state; both [nk][norb][npts],
 * device, the context's precision).  Projections on the ground-state orbitals of the same k; after the
 * field has returned to zero this is the gauge-independent count.  Synchronises.  Isolated systems
 * use Omega = the box volume.  Errors: EINVAL for NULL arguments; EUNSUPPORTED for ncell > 1. */
tdks_status tdks_excited_pairs(tdks_ctx* ctx, const void* u, const void* u_gs, double* n_eh);

/* Orbital energies (Sec. 2.1 ground-state outputs: discrete orbital energies of an isolated system,
 * energy bands at the k-points of a periodic one): for every k, the Ritz values of
 * H_q = T_q + V_loc + V_Hxc(t) + V_NL^q, q = k + Ap (Ap NULL: A' = 0), in the span of that k's orbitals
 * u (device, [nk][norb][nz][ny][nx], need not be orthonormal) -- the eigenvalues e of
 * M z = e S z, M_ij = <u_i|H_q|u_j> dV, S_ij = <u_i|u_j> dV (overlaps on the GPU, the norb x norb
 * problem on the host: Cholesky of S, Jacobi rotations of L^{-1} M L^{-H}).  eps: host [nk][norb],
 * ascending per k.  rotate = 1 also replaces u by the Ritz vectors (orthonormal, eigenvectors of the
 * projected problem; after tdks_ground_state these are the Kohn-Sham orbitals).  Synchronises.
 * Errors: EINVAL for NULL arguments, rotate outside 0..1, linearly dependent orbitals or no
 * potential yet; EUNSUPPORTED for ncell > 1 or norb > 64. */
tdks_status tdks_orbital_energies(tdks_ctx* ctx, void* u, const double Ap[3], int rotate, double* eps);

/* TB-mBJ exchange (xc = 3), the published Becke-Roussel / Becke-Johnson / Tran-Blaha forms per spin
 * channel of the unpolarised system (rho_s = rho/2, t_s = tau~/2):
 *   v_x = c v_BR + (3c - 2) (1/pi) sqrt(5/12) sqrt(2 t_s / rho_s),
 *   v_BR = -(1/b)(1 - e^-x - x e^-x / 2),  b = (x^3 e^-x / (8 pi rho_s))^(1/3),
 *   x e^(-2x/3) / (x - 2) = (2/3) pi^(2/3) rho_s^(5/3) / Q,  Q = (lap rho_s - 2 gamma D) / 6,
 *   D = 2 t_s - |grad rho_s|^2 / (4 rho_s),  gamma = 0.8,
 * with tau~ = tau - |j|^2 / (2 rho) the kinetic energy density of the orbitals whose density the
 * potential is formed from (tau = sum_k w_k sum_n |(D1 + i k) u|^2, j = sum_k w_k sum_n 2 Im(conj(u)
 * (D1 + i k) u); the current's share removed, so a uniform A' does not change it), derivatives by
 * the 8th-order differences, no potential where rho <= 1e-10.  tdks_set_mbj: c > 0 fixes c; c <= 0
 * (the default) forms c = -0.012 + 1.023 sqrt(g), g = (1/Omega) int |grad rho| / rho, from the
 * density every time the potential is formed (three kernels per potential instead of two).  The
 * setting is not part of a checkpoint.  tdks_mbj_c: the c of the last potential (synchronises).
 * Errors: EUNSUPPORTED unless the context has xc = 3; EINVAL for a non-finite c or a NULL output. */
tdks_status tdks_set_mbj(tdks_ctx* ctx, double c);
tdks_status tdks_mbj_c(tdks_ctx* ctx, double* c);

/* Longitudinal geometry (Sec. 4.1: in a thin film the vector potential is the external one plus the
 * one induced by the surface polarisation): A'(t) = A'_ext(t) + A'_ind(t) with
 * d^2 A'_ind / dt^2 = 4 pi J(t) (Gaussian units: E_ind = -4 pi P, dP/dt = J, E = -(1/c) dA/dt).  Each
 * tdks_step first advances A'_ind by the leapfrog A^{n+1} = 2 A^n - A^{n-1} + 4 pi dt^2 J(t_n) (the
 * first step from rest: A^1 = 2 pi dt^2 J(t_0)), on the device from the current the previous step
 * left, then propagates with A' = A'_ext(t + dt/2) + (A^n + A^{n+1})/2 and forms J(t + dt) with
 * A'_ext(t + dt) + A^{n+1}.  enable = 1 sets A'_ind = 0 and forms J(t0) of the orbitals u with
 * A'_ext(t0); enable = 0 switches it off.  The paper gives no equation for the induced potential;
 * this is the thin-film form of the works it cites.  Errors: EUNSUPPORTED unless the context has one
 * periodic cell, obs_at_start = 0 and no multiscale grid; EINVAL for a NULL u or enable outside 0..1.
 * tdks_longitudinal_read gives A'_ind at the end of the last step (synchronises). */
tdks_status tdks_set_longitudinal(tdks_ctx* ctx, int enable, const void* u, double t0);
tdks_status tdks_longitudinal_read(tdks_ctx* ctx, double A_ind[3]);

/* The context's field at time t (host values, no GPU work): Ap = A'(t) as tdks_step uses it, and
 * E = -dA'/dt (the electric field, E = -(1/c) dA/dt) by a central difference with step
 * h = 1e-6 max(1, |t|).  Either output may be NULL (not both).  Isolated systems report 0. */
tdks_status tdks_field_at(tdks_ctx* ctx, double t, double Ap[3], double E[3]);

/* Isolated impulse (Sec. 3.1): u <- exp(i kappa . r) u for all orbitals, in place. */
tdks_status tdks_kick(tdks_ctx* ctx, void* u_dev, const double kappa[3]);

/* rho <- rho[u] (Eq. rho), V_Hxc(t) <- V_H[rho] + V_xc[rho] (Eq. TDKS: the Hartree potential; Sec.
 * 3.1: the adiabatic LDA, with the terms the options select -- exchange, exchange + correlation, or
 * TB-mBJ exchange + correlation from the orbitals' kinetic energy density).  The first call also
 * stores rho as the reference density rho0 of the dipole.  Must be called once before tdks_step.
 * Errors: EINVAL for a NULL u; EUNSUPPORTED on an orbital shard (options.norb_total > norb). */
tdks_status tdks_update_potential(tdks_ctx* ctx, const void* u_dev);

/* hu <- H_q u for all orbitals: the Hamiltonian of Eq. (TDKS_solid) (Bloch orbitals in the velocity
 * gauge; Eq. (TDKS) for isolated grids, where q = 0) with q = k + Aprime, the current potential
 * V_loc + V_Hxc(t) and the Kleinman-Bylander projectors of Sec. 3.1 with the gauge phase of Sec. 4.1.
 * u, hu: device orbital arrays of the context's layout; they must not overlap.  Asynchronous.
 * Errors: EINVAL for NULL arrays. */
tdks_status tdks_hpsi(tdks_ctx* ctx, const void* u_dev, void* hu_dev, const double Aprime[3]);

/* u <- sum_{n=0..4} (-i dt H_q)^n u / n! in place (Horner form): the truncated Taylor expansion of the
 * evolution operator (Program summary), 4th order, with H_q as in tdks_hpsi (q = k + Aprime) and the
 * current potential V_loc + V_Hxc(t) held fixed over the step.  Asynchronous.  Errors: EINVAL for a
 * NULL u. */
tdks_status tdks_taylor_step(tdks_ctx* ctx, void* u_dev, double dt, const double Aprime[3]);

/* One predictor-corrector step t -> t + dt, in place (Program summary; Sec. 3.1, 4.1):
 *   predictor  u~ = T4[V_loc + V_Hxc(t)] u,  V~ = V_Hxc[rho(u~)];
 *   corrector  u(t+dt) = T4[V_loc + (V_Hxc(t) + V~)/2] u,  V_Hxc(t+dt) = V_Hxc[rho(t+dt)];
 * both with A'(t + dt/2).  (pc = 0: u(t+dt) = T4[V_loc + V_Hxc(t)] u.)  Afterwards J(t+dt)
 * (with A'(t+dt)) and the dipole of rho(t+dt) are in the step-observable buffer
 * (tdks_read_step_observables); with options.obs_at_start = 1, J(t) (with A'(t)) and the dipole of
 * rho(t) instead. */
tdks_status tdks_step(tdks_ctx* ctx, void* u_dev, double t, double dt);

/* Copy the observables written by the last tdks_step to the host (synchronises the stream).
 * J, dipole, n_elec, residual and fallbacks are filled; the other fields are set to 0. */
tdks_status tdks_read_step_observables(tdks_ctx* ctx, tdks_obs* out);

/* The same read without waiting, for callers that keep the stream busy while they read: enqueue on
 * the context stream the copy of the step-observable block of the last tdks_step (first cell) into
 * host_dst, TDKS_STEP_OBS_DOUBLES doubles owned by the caller:
 *   [0..2] J, [3..5] dipole, [6] n_elec, [7] 0, [8] misfit of the predicted potential, [9] 0,
 *   [10] fallbacks so far.
 * host_dst must be page-locked for the copy to run asynchronously (pageable memory makes the CUDA
 * runtime copy synchronously).  The block is valid once the stream has passed the copy (an event
 * recorded after it, or any synchronising call); tdks_unpack_step_observables then fills a
 * tdks_obs from it, exactly as tdks_read_step_observables would have.  Unpack blocks in the order
 * they were copied (the fallback count feeds the context's launch counters).
 * Errors: EINVAL for a NULL buffer or output. */
#define TDKS_STEP_OBS_DOUBLES 11
tdks_status tdks_copy_step_observables(tdks_ctx* ctx, double* host_dst);
tdks_status tdks_unpack_step_observables(tdks_ctx* ctx, const double* host_src, tdks_obs* out);

/* Compute all observables of u with A'(t) = Aprime, against the current rho0 and potential
 * (synchronises the stream): the current of Eq. (macro_current) including the nonlocal term, the
 * dipole d = -int r (rho - rho0) dr of Sec. 3.1 from the density of Eq. (rho), the orbital norms, the
 * band energy and the electron count.  rho_dev (nullable): a caller-owned device array [nz][ny][nx]
 * of doubles that receives rho[u].  Does not change the context's potential or density.  On an
 * orbital shard the sums run over the shard's orbitals only.  Errors: EINVAL for NULL u or out;
 * EUNSUPPORTED for ncell > 1. */
tdks_status tdks_observables(tdks_ctx* ctx, const void* u_dev, const double Aprime[3], double* rho_dev,
                             tdks_obs* out);

/* Copy a context array of the first cell (device-to-device, [nz][ny][nx] doubles) into a caller
 * buffer dst_dev:  which = 0: the local pseudopotential V_loc (Sec. 3.1); 1: V_Hxc(t), the Hartree
 * (Eq. TDKS) plus exchange-correlation (Sec. 3.1) potential of the last update; 2: rho(t) of Eq. (rho);
 * 3: the reference density rho0 of the dipole.  Asynchronous.  Errors: EINVAL for NULL dst_dev or
 * which outside 0..3. */
tdks_status tdks_get_grid_array(tdks_ctx* ctx, int which, double* dst_dev);

/* Wait for all work of the context's stream and report any asynchronous CUDA error. */
tdks_status tdks_check(tdks_ctx* ctx);

/* ---- Multiscale light propagation (Sec. 5) ----------------------------------------------------
 * A 1D grid of nX points (spacing dX, bohr) carries the z-component A(X) of the vector potential of
 * Eq. (Maxwell_ms); the ncell cells of the context sit at X = m0 .. m0 + ncell - 1 (1 <= m0,
 * m0 + ncell <= nX - 1), the other points are vacuum.  One tdks_ms_step: A(X, t+dt) by leapfrog from
 * the cells' currents I(X, t), first-order Mur absorbing boundaries at both ends; then every cell
 * takes one tdks_step-like predictor-corrector step with its own A'(t+dt/2) = (A(X,t)+A(X,t+dt))/(2c)
 * along z (Eq. TDKS_ms), and its current density J_z at t+dt (with A(X,t+dt)) becomes I(X, t+dt).
 * A_now, A_prev (host, [nX]): A at t = 0 and t = -dt (set the incident pulse here).
 * From the second tdks_ms_step after tdks_ms_init (or tdks_set_state) on, the step is one launch of a
 * CUDA graph holding all of its kernels (one graph per rotation of the three A levels, rebuilt when the
 * orbital array, dt or the kernel variants change; tdks_set_step_graph(ctx, 0) launches the kernels one
 * by one instead).  No host value enters the step after its first call: every cell's A' comes from the
 * device. */
tdks_status tdks_ms_init(tdks_ctx* ctx, int nX, int m0, double dX, const double* A_now,
                         const double* A_prev);
tdks_status tdks_ms_step(tdks_ctx* ctx, void* u_dev, double t, double dt);
/* Copy A(X, t) and I(X, t) (host arrays of nX, either may be NULL); synchronises the stream. */
tdks_status tdks_ms_read(tdks_ctx* ctx, double* A_host, double* I_host);

/* Points of the Maxwell grid of the multiscale mode (0 before tdks_ms_init or a restored state). */
tdks_status tdks_ms_size(const tdks_ctx* ctx, int* nX);

/* ---- Predictor of the self-consistent potential -------------------------------------------
 * TDKS_PRED_PC (default): predictor-corrector as in tdks_step.
 * TDKS_PRED_EXTRAP: the cubic through the last four potentials, V~(t+dt) = 4 V_Hxc(t)
 *   - 6 V_Hxc(t-dt) + 4 V_Hxc(t-2dt) - V_Hxc(t-3dt), replaces the predictor half-step (the
 *   no-network baseline of the learned predictor).
 * TDKS_PRED_LEARNED: V~(t+dt) = that cubic + s3 * NN(...) (network below).
 * In the two predicted modes a step runs one Taylor propagation with (V_Hxc(t) + V~)/2, forms
 * V_Hxc(t+dt) and the misfit r = ||V_Hxc(t+dt) - V~|| / ||V_Hxc(t+dt)||; if r > threshold the step is
 * undone and redone with the plain predictor-corrector (fallback).  Predicted steps need the last
 * four potentials: the first three steps after tdks_update_potential always use the PC.  The decision
 * is taken on the device: the step ends with a CUDA graph (built on the first predicted step, and again
 * when the orbital array, dt or the threshold change) whose decision kernel keeps V_Hxc(t+dt) or counts
 * a fallback and triggers a conditional node holding the restore and the plain step, so tdks_step does
 * not wait for the GPU.  The fallback count is read by tdks_read_step_observables. */
enum { TDKS_PRED_PC = 0, TDKS_PRED_EXTRAP = 1, TDKS_PRED_LEARNED = 2 };
tdks_status tdks_set_predictor(tdks_ctx* ctx, int mode, double threshold);

/* How predicted steps and multiscale steps are issued (no counterpart in the paper).  enable = 1
 * (default): as the CUDA graphs described above (for predicted steps one per slot of the four-potential
 * history, so that the graph's buffers are fixed, with the decision on the device; for multiscale steps
 * one per rotation of the A levels).  enable = 0: the same kernels launched one by one on the stream;
 * a predicted step then copies the misfit to the host and enqueues the fallback from there (one
 * synchronisation per step; every kernel appears as its own launch to profilers, which do not time the
 * kernel nodes of graphs that hold conditional nodes).  Both give the same results.  Errors: EINVAL for
 * enable outside 0..1. */
tdks_status tdks_set_step_graph(tdks_ctx* ctx, int enable);

/* ---- Learned potential predictor ------------------------------------------------------------
 * A 3-layer 3D convolutional network (4 -> 16 -> 16 -> 1 channels, 3^3 kernels with bias, SiLU,
 * circular padding for periodic grids, zero padding for isolated ones) with BF16 weights and
 * activations and FP32 accumulation.  From V0..V3 = V_Hxc(t), V_Hxc(t-dt), V_Hxc(t-2dt),
 * V_Hxc(t-3dt) and the backward differences D1 = V0-V1, D2 = V0-2V1+V2, D3 = V0-3V1+3V2-V3 (FP64),
 * the inputs are D1/s1, D2/s2, D3/s3, (V0-<V0>)/s_V, each s the root mean square of its field
 * (floored at 1e-13 rms(V0)); the output y corrects the cubic extrapolation C = 4 V0 - 6 V1 + 4 V2
 * - V3: V~ = C + s3 y.  Loss: mean squared error of y against (V_Hxc(t+dt) - C)/s3.  TDKS_NN_NPARAMS FP32 parameters, laid out W1[16][4][27], b1[16],
 * W2[16][16][27], b2[16], W3[1][16][27], b3[1]. */
#define TDKS_NN_NPARAMS 9105

/* Allocate the network buffers and initialise the parameters from `seed` (uniform in
 * +-1/sqrt(fan_in), last layer x0.1, biases 0) with a zeroed Adam state. */
tdks_status tdks_nn_init(tdks_ctx* ctx, unsigned long long seed);

/* Get (set = 0) or set (set = 1) the FP32 parameters through a host array of n = TDKS_NN_NPARAMS. */
tdks_status tdks_nn_params(tdks_ctx* ctx, float* host, int n, int set);

/* Train on a trajectory of potentials vseq_dev = [nt][npts] (device, FP64, V_Hxc at consecutive
 * steps): samples t = 3..nt-2, shuffled with `seed`, mini-batches of `batch`, Adam with learning
 * rate lr, `epochs` passes.  loss_out (host, nullable) receives the mean loss of every epoch.
 * Synchronises the stream once per epoch. */
tdks_status tdks_nn_train(tdks_ctx* ctx, const double* vseq_dev, int nt, int epochs, int batch,
                          double lr, unsigned long long seed, double* loss_out);

/* vpred_dev <- V~ from vhist_dev = [4][npts] (V0, V1, V2, V3): mode 0 = linear extrapolation
 * 2 V0 - V1, 1 = cubic extrapolation, 2 = the network. */
tdks_status tdks_nn_predict(tdks_ctx* ctx, const double* vhist_dev, double* vpred_dev, int mode);

/* Loss and parameter gradient of one sample (vhist_dev = [4][npts], vnext_dev = V_Hxc(t+dt)), without
 * updating the parameters; grad_host = [TDKS_NN_NPARAMS] (synchronises the stream). */
tdks_status tdks_nn_gradient(tdks_ctx* ctx, const double* vhist_dev, const double* vnext_dev,
                             double* loss_host, float* grad_host);

/* Phase timing and launch counting.
 * Phases: 0 predictor Taylor kernel, 1 corrector Taylor kernel (and tdks_taylor_step),
 * 2 tdks_hpsi kernel, 3 Hartree + exchange (density-to-potential), 4 observables,
 * 5 everything else (potential combination, memsets), 6 the orbital stencil kernel launches alone
 * (the shared-memory cell kernel, or the tile stencil kernel of large grids), nested inside phases
 * 0-2 and also counted there.  With timing enabled the library records a CUDA event pair around
 * each phase on the context stream (a few microseconds of overhead per step).  `launches` counts
 * this library's kernel launches since the last reset, timing on or off. */
#define TDKS_NPHASE 7
typedef struct {
  long long launches;
  long long calls[TDKS_NPHASE];
  double ms[TDKS_NPHASE];
} tdks_stats;

/* enable = 1 starts recording phase events, 2 records only the pair around the orbital stencil kernel
 * launches (phase 6; the other phases are counted but not timed, which keeps the event overhead of a
 * step small), 0 stops.  Errors: EINVAL for enable outside 0..2. */
tdks_status tdks_profile(tdks_ctx* ctx, int enable);

/* Sum the recorded phase times (synchronises the stream); reset = 1 clears counters and times. */
tdks_status tdks_stats_read(tdks_ctx* ctx, tdks_stats* out, int reset);

/* Sizes of the context (any pointer may be NULL). */
tdks_status tdks_query(const tdks_ctx* ctx, int* npts, int* nk, int* norb, int* precision,
                       int* nsphere_points);

/* Stencil kernel of large isolated grids (the TMA tile kernels; no counterpart in the paper, whose
 * stencil runs on CPU cores).  At tdks_init a context that uses them times every variant once on its
 * own grid and orbital count (the stencil alone, as H v and as a Horner stage, on zeroed work buffers)
 * and keeps the fastest for each of the two.
 * Variants (FP32): 0 = one grid point per thread, registers capped for 3 CTAs per SM, no L2 prefetch;
 * 1 = one point per thread, 2 CTAs per SM, TMA L2 prefetch of the planes 8 ahead; 2 = 2 x 2 points
 * per thread, 8 consumer warps, prefetch 8; 3 = 2 x 1 points per thread (one row), 8 consumer warps,
 * 2 CTAs per SM, prefetch 8; 4 = the same with 4 consumer warps and 4 CTAs per SM; 5, 6 = 3, 4 with
 * the potential (and for a Horner stage psi) of each plane delivered by TMA next to the orbital
 * plane instead of loaded per thread (grids with nx divisible by 4).  FP64: 0 and 1 (one CTA per SM,
 * without / with prefetch).
 *   set       : -1 leaves the choice as it is; 0..6 forces that variant for both uses.
 *   variant   : receives the variants in use [H v, Horner stage] (may be NULL).
 *   tune_ms   : receives the 14 tuning times in ms [use][variant], -1 where not timed (may be NULL).
 * Errors: EUNSUPPORTED if the context does not use the tile kernels or the variant does not apply
 * (FP32 only; nx % 4 for 5 and 6); EINVAL for set outside -1..6. */
tdks_status tdks_tile_variant(tdks_ctx* ctx, int set, int* variant, float* tune_ms);

/* Schedule of the FP32 projections of large grids (the batched contraction [orbitals x sphere points]
 * x [sphere points x 4] of the Kleinman-Bylander projections, Sec. 3.1, on the tensor cores; no
 * counterpart in the paper).  A CTA takes one atom and 16 orbitals; its warps take interleaved steps
 * of 8 sphere points: 0 = 2 warps, 1 = 4 warps, 2 = 8 warps per CTA.  At tdks_init a context that
 * uses the tile kernels in FP32 times the three on its own orbital count (zeroed orbitals) and keeps
 * the fastest.  The sums are the same products added in another grouping.
 *   set       : -1 leaves the choice as it is; 0..2 forces that schedule.
 *   variant   : receives the schedule in use (may be NULL).
 *   tune_ms   : receives the 3 tuning times in ms, -1 where not timed (may be NULL).
 * Errors: EUNSUPPORTED if the context does not use the FP32 tile kernels; EINVAL for set outside
 * -1..2. */
tdks_status tdks_project_variant(tdks_ctx* ctx, int set, int* variant, float* tune_ms);

/* Buffer scheme of the shared-memory cell kernels for the Taylor propagator (Eq. taylor, Horner
 * form; no counterpart in the paper).  0 = two orbital copies in shared memory (or a global scratch
 * slice when two do not fit), one stage reading one and writing the other; 1 = one copy swept in
 * place plane by plane, one thread per (x, y) column, for planes of at most 448 points -- half the
 * shared memory, so two FP32 CTAs share an SM; 2 = scheme 0 compiled for a fixed grid size (the
 * periodic 20^3 and 16^3 grids), each thread's column segment unrolled over its planes (FP32: two
 * x-adjacent points per thread); 3 = scheme 1 compiled for those grids with two points per thread
 * (FP32 only).  The arithmetic per grid point and per projection is the same in all four; the norm and
 * current sums of an orbital are split over the CTA's warps and may add in another order.  At
 * tdks_init a cell context on which scheme 1, 2 or 3 applies times one Taylor launch of each scheme
 * that applies on zeroed orbitals and keeps the fastest.
 *   set       : -1 leaves the choice as it is; 0..3 forces that scheme.
 *   variant   : receives the scheme in use (may be NULL).
 *   tune_ms   : receives the 4 tuning times in ms, -1 where not timed (may be NULL).
 * Errors: EUNSUPPORTED if the context uses the tile kernels, or set = 1, 2 or 3 where that scheme
 * does not apply; EINVAL for set outside -1..3. */
tdks_status tdks_cell_variant(tdks_ctx* ctx, int set, int* variant, float* tune_ms);

/* Checkpoint and restart of the time stepping (no counterpart in the paper's formulation; the
 * paper's code restarts from files).  The state is everything a context carries from step to step
 * besides the orbitals, which the caller owns and saves itself:
 *   V_Hxc(t), rho(t) and the reference density rho0 of every cell; the last four V_Hxc of the
 *   predictor history; the predictor mode, threshold, fallback count and network parameters; the
 *   multiscale field levels A^n, A^{n-1}, A^{n+1}, the cell currents and the grid geometry; the
 *   field settings (tdks_set_field, tdks_add_pulse, tdks_set_field_table) and the longitudinal
 *   geometry's induced potential and current.
 * tdks_state_size gives the bytes; tdks_get_state writes them to host memory (synchronises);
 * tdks_set_state restores them into a context created for the same system and options (grid
 * points, cells, k-points, orbitals, precision, atoms, hartree/xc/pc), checked against the
 * state's header: TDKS_EINVAL for a foreign or truncated state.  A restored context continues
 * exactly as the original would from the same orbitals. */
tdks_status tdks_state_size(const tdks_ctx* ctx, size_t* bytes);
tdks_status tdks_get_state(tdks_ctx* ctx, void* host_buf, size_t bytes);
tdks_status tdks_set_state(tdks_ctx* ctx, const void* host_buf, size_t bytes);

/* Measured FP64 FMA throughput of the current device in TFLOP/s (a 2-flop FMA counts 2), for the
 * roofline of the FP64 path; runs some tens of milliseconds of FMA chains on every SM (synchronises the
 * device; no context needed).  No counterpart in the paper. */
tdks_status tdks_probe_fp64(double* tflops);

/* Measured FP32 FMA throughput of the current device in TFLOP/s (an FMA counts 2): the higher of
 * scalar FMA chains and packed two-lane (f32x2) FMA chains on every SM, for the roofline of the FP32
 * cell kernels (synchronises the device; no context needed).  No counterpart in the paper. */
tdks_status tdks_probe_fp32(double* tflops);

/* Test hook of the device-side timeout path (no counterpart in the paper).  The tile kernels of large
 * isolated grids wait on shared-memory barriers for their TMA plane copies; every wait gives up after
 * a number of polls, sets the context's error word and the kernel returns (tdks_check then reports
 * TDKS_ETIMEOUT and clears the word; the context stays usable).
 *   wait_limit : polls per wait, 0 restores the default (2^22).  The final wait for the kernel's own
 *                copies in flight always uses the default, so no copy lands after its CTA exits.
 *   stop_after : >= 0 makes the copy producer issue only that many planes, so the stencil warps wait
 *                for a plane that never arrives and must give up; -1 (default) issues all planes.
 * Errors: EINVAL for wait_limit < 0. */
tdks_status tdks_set_wait_test(tdks_ctx* ctx, long long wait_limit, int stop_after);

/* Hartree + exchange potential of a density without allocating device memory.
 * For callers that cannot call cudaMalloc -- hosts whose device memory belongs to a pool they do not
 * control, loops that must never allocate -- this
 * computes vhxc = V_H[rho] + V_xc[rho] (hartree / xc select the terms, as in tdks_options; xc = 3,
 * TB-mBJ, needs the orbitals and returns TDKS_EINVAL here) for a
 * periodic or isolated grid with the same kernels as tdks_update_potential, using a fixed work area
 * built into the library (6 MiB of device memory per GPU that loads the library, held until the
 * process exits) instead of context buffers.  rho_dev and vhxc_dev are caller-owned device arrays
 * [nz][ny][nx] of doubles; stream is a cudaStream_t (NULL = legacy default stream); the call is
 * asynchronous.  Limit: FFT length <= 64 per axis (periodic n <= 64, isolated n <= 32) with prime
 * factors <= 31 and at most 64^3 FFT points; larger grids return TDKS_EUNSUPPORTED.  The first call
 * on each device looks up the work area's device address.  All calls share the one work area, so
 * calls that overlap on the GPU race.  The paper
 * has no counterpart: this is an interface variant of the Hartree/exchange step. */
tdks_status tdks_hxc_noalloc(const tdks_grid* grid, const double* rho_dev, double* vhxc_dev,
                             int hartree, int xc, void* stream);

/* Response analysis of a finished run (no context needed; FP64 on the GPU; host arrays in and out;
 * synchronous on `stream`, a cudaStream_t or NULL for the legacy default stream; device scratch is
 * allocated and freed inside the call).  Both transform a series x_i sampled at t_i = i dt,
 * i = 0..nt-1, with the cubic mask f(s) = 1 - 3 s^2 + 2 s^3 of s = t_i / T, T = (nt - 1) dt:
 *   F(w) = dt sum_i f(t_i / T) (x_i - xbar) exp(i w t_i).
 * Errors: EINVAL for a null array, nt < 2, nw outside 1..2^24, dt <= 0, kappa or Ap0 zero, or (eps
 * requested) a frequency <= 0; ENOMEM / ECUDA from the device. */

/* Oscillator-strength distribution, Sec. 3.1 Eq. (distribution), in Hartree units (m = hbar = e = 1):
 * dfdE[j] = -(2 E_j / (pi kappa)) Im F(E_j) for the dipole series d[nt] (one Cartesian component)
 * after the kick exp(i kappa r_nu) of tdks_kick (field impulse F0 = -kappa; dividing by the kick
 * strength makes the distribution positive and its integral over E the f-sum); xbar = 0. */
tdks_status tdks_oscillator_strength(const double* d, int nt, double dt, double kappa, const double* E,
                                     int nE, double* dfdE, void* stream);

/* Density of states (Sec. 2.1 ground-state outputs), spin-saturated, each level broadened by a
 * normalised Gaussian of width sigma: dos[j] = sum_k kw[k] sum_n 2 exp(-(E_j - eps[k][n])^2 /
 * (2 sigma^2)) / (sigma sqrt(2 pi)).  eps: [nk][norb] (tdks_orbital_energies), kw[nk], E[nE]; host
 * arrays, FP64 on the GPU, synchronous on `stream`.  Errors: EINVAL for a null array, nk * norb or nE
 * outside 1..2^24, sigma <= 0. */
tdks_status tdks_dos(const double* eps, int nk, int norb, const double* kw, const double* E, int nE, double sigma,
                     double* dos, void* stream);

/* Conductivity and dielectric function, Sec. 4.1 Eq. (sigma_ft):
 * sigma[2j], sigma[2j+1] = Re, Im of -(c / A0) F(w_j) = -F(w_j) / Ap0 for the current series I[nt]
 * (one component) after the vector-potential step A'(t) = Ap0 theta(t) (A' = A/c, as in
 * tdks_set_field); eps (nullable) = 1 + 4 pi i sigma / w in the same layout.  subtract_mean != 0
 * first removes the mask-weighted mean xbar = sum f I / sum f, which makes sigma(0) = 0 exactly
 * (the Sec. 4.1 example removes a small constant current for this reason); otherwise xbar = 0. */
tdks_status tdks_conductivity(const double* I, int nt, double dt, double Ap0, const double* w, int nw,
                              int subtract_mean, double* sigma, double* eps, void* stream);

/* Work done by the field per unit volume, Sec. 4.1: W(t_i) = int_0^{t_i} I(t').E(t') dt' for samples
 * I[3 i + a], E[3 i + a] at t_i = i dt (a cumulative trapezoid sum, W[0] = 0; host arrays, FP64 on the
 * GPU, synchronous on `stream`).  This is the electronic excitation energy per volume
 * (E_el(t) - E_el(0)) / Omega when the xc potential derives from an energy functional.  The sign is
 * the one that makes the work of the field on the electrons positive with I of Eq. (macro_current)
 * and E = -dA'/dt (the paper prints W = -int I.E dt', i.e. the opposite sign convention for one of
 * them).  Errors: EINVAL for a null array, nt outside 1..2^26 or dt <= 0; ENOMEM / ECUDA. */
tdks_status tdks_work(const double* I, const double* E, int nt, double dt, double* W, void* stream);

const char* tdks_last_error(void);
int tdks_abi_version(void);
void tdks_destroy(tdks_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* TDKS_H_ */
