/*
 * qlbm.h -- C ABI of a GB300 (sm_103a) library for the matrix-valued quantum
 * lattice Boltzmann method of C. B. Mendl, "Matrix-valued Quantum Lattice
 * Boltzmann Method" (2015).
 *
 * The library advances populations W_i(x,t), each a Hermitian 2x2 matrix
 * (Sec. 2), on a periodic D2Q9 or D3Q19 lattice (Sec. 3) with the step of
 * Sec. 3.3: moments (Eq. DiscrAvr), polynomial Fermi-Dirac equilibrium
 * (Eq. WeqAlgo, coefficients of the appendix), BGK collision
 * (Eq. CollisionStep) and streaming (Eq. TransportStep).  All compute runs in
 * the library's own CUDA kernels on one GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice: QLBM_D2Q9 (d = 2, b = 9) or QLBM_D3Q19 (d = 3, b = 19).  Direction
 *   q has lattice vector i_q in {-1,0,1}^d (D3Q19: |i1|+|i2|+|i3| <= 2) and
 *   velocity e_q = xi * i_q (Sec. 3.1); q enumerates the vectors with i1
 *   varying fastest, then i2, then i3, so the opposite of q is b-1-q.
 * Sites: dims = {nx, ny, nz} (nz = 1 for D2Q9), N = nx*ny*nz, flat site
 *   index s = x + nx*(y + ny*z), periodic in every direction (Sec. 3).
 * Pauli form: a Hermitian W is given by four reals (f, s_x, s_y, s_z) with
 *   W = (f 1 + s_x sigma_x + s_y sigma_y + s_z sigma_z)/2, i.e. f = tr W and
 *   s = tr(W sigma), the Bloch-vector convention of Sec. 4.
 * Canonical state layout: double [b][4][N] (direction, Pauli component,
 *   site); this is the order of get/set_state and of adjoint cotangents.
 * Moment fields: rho4 double [4][N] = (tr rho, tr(rho sigma_x),
 *   tr(rho sigma_y), tr(rho sigma_z)); u double [d][N]; eps double [N].
 * Units: tau and dt in the same time unit, omega = dt/tau (Eq. CollisionStep);
 *   streaming moves one cell per step (dt xi = dx, Sec. 3.3).
 * Pointers: every pointer argument is owned by the caller and only read or
 *   written during the call (asynchronously on the handle's stream for
 *   device pointers, see each entry point); ptr_kind says whether it is host
 *   memory (QLBM_HOST) or device memory of the handle's GPU (QLBM_DEVICE).
 *   Host buffers are copied synchronously.  The library owns all memory it
 *   allocates and frees it in qlbm_destroy.
 * Errors: every int-returning call returns QLBM_OK (0) or a negative
 *   qlbm_status; no exception crosses the ABI.  The message of the last
 *   failure is available from qlbm_last_error.  The step kernels record
 *   non-finite or non-positive densities in a device flag word that the next
 *   synchronising call (qlbm_sync, qlbm_moments, qlbm_conserved,
 *   qlbm_get_state, qlbm_rollout_adjoint) reports and clears.
 * Streams: all device work is issued on the stream given to qlbm_create
 *   (NULL = the legacy default stream).  A handle must not be used from two
 *   host threads at once.
 */
#ifndef QLBM_H
#define QLBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum qlbm_status {
    QLBM_OK = 0,
    QLBM_ERR_INVALID_ARG = -1,        /* bad size, pointer, parameter or lattice */
    QLBM_ERR_UNSUPPORTED = -2,        /* combination not provided by the library */
    QLBM_ERR_OOM = -3,                /* device allocation failed */
    QLBM_ERR_CUDA = -4,               /* a CUDA runtime call failed */
    QLBM_ERR_NONFINITE = -5,          /* a step met a NaN or infinite moment */
    QLBM_ERR_NONPOSITIVE_DENSITY = -6,/* a step met tr rho <= 0 */
    QLBM_ERR_STATE = -7               /* call not valid in the handle's state */
} qlbm_status;

typedef enum qlbm_lattice { QLBM_D2Q9 = 2, QLBM_D3Q19 = 3 } qlbm_lattice;

/* Storage precision of the populations.  QLBM_FP64 computes in double;
   QLBM_FP32 stores and computes in float; QLBM_FP16_DEV stores the deviation
   W_i - W_i^ref from a uniform reference equilibrium in half precision and
   computes in float; QLBM_DF64 stores each value as an unevaluated sum of two
   floats (8 bytes, 48-bit significand) and computes in double-float
   arithmetic on the single-precision pipes (results within ~1e-14 of double
   per step; no reverse mode: the adjoint calls return
   QLBM_ERR_UNSUPPORTED).  QLBM_FP64_DF stores IEEE doubles exactly as
   QLBM_FP64 does (same layout, same exact state read-out and set-up, same
   moments, reductions and Fermi-Dirac kernels) but steps in double-float
   arithmetic: each double is split into two floats, the step runs on the
   single-precision pipes and rounds its result to double (within ~1e-14 of
   the QLBM_FP64 step per step; no reverse mode).  Both double-float
   precisions have single precision's exponent range: magnitudes below
   2^-126 (~1.2e-38) are read as signed zeros and every stepped value
   carries an absolute error up to ~2^-126 besides the relative one;
   magnitudes from 2^128 on are flagged as non-finite. */
typedef enum qlbm_precision {
    QLBM_FP64 = 0,
    QLBM_FP32 = 1,
    QLBM_FP16_DEV = 2,
    QLBM_DF64 = 3,
    QLBM_FP64_DF = 4
} qlbm_precision;

typedef enum qlbm_ptr_kind { QLBM_HOST = 0, QLBM_DEVICE = 1 } qlbm_ptr_kind;

typedef struct qlbm_ctx *qlbm_handle;

/* qlbm_create -- set up a lattice (Sec. 3.3: the scheme's inputs are the
 * relaxation time tau and the reference inverse temperature beta0 of the
 * quadrature).
 *   out        receives the handle (unchanged on failure)
 *   lattice    QLBM_D2Q9 or QLBM_D3Q19
 *   dims       {nx, ny, nz}; nz must be 1 for D2Q9; every entry >= 1
 *   tau        relaxation time, > 0
 *   beta0      reference inverse temperature of the quadrature (Sec. 3.1), > 0;
 *              fixes xi = const/sqrt(beta0) and the weights (Eqs.
 *              QuadSolution2Dmu0, QuadSolution3Dmu0)
 *   dt         time step, > 0 (omega = dt/tau)
 *   precision  qlbm_precision
 *   stream     cudaStream_t to issue work on, or NULL
 * Allocates the single in-place population buffer (b*4*N values of the
 * storage type, padded per plane) and small scratch on the current device.
 * The state is undefined until qlbm_init_equilibrium or qlbm_set_state.
 * Returns QLBM_ERR_OOM if the buffer does not fit. */
int qlbm_create(qlbm_handle *out, int lattice, const int64_t dims[3], double tau,
                double beta0, double dt, int precision, void *stream);

/* Releases all device memory of the handle (after synchronising its stream).
   NULL is accepted. */
void qlbm_destroy(qlbm_handle h);

/* Message of the most recent failure on this handle, or of the last failed
   qlbm_create when h is NULL.  Valid until the next call on the handle. */
const char *qlbm_last_error(qlbm_handle h);

/* qlbm_info -- the lattice constants this handle uses, computed in double on
 * the host at qlbm_create from the quadrature's moment conditions (Eqs.
 * quadrature2D/3D) and the equilibrium's (Sec. 3.2, appendix).
 * out[0..15] = {d, b, xi, a, w_rest, w_axis, w_diag, beta0*eps0 (= c),
 *               beta0^2 <(p^2/2)^2>_0 (= m), alpha3, alpha4, alpha5,
 *               tau, beta0, dt, precision}; n must be >= 16. */
int qlbm_info(qlbm_handle h, double *out, int n);

/* qlbm_init_equilibrium -- initial state W_i(x,t0) = W_i^eq(rho(x), u(x),
 * eps(x)) of Eq. WeqAlgo at every site (Sec. 3.3: the scheme starts from
 * given populations at t0).
 *   rho4  [4][N] Pauli density (tr rho must be > 0)
 *   u     [d][N] velocity
 *   eps   [N] internal energy, or NULL for eps0, the internal energy of the
 *         quadrature's own Fermi-Dirac weight (beta0, mu0 = 0)
 * Resets the step counter to 0.  Device inputs are read on the stream;
 * host inputs are staged through the library and copied before return. */
int qlbm_init_equilibrium(qlbm_handle h, const double *rho4, const double *u,
                          const double *eps, int ptr_kind);

/* qlbm_step -- nsteps >= 0 time steps t -> t + dt of Sec. 3.3, each one
 * fused kernel launch (moments, equilibrium, collision and in-place
 * streaming).  Asynchronous: returns after queueing the launches. */
int qlbm_step(qlbm_handle h, int64_t nsteps);

/* Number of steps taken since the last init/set_state. */
int64_t qlbm_time(qlbm_handle h);

/* Waits for the handle's stream and reports (then clears) the step kernels'
   device flags as QLBM_ERR_NONFINITE / QLBM_ERR_NONPOSITIVE_DENSITY. */
int qlbm_sync(qlbm_handle h);

/* qlbm_moments -- local moments of Eq. DiscrAvr at the current time:
 * rho4 [4][N], u [d][N], eps [N] (any of the three may be NULL).  Computed
 * in double from the stored populations.  Synchronising. */
int qlbm_moments(qlbm_handle h, double *rho4, double *u, double *eps, int ptr_kind);

/* qlbm_conserved -- global averages of Eqs. GlobalDensity, GlobalVelocity
 * and GlobalTotalEnergy, reduced in double on the device (deterministic):
 *   out[0..3] = Pauli components of (1/|Lambda|) sum_x rho(x)
 *   out[4..6] = (1/|Lambda|) sum_x sum_i e_i tr W_i   (zero beyond d)
 *   out[7]    = (1/|Lambda|) sum_x sum_i |e_i|^2/2 tr W_i
 * out is host memory of 8 doubles.  Synchronising. */
int qlbm_conserved(qlbm_handle h, double *out);

/* qlbm_get_state / qlbm_set_state -- the populations at the current time in
 * the canonical layout double [b][4][N] (checkpoint and exchange format).
 * set_state resets the step counter to 0; values are rounded to the storage
 * precision.  get_state is synchronising. */
int qlbm_get_state(qlbm_handle h, double *buf, int ptr_kind);
int qlbm_set_state(qlbm_handle h, const double *buf, int ptr_kind);

/* Round trip through the canonical layout: get_state returns each value of
 * the storage precision in double; set_state rounds to the storage precision.
 * The trip get -> set is exact for QLBM_FP64, QLBM_FP64_DF and QLBM_FP16_DEV
 * (a half deviation survives the double sum with its reference weight and the
 * subtraction); for QLBM_FP32 it is exact for every spin component and every
 * trace deviation f_i - w_i of magnitude >= 2^-29, and changes a smaller
 * nonzero deviation by at most 2^-54 absolute; for QLBM_DF64 a value moves
 * by at most 2^-48 relative (a double-float pair holds 48 significant bits,
 * possibly far apart, a double 53 contiguous ones).  For a bit-exact restart
 * in every precision use the checkpoint image below. */

/* qlbm_checkpoint_bytes -- size in bytes of a checkpoint image of this
 * handle (-1 for a bad handle). */
int64_t qlbm_checkpoint_bytes(qlbm_handle h);

/* qlbm_save_checkpoint / qlbm_load_checkpoint -- checkpoint and restart
 * (Sec. 3.3: the scheme's state at time t is the populations W_i(x,t)).  The
 * image holds the populations in the storage precision, bit for bit, in
 * natural order (the AA parity is resolved on saving): b slot planes, each
 * of N four-component vectors (f, s_x, s_y, s_z) of the storage type, site
 * fastest (double-float storage: the b planes of hi parts, then the b planes
 * of lo parts; the deviation codecs store f_i - w_i).  It is valid only for
 * a handle with the same lattice,
 * dims and precision.  Stepping a handle loaded from an image taken after k
 * steps gives, after n more steps, exactly the state of k + n uninterrupted
 * steps.  buf holds qlbm_checkpoint_bytes(h) bytes on the side ptr_kind
 * says.  load resets the step counter to 0 (as set_state).  Both calls are
 * synchronising. */
int qlbm_save_checkpoint(qlbm_handle h, void *buf, int ptr_kind);
int qlbm_load_checkpoint(qlbm_handle h, const void *buf, int ptr_kind);

/* qlbm_set_magnetic_field -- adds the Vlasov commutator of an external
 * magnetic field, -i[mu sigma.B, W] (Sec. 5, Eq. sigmaB_comm), as part of
 * the collision: integrated exactly over each time step it is
 * W_i -> U W_i U*, U = exp(-i mu dt sigma.B), a rotation of every Bloch
 * vector s_i by 2 mu |B| dt about B.  This call sets one field for the
 * whole lattice; it commutes with the SU(2)-covariant collision, so it is
 * applied to the post-collision populations in the same fused kernel.
 * mu = 0 or B = 0 switches it off (and so replaces a per-site field).
 * Applies to qlbm_step (both equilibrium paths), qlbm_step_fd_output,
 * qlbm_rollout and the reverse mode.  Discards a recorded rollout. */
int qlbm_set_magnetic_field(qlbm_handle h, double mu, const double B[3]);

/* qlbm_set_magnetic_field_array -- the same term with a field that varies
 * over the lattice, -i[mu sigma.B(x), W] (Sec. 5, Eq. sigmaB_comm): every
 * post-collision Bloch vector at site x is rotated by 2 mu |B(x)| dt about
 * B(x), exactly U(x) W U(x)* with U(x) = exp(-i mu dt sigma.B(x)).  Still
 * a rotation per site, it commutes with that site's collision, so it is
 * applied in the same fused kernels.
 *   mu  magnetic moment (finite)
 *   B   double [3][N]: B_x, B_y, B_z of every site (host or device, as
 *       ptr_kind says); non-finite values are refused with
 *       QLBM_ERR_INVALID_ARG and leave the field off
 * The library keeps, per site, the unit quaternion (cos phi, sin phi
 * B/|B|), phi = mu |B(x)| dt (16 bytes in single-precision storage, 32 in
 * the 64-bit precisions), which each step reads once per site.  A field B(x, t) that changes
 * in time is given by calling this again between steps: the new field
 * applies from the next step.  Applies to qlbm_step (both equilibrium
 * paths), qlbm_step_fd_output, qlbm_rollout and the reverse mode (which
 * uses the field set when the rollout was recorded: a call discards a
 * recorded rollout).  Every storage precision (32 bytes per site for the
 * 64-bit ones).  qlbm_set_magnetic_field replaces it.
 * Synchronising. */
int qlbm_set_magnetic_field_array(qlbm_handle h, double mu, const double *B, int ptr_kind);

/* qlbm_negative_eq_count -- diagnostic of the negative-definite equilibria
 * that Sec. 3.2 (end) and Sec. 3.3 (end) allow: the discrete equilibrium
 * W_i^eq = w_i rho P_i (Eq. WeqAlgo) can have a negative eigenvalue, and
 * the scheme neither clips it nor adapts tau (nor does this library).  From
 * the current state it forms the moments (Eq. DiscrAvr) and every P_i that
 * the next collision uses and flags direction i at a site when W_i^eq has a
 * negative eigenvalue, i.e. when P_i n < |P_i| |S| (the eigenvalues of
 * w_i P_i rho are w_i P_i (n +- |S|)/2).  The decision is taken in double
 * whatever the storage precision.  Read only: the state is not changed.
 *   count  host, receives the number of flagged (site, direction) pairs
 *   mask   uint32 [N] or NULL: bit i of mask[s] set when direction i is
 *          flagged at site s (host or device as ptr_kind says)
 * Every precision.  Synchronising. */
int qlbm_negative_eq_count(qlbm_handle h, int64_t *count, uint32_t *mask, int ptr_kind);

/* ------------------------------------------------------------------------
 * Fermi-Dirac parameters of the local equilibrium (Sec. 2.2, Prop. 1).
 * ---------------------------------------------------------------------- */

/* qlbm_fd_params -- per site, the parameters of the matrix-valued Fermi-Dirac
 * distribution whose moments are the site's density matrix rho and internal
 * energy eps (Eq. DiscrAvr): the analytic eigen-decomposition of rho gives
 * the occupations n_up/dn = (tr rho +- |S|)/2 and the Bloch axis S/|S| of U;
 * (beta, mu_up, mu_dn) then solve Eqs. nFDstdOmega and energyFDstdOmega,
 *   n_s = (2 pi/beta)^(d/2) F_{d/2-1}(beta mu_s),
 *   tr(rho) eps = (d/2) beta^-1 (2 pi/beta)^(d/2) sum_s F_{d/2}(beta mu_s),
 * by Newton's method on the logarithms of the three equations in
 * (log beta, beta mu_up, beta mu_dn) from the classical limit (a site where it
 * does not settle is solved again by a per-eigenvalue Newton inversion nested
 * in a bracketed Newton iteration on log beta), in double precision whatever
 * the storage precision.
 *   beta, mu_up, mu_dn  [N] (any may be NULL);  axis [3][N] (or NULL), zero
 *   where |S| = 0 (U arbitrary).  Sites where rho is not positive definite
 *   or no beta fits (eps below the zero-temperature limit) get NaN and are
 *   counted in *nfail (if not NULL).  All arrays on one side (ptr_kind).
 * Synchronising. */
int qlbm_fd_params(qlbm_handle h, double *beta, double *mu_up, double *mu_dn, double *axis,
                   int64_t *nfail, int ptr_kind);

/* qlbm_step_fd_output -- one time step (exactly as qlbm_step(h, 1)) that also
 * writes the Fermi-Dirac parameters of the state it started from (Sec. 2.2,
 * Prop. 1; the collision conserves the moments they depend on), fused into
 * the step kernel: the same solve as qlbm_fd_params in single precision
 * (in double only where the single-precision iteration does not settle).
 * Parameters to 2e-5 relative.  The spin splitting mu_up - mu_dn carries
 * the float iteration's absolute error whatever |S|: within
 * 1e-4 |mu_up - mu_dn| + 2e-6 / beta of the double solution for QLBM_FP32
 * storage (2e-5 / beta for QLBM_FP16_DEV, whose spin components are stored
 * in half precision), tested for |S| / tr rho down to 1e-8.  Near degenerate
 * eigenvalues (|S| << tr rho), where that absolute error exceeds the
 * splitting itself, use qlbm_fd_params, which solves and returns double.
 * QLBM_FP32 and
 * QLBM_FP16_DEV storage, direct equilibrium path (QLBM_ERR_UNSUPPORTED
 * otherwise).
 *   beta, mu_up, mu_dn  float [N];  axis float [3][N] (zero where |S| = 0);
 *   all required, all on one side (ptr_kind).  Sites without a solution get
 *   NaN; their count is written to *nfail if nfail is not NULL.
 * Asynchronous for device pointers with nfail == NULL; synchronising
 * otherwise. */
int qlbm_step_fd_output(qlbm_handle h, float *beta, float *mu_up, float *mu_dn, float *axis, int64_t *nfail,
                        int ptr_kind);

/* qlbm_init_fd_params -- equilibrium initial state from physical Fermi-Dirac
 * parameters (Sec. 2.2), as the paper sets up its Riemann problem: per site
 * n_s = (2 pi/beta)^(d/2) F_{d/2-1}(beta mu_s) (Eq. nFDstdOmega), eps from
 * Eq. energyFDstdOmega, rho = U diag(n_up, n_dn) U* with Bloch axis `axis`
 * (unit vector, or zero), then W_i = W_i^eq(rho, u, eps) (Eq. WeqAlgo).
 *   beta, mu_up, mu_dn [N];  axis [3][N];  u [d][N];  one side (ptr_kind).
 * Resets the step counter. */
int qlbm_init_fd_params(qlbm_handle h, const double *beta, const double *mu_up,
                        const double *mu_dn, const double *axis, const double *u, int ptr_kind);

/* qlbm_fd_params_adjoint -- reverse mode of qlbm_fd_params at the current
 * state, by the implicit-function rule: with p = (beta, beta mu_up,
 * beta mu_dn) solving G(p; n_up, n_dn, tr(rho) eps) = 0 (the two equations
 * above), dp/d(n_up, n_dn, tr(rho) eps) = (dG/dp)^-1.  Given the cotangents
 * g_beta, g_mu_up, g_mu_dn [N] and g_axis [3][N] (any may be NULL = 0) of
 * the outputs, writes lam = dJ/dW [b][4][N] through n_up/dn = (tr rho +-
 * |S|)/2, axis = S/|S| and the moments of Eq. DiscrAvr.  Sites without a
 * solution get lam = 0.  All arrays on one side (ptr_kind).  Synchronising. */
int qlbm_fd_params_adjoint(qlbm_handle h, const double *g_beta, const double *g_mu_up,
                           const double *g_mu_dn, const double *g_axis, double *lam, int ptr_kind);

/* Equilibrium path of qlbm_step.  QLBM_EQ_DIRECT (default): W_i^eq = w_i rho
 * P_i (Eq. WeqAlgo: only rho enters, U is never formed).
 * QLBM_EQ_FD_PARAMS: W_i^eq = w_i U diag(n_up, n_dn) U* P_i (Eq. WeqDiscr)
 * with U, beta, mu_s recovered per site as in qlbm_fd_params and
 * n_s = (2 pi/beta)^(d/2) F_{d/2-1}(beta mu_s); it agrees with the direct path
 * to the accuracy of the solve, and sites without a solution keep rho.
 * QLBM_FP64 and QLBM_FP64_DF handles only (QLBM_ERR_UNSUPPORTED otherwise;
 * both step this path in double); forward stepping
 * only (qlbm_rollout returns QLBM_ERR_UNSUPPORTED on this path). */
#define QLBM_EQ_DIRECT 0
#define QLBM_EQ_FD_PARAMS 1
int qlbm_set_equilibrium_path(qlbm_handle h, int path);

/* ------------------------------------------------------------------------
 * Reverse mode.  The gradient of an observable J of the state is carried as
 * a cotangent lambda = dJ/dW in the canonical layout double [b][4][N]: for
 * each population, (dJ/df, dJ/ds_x, dJ/ds_y, dJ/ds_z) of its Pauli
 * components.  The step of Sec. 3.3 (Eqs. DiscrAvr, WeqAlgo, CollisionStep,
 * TransportStep) is differentiated exactly by the chain rule; streaming is a
 * permutation, so its adjoint pulls lambda_i(x + e_i).  dJ/dtau follows from
 * omega = dt/tau in Eq. CollisionStep.  Single-precision handles carry the
 * cotangents in float internally.  QLBM_DF64 and QLBM_FP64_DF handles have
 * no reverse mode: these calls return QLBM_ERR_UNSUPPORTED.
 * ---------------------------------------------------------------------- */

/* qlbm_step_adjoint -- one reverse step at the handle's current state W^n:
 * from lam_next = dJ/dW^{n+1} returns lam = dJ/dW^n and (if dJ_dtau is not
 * NULL) this step's contribution to dJ/dtau.  The state is not changed.
 * lam_next and lam: [b][4][N], both host or both device (ptr_kind).
 * Synchronising. */
int qlbm_step_adjoint(qlbm_handle h, const double *lam_next, double *lam, double *dJ_dtau,
                      int ptr_kind);

/* qlbm_rollout -- nsteps forward steps (as qlbm_step) that also keep, in
 * library-owned device memory, a copy of the state every `interval` steps
 * for qlbm_rollout_adjoint.  interval = 1 keeps every state (written by the
 * forward steps themselves, no extra copies; the reverse sweep recomputes
 * nothing); interval = 0 chooses: 1 when nsteps states fit in 3/4 of the
 * device memory available to the handle (and their allocation succeeds),
 * else ceil(sqrt(nsteps)), the square-root checkpointing schedule.  Memory: ceil(nsteps/interval) +
 * interval - 1 state copies; QLBM_ERR_OOM (nothing run) if they do not fit.
 * A later step, init or set_state discards the record. */
int qlbm_rollout(qlbm_handle h, int64_t nsteps, int64_t interval);

/* The checkpoint interval the last qlbm_rollout used (-1: none recorded). */
int64_t qlbm_rollout_interval(qlbm_handle h);

/* Identifier of the recorded rollout: 1 for the handle's first qlbm_rollout,
 * incremented by each later one; -1 when none is recorded (none yet, or a
 * step, init or set_state discarded it).  A caller that keeps several
 * forward passes apart (e.g. an autograd graph) compares it before calling
 * qlbm_rollout_adjoint, which always sweeps over the last rollout. */
int64_t qlbm_rollout_id(qlbm_handle h);

/* qlbm_rollout_adjoint -- reverse sweep over the last qlbm_rollout: for each
 * checkpoint segment, last first, recompute the segment's states from its
 * checkpoint (two-buffer forward steps), then apply the reverse step to them
 * in reverse order.  lam_T = dJ/dW at the end of the rollout, lam_0 =
 * dJ/dW at its start, *dJ_dtau (if not NULL) = the whole rollout's dJ/dtau.
 * The live state (the rollout's end state) is left unchanged.  Errors:
 * QLBM_ERR_STATE if no rollout is recorded.  Synchronising. */
int qlbm_rollout_adjoint(qlbm_handle h, const double *lam_T, double *lam_0, double *dJ_dtau,
                         int ptr_kind);

/* qlbm_init_equilibrium_adjoint -- gradients through the initial state of
 * qlbm_init_equilibrium (W_i = w_i P_i(u, eps) rho, Eq. WeqAlgo with u and
 * eps given): from lam0 = dJ/dW^0 and the same (rho4, u, eps) (eps may be
 * NULL = eps0), writes g_rho4 = dJ/drho4 [4][N], g_u = dJ/du [d][N] and
 * g_eps = dJ/deps [N] (any output may be NULL).  All arrays on the same side
 * (ptr_kind).  Synchronising. */
int qlbm_init_equilibrium_adjoint(qlbm_handle h, const double *rho4, const double *u,
                                  const double *eps, const double *lam0, double *g_rho4,
                                  double *g_u, double *g_eps, int ptr_kind);

/* qlbm_conserved_static -- the same eight averages as qlbm_conserved, for a
 * caller-owned state, without allocating any device memory.  The paper has
 * no counterpart: this entry point exists for callers that cannot allocate
 * at the point of the call -- code running under another component's memory
 * manager (a framework's caching allocator or a fixed arena that owns the
 * device's memory) and latency-critical loops that cannot afford
 * cudaMalloc/cudaFree, which may synchronise the whole device.
 *   lattice  QLBM_D2Q9 or QLBM_D3Q19
 *   dims     {nx, ny, nz} (nz = 1 for D2Q9); at most QLBM_STATIC_MAX_SITES
 *            sites in total, else QLBM_ERR_INVALID_ARG
 *   beta0    reference inverse temperature (fixes xi for the momentum and
 *            energy scaling)
 *   state    device, canonical layout double [b][4][N] (as qlbm_get_state
 *            writes it), read only
 *   out      device, 8 doubles, written: out[0..3] density matrix (Pauli),
 *            out[4..6] momentum, out[7] total energy, lattice averages
 *   stream   cudaStream_t or NULL; the call is asynchronous on it
 * Scratch: the partial sums live in one file-scope __device__ array of
 * QLBM_STATIC_SCRATCH_BLOCKS x 8 doubles (64 KiB) that every GPU loading the
 * library holds until the process exits.  All calls on a device share it and
 * it keeps the last call's contents (each call overwrites every row it
 * reads, so nothing needs clearing); calls whose kernels overlap on the GPU
 * (different streams, or different host threads) race on it and must be
 * serialised by the caller.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  The address is kept for
 * the life of the process: destroying the device's primary context between
 * calls (cudaDeviceReset) is not supported.  No cudaMalloc, cudaFree
 * or allocating library routine is called.  Errors: QLBM_ERR_INVALID_ARG,
 * QLBM_ERR_CUDA; message via qlbm_last_error(NULL). */
#define QLBM_STATIC_SCRATCH_BLOCKS 1024
#define QLBM_STATIC_MAX_SITES 2147483647LL
int qlbm_conserved_static(int lattice, const int64_t dims[3], double beta0, const double *state,
                          double *out, void *stream);

/* ------------------------------------------------------------------------
 * Synthetic input fields.
 * ---------------------------------------------------------------------- */

/* qlbm_fourier_field -- a real Fourier sum at every site of a periodic box,
 * evaluated on the device in double precision:
 *   out[s] = offset + scale * sum_m (A_m cos(phi_m) + B_m sin(phi_m)),
 *   phi_m = 2 pi (k_m[0] x / nx + k_m[1] y / ny + k_m[2] z / nz),
 *   s = x + nx*(y + ny*z).
 * The paper's method has no counterpart: this generates the smooth, seeded
 * density / velocity / spin perturbations of the synthetic workloads (the
 * shape of the smooth initial data of Sec. 4's tests) directly in device
 * memory, so that a 512^3 field needs neither host memory nor a host FFT.
 * The coefficients are inputs: nothing random is drawn here.
 *   dims    {nx, ny, nz}, each in [1, 2^30] (nz = 1 for a 2D box)
 *   nmodes  number of modes, 0 .. QLBM_FOURIER_MAX_MODES
 *   k       host, int32 [nmodes][3] integer wave vectors, each component in
 *           [-QLBM_FOURIER_MAX_K, QLBM_FOURIER_MAX_K]
 *   A, B    host, double [nmodes] cosine and sine coefficients
 *   out     device, double [nx*ny*nz], written
 *   stream  cudaStream_t or NULL; the call is asynchronous on it and
 *           allocates no memory (the modes travel as a kernel argument)
 * Deterministic: the result does not depend on the launch.  Errors:
 * QLBM_ERR_INVALID_ARG, QLBM_ERR_CUDA; message via qlbm_last_error(NULL). */
#define QLBM_FOURIER_MAX_MODES 512
#define QLBM_FOURIER_MAX_K 64
int qlbm_fourier_field(const int64_t dims[3], int nmodes, const int32_t *k, const double *A, const double *B,
                       double scale, double offset, double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* QLBM_H */
