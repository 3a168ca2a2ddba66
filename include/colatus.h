/*
 * colatus.h -- C ABI of the B300 (sm_103a) library for the hot path of
 * COLATUS (Stalder et al., "A new gravitational N-body simulation algorithm
 * for investigation of cosmological chaotic advection", arXiv 1208.3444).
 *
 * What the library computes
 *   The softened all-pairs gravitational acceleration in comoving coordinates
 *   (Eq. 1), oriented attractively,
 *       acc_k = a^-3 G sum_{j != k} m_j (x_j - x_k) / (|x_j - x_k|^2 + eps^2)^{3/2},
 *   with isolated boundaries, integrated by the Hubble-drag leapfrog of
 *   Eqs. 3-5 (drift-kick-drift, "DKD") or its kick-drift-kick form ("KDK"),
 *   with the scale factor a(t) driven by the Friedmann equation (Eq. 2),
 *       da/dt = a H(a),  H = H0 sqrt(Omega_R a^-4 + Omega_M a^-3 + Omega_K a^-2 + Omega_L).
 *   The paper's Appendix A kernel (one GPU thread per body, forces then
 *   integration) is the operation; its design is not reused.
 *
 * Conventions shared by every entry point
 *   - Every function returns a colatus_status and never aborts the process.
 *     colatus_last_error() describes the most recent failure of a context.
 *   - Array arguments are plain pointers.  `on_device` = 0 means a host
 *     pointer, 1 means a device pointer on the context's device.  `dtype`
 *     selects float (COLATUS_F32) or double (COLATUS_F64) elements.
 *   - Vector arrays are N x 3, row-major (x0 y0 z0 x1 ...).
 *   - The caller owns every pointer it passes; the library copies what it
 *     needs before returning (or, for asynchronous device-to-device calls,
 *     before the work it enqueued on the context's stream completes).
 *   - A context is bound to one device and one CUDA stream.  Calls on one
 *     context are not thread-safe.  All GPU work is enqueued on the context's
 *     stream; functions that return host data synchronise that stream.
 *   - Time t is absolute code time with t = 0 at a_start; G defaults to 1.
 */
#ifndef COLATUS_H
#define COLATUS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque context, owned by the library (create with colatus_init). */
typedef struct colatus_ctx *colatus_t;

typedef enum {
    COLATUS_OK = 0,
    COLATUS_E_ARG = 1,        /* invalid argument (sizes, pointers, eps <= 0, ...)   */
    COLATUS_E_CUDA = 2,       /* a CUDA runtime call failed                           */
    COLATUS_E_NONFINITE = 3,  /* a position or velocity became NaN or Inf             */
    COLATUS_E_FRIEDMANN = 4,  /* H^2 < 0 in Eq. 2 (e.g. recollapse), or a <= 0        */
    COLATUS_E_STATE = 5,      /* call out of order (e.g. step before set_state)       */
    COLATUS_E_OOM = 6,        /* device allocation failed                             */
    COLATUS_E_TIMEOUT = 7     /* a bounded device-side wait gave up (no hang)         */
} colatus_status;

typedef enum {
    COLATUS_FP32 = 0,       /* FP32 pair arithmetic, blocked FP32 accumulation         */
    COLATUS_FP32_COMP = 1,  /* FP32 pair arithmetic (the same bare SFU rsqrt.approx as
                               COLATUS_FP32); the j-sum is accumulated in FP32 blocks of
                               32 to 256 j-bodies (by tile shape), each block folded into
                               a two-float (TwoSum) hi/lo total; only
                               colatus_diagnostics refines its rsqrt                   */
    COLATUS_FP64 = 2        /* FP64 everywhere (state, pair arithmetic, sums)          */
} colatus_prec;

typedef enum {
    COLATUS_DKD = 0,  /* Eqs. 3-5: half drift, kick at t^{n+1/2}, half drift             */
    COLATUS_KDK = 1,  /* half kick at t^n, drift, half kick at t^{n+1} (span tau/2 each) */
    COLATUS_KDK_CANONICAL = 2  /* the symplectic canonical leapfrog of Sec. II: p = a^2 v,
                                  kick p += G F int dt/a over each half step, drift
                                  x += p int dt/a^2 over the step (FP64 RK4 quadrature
                                  along a(t)); takes KDK's place everywhere KDK is accepted */
} colatus_scheme;

typedef enum { COLATUS_F32 = 0, COLATUS_F64 = 1 } colatus_dtype;

/* Number of doubles written by colatus_diagnostics. */
#define COLATUS_NDIAG 16

/* Create a context for N bodies on the current CUDA device.
 *   masses:  host array of N doubles (copied; may be changed later with
 *            colatus_set_masses).
 *   eps:     Plummer softening of Eq. 1 (the kernel's min_dist); must be > 0.
 *   Omega_*, H0: Eq. 2 parameters; a_start > 0 is the scale factor at t = 0.
 * Defaults: COLATUS_FP32, COLATUS_KDK, G = 1, a library-owned stream.
 * Errors: COLATUS_E_ARG (N < 1, eps <= 0 or not finite, a_start <= 0, NULL
 * pointers, H^2(a_start) < 0), COLATUS_E_OOM, COLATUS_E_CUDA.  On error *out
 * is set to NULL and nothing is leaked.
 * Checkpoint and resume: after any colatus_step, colatus_get_state gives
 * (x, v, t, a).  A new context created with a_start = a and the same masses,
 * eps, Omega_*, H0, precision, scheme and G, given x and v with
 * colatus_set_state, continues the run bit for bit with the same step size
 * (its time restarts at 0, so add t). */
colatus_status colatus_init(colatus_t *out, int64_t N, const double *masses, double eps,
                            double Omega_R, double Omega_M, double Omega_K, double Omega_L,
                            double H0, double a_start);

/* Precision, integrator, gravitational constant and stream (a cudaStream_t;
 * NULL keeps the library-owned stream).  The integrators: the paper's DKD
 * leapfrog (Eqs. 3-5), KDK with the same drag coefficients, and the
 * symplectic KDK of the canonical variables (Sec. II); G is the constant of
 * Eq. 1.  Changing precision keeps the state (converted).  Errors:
 * COLATUS_E_ARG. */
colatus_status colatus_set_config(colatus_t ctx, colatus_prec prec, colatus_scheme scheme,
                                  double G, void *cuda_stream);

/* Deformation potential of Eq. 6: adds to every body's pull
 *     C psi (x_psi - x_k) / (|x_k - x_psi|^2 + eps^2)^{3/2}
 * inside the a^-3-scaled force (the pull of a point "mass" C psi / G fixed at
 * x_psi, host double[3]).  C psi = 0 switches it off.  It enters the forces,
 * the steps, the adjoint and the tangent model (not the ensemble).  Needs
 * G != 0 (COLATUS_E_ARG otherwise). */
colatus_status colatus_set_deformation(colatus_t ctx, double Cpsi, const double *x_psi);

/* Periodic boundaries (Sec. II) in a cube of side L: every body pulls with
 * all its images, the uniform mean density is removed (a homogeneous box
 * feels no force), and the nearest image is Plummer-softened with eps:
 *   F_k = sum_j m_j [ sum_n N(d_j + n L) - N(d_j) + P(d_j) ],
 *   d_j = minimum image of x_j - x_k, N(d) = d/|d|^3, P(d) = d/(|d|^2+eps^2)^1.5,
 * evaluated by Ewald summation: a real-space all-pairs kernel over minimum
 * images and a reciprocal-space sum over 0 < |n| <= nk, k = 2 pi n / L.
 * alpha <= 0 and nk <= 0 choose them from the precision (truncation below
 * 1e-8 of a pair term in the FP32 modes, 1e-15 in FP64); nk <= 63.  Positions
 * are not wrapped: the minimum image is taken per pair.  L = 0 restores
 * isolated boundaries.  Forces, both step schemes, the force VJP, the
 * adjoint and the tangent model honour it (their derivatives differentiate
 * the Ewald sum: the real-space pair Jacobian over minimum images plus the
 * reciprocal sum's); autotuning returns COLATUS_E_STATE while it is on, and
 * it does not combine with the deformation term (COLATUS_E_ARG).
 * colatus_diagnostics keeps the isolated potential. */
colatus_status colatus_set_periodic(colatus_t ctx, double L, double alpha, int nk);

/* The Ewald parameters in use: alpha, nk and the number of k-vectors of the
 * half space (any pointer may be NULL).  COLATUS_E_STATE if not periodic. */
colatus_status colatus_periodic_params(colatus_t ctx, double *alpha_out, int *nk_out, int *nkv_out);

/* Replace the N masses (dtype elements, host or device). */
colatus_status colatus_set_masses(colatus_t ctx, const void *m, int dtype, int on_device);

/* Set positions x and velocities v (N x 3 each, dtype elements, host or
 * device) at the current (t, a).  This is the host-to-device copy of the
 * initial conditions in the paper's Appendix A host program (read the data
 * file, copy the bodies to the GPU); here it may also restore a saved state.  v may be NULL for bodies at rest.  The
 * FP32 modes store float state: double input is rounded to float.
 * Errors: COLATUS_E_ARG, COLATUS_E_NONFINITE (a non-finite input value). */
colatus_status colatus_set_state(colatus_t ctx, const void *x, const void *v, int dtype,
                                 int on_device);

/* Read positions and velocities (N x 3, dtype) and the current t and a
 * (either may be NULL).  This is the paper's Appendix A device-to-host copy
 * of every position and velocity, which the paper makes after every step and
 * which here is made on request.  Synchronises the stream and reports any device
 * error flag raised since the last check (COLATUS_E_NONFINITE,
 * COLATUS_E_FRIEDMANN, COLATUS_E_TIMEOUT). */
colatus_status colatus_get_state(colatus_t ctx, void *x, void *v, int dtype, int on_device,
                                 double *t, double *a);

/* Asynchronous read-back of positions and velocities (N x 3, dtype) into
 * HOST memory: the state after the steps enqueued so far is snapshotted on
 * the device (in order on the context's stream) and copied to x and v on a
 * separate copy stream, so the copy overlaps the steps enqueued after it
 * (pinned host memory is needed for the overlap).  Returns without waiting,
 * except when four earlier read-backs are still copying (four slots).  x and v
 * must stay valid and untouched until colatus_wait_state,
 * colatus_synchronize or colatus_get_state returns.  Either may be NULL, not
 * both.  The first call on a context creates the copy stream and the four
 * device slots (N x 3 doubles each for x and v); its cudaMalloc calls
 * synchronise the device once.  Errors: COLATUS_E_ARG, COLATUS_E_STATE (no
 * state), COLATUS_E_CUDA. */
colatus_status colatus_get_state_async(colatus_t ctx, void *x, void *v, int dtype);

/* Wait for every read-back started by colatus_get_state_async and for the
 * context's stream; reports device error flags as colatus_synchronize does. */
colatus_status colatus_wait_state(colatus_t ctx);

/* Comoving acceleration of Eq. 1 at the current state and scale factor:
 * acc_out (N x 3, dtype) = a^-3 G sum_{j != k} m_j (x_j - x_k) / s^3.
 * Device output is asynchronous on the context's stream; host output
 * synchronises.  Errors: COLATUS_E_STATE (no state set), COLATUS_E_TIMEOUT. */
colatus_status colatus_forces(colatus_t ctx, void *acc_out, int dtype, int on_device);

/* Advance nsteps steps of size dt (> 0) with the configured scheme (Eqs.
 * 3-5: drift, the Eq. 1 force, the kick with Hubble drag).  The scale factor
 * of Eq. 2 is advanced on the GPU in FP64 (RK4, 8 sub-steps per half
 * step).  Asynchronous: device error flags are reported by the next
 * colatus_synchronize / colatus_get_state.  Errors: COLATUS_E_ARG,
 * COLATUS_E_STATE. */
colatus_status colatus_step(colatus_t ctx, double dt, int64_t nsteps);

/* Wait for all enqueued work and report device error flags. */
colatus_status colatus_synchronize(colatus_t ctx);

/* Tracers: the paper follows the velocity of single bodies at every step
 * (Sec. I; Appendix A copies every body's state back after each step).
 * Record (x, v) of ntr bodies idx[0..ntr) (host int64 indices, distinct,
 * in [0, N)) after every subsequent step, into a device ring buffer of
 * capacity_steps records (the oldest are overwritten).  ntr = 0 stops
 * recording.  Replaces any earlier recording. */
colatus_status colatus_record_tracers(colatus_t ctx, const int64_t *idx, int ntr,
                                      int64_t capacity_steps);

/* The single-body records of Sec. I, read back (the part of Appendix A's
 * per-step device-to-host copy that the tracer study needs).
 * Copy the recorded tracers, oldest first, to host memory xv_out laid out
 * [nrec][ntr][6] floats (x, y, z, vx, vy, vz); *nrec_out = records copied
 * (<= capacity).  xv_out may be NULL to query *nrec_out.  Synchronises. */
colatus_status colatus_read_tracers(colatus_t ctx, float *xv_out, int64_t *nrec_out);

/* FP64 diagnostics at the current state (synchronises).  Their definitions
 * come from the Hamiltonian of Sec. II (canonical momentum p = m a^2 v):
 *   out[0] K = (1/2) sum m a^2 |v|^2      out[1] W = W_x / a
 *   out[2..4] P = sum m a^2 v             out[5..7] L = sum m a^2 x cross v
 *   out[8..10] centre of mass             out[11] a   out[12] t   out[13] H(a)
 *   out[14] W_x = -(G/2) sum_{j != k} m_k m_j / s_kj   out[15] step count
 * (K + W obeys the Layzer-Irvine equation d(K+W)/dt = -H (2K + W)).
 * The first call allocates the context's scratch
 * for the per-split potential sums, at most 64 MB.  Errors: COLATUS_E_STATE
 * (no state set), COLATUS_E_CUDA (the allocation or a launch failed). */
colatus_status colatus_diagnostics(colatus_t ctx, double out[COLATUS_NDIAG]);

/* ---- Tracer velocity energy spectrum (Sec. I, Sec. IV: the velocity of
 * single bodies at every step and its energy power spectrum).
 *
 * For T samples per tracer at uniform spacing dt, u = v - mean(v) when
 * detrend != 0 (else u = v), w_n = 1 (window 0) or the periodic Hann window
 * (1 - cos(2 pi n / T)) / 2 (window 1), U = (1/T) sum_n w_n^2:
 *     E_k(f_j) = c_j dt / (T U) * 1/2 sum_c |sum_n w_n u_{n,k,c} e^{-2 pi i j n/T}|^2
 * for j = 0 .. T/2 (integer division), f_j = j / (T dt); c_j = 2 except
 * c_0 = 1 and c_{T/2} = 1 for even T.  Then sum_j E_k(f_j) / (T dt) is the
 * window-weighted mean of |u|^2 / 2 (Parseval).  Computed on the GPU in FP64
 * by a direct DFT with exactly reduced angles.  Output E is [ntr][T/2 + 1]
 * doubles, row-major.  Needs 2 <= T <= 2^24. */

/* Energy spectrum (Sec. I, Sec. IV) of a velocity series v laid out [T][ntr][stride] (dtype
 * elements; the three velocity components are the first three of each
 * stride).  on_device / out_on_device say where v and E_out live.  Runs on
 * cuda_stream (NULL: the legacy default stream) and synchronises it unless both
 * v and E_out are device memory.  Errors: colatus_last_error(NULL). */
colatus_status colatus_velocity_spectrum(const void *v, int dtype, int on_device, int64_t T,
                                         int64_t ntr, int64_t stride, double dt, int window,
                                         int detrend, double *E_out, int out_on_device,
                                         void *cuda_stream);

/* Energy spectrum (Sec. I, Sec. IV) of the velocities recorded by colatus_record_tracers (the kept
 * records, oldest first, read in place on the device); dt is the step size
 * the records were taken with.  *nrec_out = T used; E_out (host) may be NULL
 * to query it.  COLATUS_E_STATE if nothing is recorded.  Synchronises. */
colatus_status colatus_tracer_spectrum(colatus_t ctx, double dt, int window, int detrend,
                                       double *E_out, int64_t *nrec_out);

/* Self-test of the device-side failure path: one CTA waits on a barrier
 * that nothing completes, gives up after limit_cycles SM cycles (1 ..
 * 2e9; the pipelined kernels use 2e9, about a second) and raises the same
 * timeout flag the force, VJP and JVP kernels raise when a bulk-copy wait
 * gives up.  Returns COLATUS_E_TIMEOUT when the path works (the flag is
 * cleared; the context stays usable), COLATUS_E_ARG for a bad limit. */
colatus_status colatus_selftest_wait(colatus_t ctx, int64_t limit_cycles);

/* Host-only self-test of the scheduling tables of the kernels that evaluate
 * each pair once (Eq. 1 summed over unordered pairs, Newton's third law):
 * builds the tables a context builds for n_pad bodies in tiles of T (the
 * tile pairs it <= jt, NW phases each, split over G CTAs by the costs
 * cost_diag : cost_sym of a diagonal and a symmetric phase), then replays
 * every CTA's walk over them as the kernels take it.  It checks that every
 * phase of every tile pair is taken exactly once, that every row segment and
 * column slot is written exactly once and lies in bounds, and that each
 * tile's column run holds exactly the slots of its tile pairs (t', t),
 * t' < t, in order.  Needs no GPU.  T/2 a multiple of 32 NW, n_pad a
 * multiple of T with at most 2048 tiles, G >= 1.  out (may be NULL): [0]
 * tiles, [1] tile pairs, [2] CTAs, [3] most row segments of a tile, [4]
 * column slots.  COLATUS_OK if all hold, COLATUS_E_STATE with the first
 * failure in colatus_last_error(NULL), COLATUS_E_ARG for bad arguments. */
colatus_status colatus_selftest_sym_tables(int64_t n_pad, int T, int NW, int G, int cost_diag, int cost_sym,
                                           int64_t out[5]);

/* The same for the ensemble's tables (colatus_ensemble_init, tile shape 3):
 * R realisations of n_bodies[r] bodies (host array; 1 .. 2^26 each), stored
 * padded to 256 and cut into 512-body tiles (at most 2048 in all).  out as
 * above, [0] the tiles of all realisations. */
colatus_status colatus_selftest_ens_sym_tables(int R, const int64_t *n_bodies, int G, int cost_diag,
                                               int cost_sym, int64_t out[5]);

/* Human-readable description of the last error on ctx ("" if none);
 * colatus_last_error(NULL) describes the last colatus_init failure. */
const char *colatus_last_error(colatus_t ctx);

/* Counters of a context: out[0] kernel launches enqueued, out[1] pair
 * interactions enqueued (N^2 per force evaluation), out[2] steps taken,
 * out[3] N. */
colatus_status colatus_stats(colatus_t ctx, double out[4]);

/* The force kernel that colatus_forces and colatus_step launch for the
 * current precision, masses, boundaries and tuning, for measurement (the
 * Eq. 1 sum of the paper's Appendix A kernel; this names its launch shape):
 * out[0] kind (0 FP32 all-pairs, 1 FP64 all-pairs, 2 FP32 periodic real
 * space, 3 FP64 periodic real space, 4 FP32 all-pairs with every pair
 * evaluated once, 5 FP32 periodic real space with every pair evaluated
 * once), out[1] threads per CTA, out[2] i-bodies per thread,
 * out[3] j-tile bodies, out[4] compensated accumulation (0/1), out[5]
 * equal-mass form (0/1), out[6] persistent grid (CTAs), out[7] work units
 * (i-tile x j-tile; for kinds 4 and 5 the tile pairs it <= jt), out[8] i-bodies per
 * thread whose 1/s^2 is an rcp on the MUFU pipe rather than a square of the
 * rsqrt on the FMA pipe.  Errors: COLATUS_E_ARG. */
colatus_status colatus_force_plan(colatus_t ctx, int64_t out[9]);

/* The VJP kernel that colatus_adjoint_backward launches for the current
 * precision, masses, boundaries, deformation term and scheme, for
 * measurement (the VJP of the Eq. 1 sum, see colatus_force_vjp; the
 * equal-mass forms need equal masses, isolated boundaries, no Eq. 6 term, a
 * KDK scheme and N a multiple of 1024; colatus_force_vjp itself always takes
 * a form for any masses): out[0] kind (0 FP32 general, 1 FP64, 2 FP32 periodic
 * real space, 3 FP64 periodic real space, 4 FP32 equal-mass, 5 FP32
 * equal-mass with every pair evaluated once, from 8 tiles of 1024 bodies,
 * 6 FP32 any masses with every pair evaluated once, from 8 tiles: also the
 * kernel of colatus_force_vjp then, 7 FP32 periodic real space with every
 * pair evaluated once, from 8 tiles of 1024 bodies under tuning shape 3 or
 * the built-in choice, as the periodic force),
 * out[1] threads per CTA, out[2] i-bodies per thread, out[3] j-tile bodies,
 * out[4] persistent grid (CTAs), out[5] work units (i-tile x j-tile; for
 * kinds 5 to 7 the tile pairs it <= jt).  Errors: COLATUS_E_ARG. */
colatus_status colatus_vjp_plan(colatus_t ctx, int64_t out[6]);

/* Kernel timing for measurement: with on != 0 every launch of the force
 * kernel, the VJP kernel and the adjoint's per-step update kernel is
 * bracketed by a pair of CUDA events recorded on the context's stream
 * (on = 0 stops and discards them). */
colatus_status colatus_profile_forces(colatus_t ctx, int on);

/* Durations since the last read, from the event pairs of
 * colatus_profile_forces: out[0] total milliseconds and out[1] number of
 * force-kernel launches, out[2] milliseconds and out[3] number of VJP-kernel
 * launches.  Synchronises the stream and resets the totals. */
colatus_status colatus_profile_read(colatus_t ctx, double out[4]);

/* The same with a third kind: out[0..3] as colatus_profile_read, out[4]
 * milliseconds and out[5] number of launches of the discrete adjoint's
 * per-step update kernel (the transposed kick-drift-kick update that follows
 * each VJP in colatus_adjoint_backward).  Synchronises the stream and resets
 * the totals. */
colatus_status colatus_profile_read_kinds(colatus_t ctx, double out[6]);

/* Force-kernel tuning.  The FP32 force kernel exists in four tile shapes
 * (threads x i-bodies per thread, j-tile): 0 = 512 x 4, 512 bodies (one CTA
 * per SM); 1 = 256 x 4, 512 (two CTAs per SM); 2 = 128 x 2, 64 (small N);
 * 3 = 512 x 4 on 2048-body tiles with every pair evaluated once and applied
 * to both bodies (Newton's third law: the same sum with about two thirds of
 * the arithmetic).  Shape 3 fits from 2 tiles (N > 2048) while its partial
 * sums, about N^2 / 2048 x 8 bytes (x 2 compensated), take at most an eighth
 * of the device's memory (on a 288 GB B300: 17 GB at N = 2^21 in FP32, 34 GB
 * compensated); it is the built-in choice from 8 tiles (N > 14336) on, and
 * shape 0 the choice that needs no such buffer.  colatus_autotune times reps launches of every shape that fits N on
 * the current state (for the context's FP32 precision and mass type), keeps
 * the fastest for this context and returns it in *chosen; out_ms[4] (may be
 * NULL) receives the mean milliseconds per launch (0 for shapes that do not
 * fit).  colatus_set_tuning applies a known choice (-1: built-in choice);
 * COLATUS_E_ARG for a shape that does not fit.  Under periodic boundaries
 * the real-space kernel comes in two forms: every pair once (1024-body
 * tiles, from 8 tiles on; the built-in choice and shape 3) and every ordered
 * pair (any other shape); colatus_autotune refuses periodic contexts. */
colatus_status colatus_autotune(colatus_t ctx, int reps, double out_ms[4], int *chosen);
colatus_status colatus_set_tuning(colatus_t ctx, int shape);

/* Vector-Jacobian product of the Eq. 1 acceleration at the current state:
 * for a co-vector w (N x 3), gx = d(sum_k w_k . acc_k)/dx (N x 3) and
 * gm = d(sum_k w_k . acc_k)/dm (N), with acc = G a^-3 F as in colatus_forces:
 *     gx_i = G a^-3 sum_{j != i} J(d_ij) (m_i w_j - m_j w_i),
 *     gm_i = -G a^-3 sum_{j != i} (w_j . d_ij) / s_ij^3,
 * J(d) = I/s^3 - 3 d d^T/s^5 (the derivative of the Eq. 1 pair term).
 * Either output may be NULL.  Same dtype / on_device conventions as
 * colatus_forces (the precision is the context's). */
colatus_status colatus_force_vjp(colatus_t ctx, const void *w, void *gx, void *gm, int dtype,
                                 int on_device);

/* Forward pass of the discrete adjoint (the transpose of the steps of
 * Eqs. 3-5 with the Eq. 1 force), for any of the three schemes:
 * advances the state by nsteps steps of size dt exactly as colatus_step
 * does, keeping a checkpoint of (x, v) every checkpoint_every steps (device
 * memory: nsteps / checkpoint_every checkpoints of N bodies, plus
 * checkpoint_every positions for recomputation, and as many velocities for
 * DKD).  Errors: COLATUS_E_ARG (sizes), COLATUS_E_STATE (no state). */
colatus_status colatus_adjoint_forward(colatus_t ctx, double dt, int64_t nsteps,
                                       int64_t checkpoint_every);

/* Backward pass: given the gradient of a loss with respect to the final
 * positions, velocities and masses (gx_T, gv_T: N x 3; gm_T: N; any may be
 * NULL for zero), return its gradient with respect to the positions and
 * velocities at the start of the forward pass and the masses (gx_0, gv_0:
 * N x 3, gm: N; any may be NULL).  It is the exact transpose of the FP32 (or
 * FP64) leapfrog that was run: each segment between checkpoints is
 * recomputed with the forward's own kernels, then swept backwards with one
 * VJP (colatus_force_vjp's kernel) per step, at x_{n+1} for KDK and at the
 * half-drift position x_n + (dt/2) v_n for DKD (Eqs. 3-5), plus one at x_0
 * for KDK.  The state (the forward's end) is left as it was.  Errors:
 * COLATUS_E_STATE (no forward pass, or the state was stepped, or the
 * precision, scheme or G changed since). */
colatus_status colatus_adjoint_backward(colatus_t ctx, const void *gx_T, const void *gv_T,
                                        const void *gm_T, void *gx_0, void *gv_0, void *gm,
                                        int dtype, int on_device);

/* Allocation-free FP32 force, for callers that cannot call cudaMalloc (code
 * running inside another framework's memory pool or under a fixed
 * device-memory budget, or latency-bound loops that must not pay cudaMalloc's
 * implicit device synchronisation).  The paper has no counterpart; it is the
 * colatus_forces computation without a context:
 *   acc_out[3k..3k+2] = G a^-3 sum_{j != k} m_j (x_j - x_k) / (|x_j - x_k|^2 + eps^2)^{3/2}
 *   pos:     device array of N float4 (x, y, z, m), 16-byte aligned.
 *   acc_out: device array of N x 3 floats.
 *   N:       1 <= N <= 32768 on any device; eps > 0, a > 0, G finite.
 *   cuda_stream: the cudaStream_t to run on (NULL: the legacy default stream).
 * pos, acc_out and the stream must belong to the current device, and pos must
 * be 16-byte aligned; otherwise, and for sizes or parameters out of range, the
 * call returns COLATUS_E_ARG before it launches anything.
 * It allocates nothing: its scratch (packed bodies, force segments, error
 * flags) is one fixed static device array of about 8.6 MiB, which a GPU holds
 * from the first use of the library's kernels on it until the process exits.
 * The first call on a device also resolves that array's device address
 * (cudaGetSymbolAddress).  The call copies the error flags to the host and
 * synchronises `cuda_stream` before it returns, so it cannot be called while
 * that stream is being captured into a CUDA graph (COLATUS_E_STATE).  Every
 * call shares the scratch, so calls whose GPU work overlaps (different streams
 * or threads) race: serialise them.  A device-side wait that gave up is
 * reported as COLATUS_E_TIMEOUT. */
colatus_status colatus_forces_noalloc(const float *pos, int64_t N, double eps, double G, double a,
                                      float *acc_out, void *cuda_stream);

/* ------------------------------------------------------------ ensembles
 * Many independent realisations of the same system of equations (Eqs. 1-5,
 * KDK, FP32 compensated-free plain accumulation, FP64 a(t) shared by all, one
 * softening per realisation), stepped together: each step is one persistent
 * force launch over every realisation's interactions plus one fused
 * kick/drift launch, and colatus_ensemble_step replays a captured CUDA graph
 * of 16 steps at a time.  Arrays are dense concatenations: realisation r's
 * N_r bodies follow those of realisations 0..r-1 (N_tot = sum N_r rows). */
typedef struct colatus_ensemble *colatus_ens_t;

/* R realisations with N_r[r] bodies (host array), masses (host, N_tot
 * doubles), softenings eps_r (host, R doubles, > 0), the Eq. 2 parameters,
 * a_start, G and a cudaStream_t (NULL: a library-owned stream). */
colatus_status colatus_ensemble_init(colatus_ens_t *out, int R, const int64_t *N_r,
                                     const double *masses, const double *eps_r, double Omega_R,
                                     double Omega_M, double Omega_K, double Omega_L, double H0,
                                     double a_start, double G, void *cuda_stream);
/* Positions and velocities, N_tot x 3 (dtype, host or device; v may be NULL). */
colatus_status colatus_ensemble_set_state(colatus_ens_t e, const void *x, const void *v, int dtype,
                                          int on_device);
colatus_status colatus_ensemble_get_state(colatus_ens_t e, void *x, void *v, int dtype,
                                          int on_device, double *t, double *a);
/* Comoving accelerations G a^-3 F of every body (Eq. 1 within each
 * realisation; N_tot x 3). */
colatus_status colatus_ensemble_forces(colatus_ens_t e, void *acc_out, int dtype, int on_device);
/* nsteps steps of size dt > 0 (Eqs. 3-5, the scale factor of Eq. 2) for
 * every realisation (asynchronous), of the scheme set by
 * colatus_ensemble_set_scheme (KDK by default). */
colatus_status colatus_ensemble_step(colatus_ens_t e, double dt, int64_t nsteps);
/* Integration scheme of the ensemble's steps, as colatus_set_config's for
 * one system: COLATUS_DKD (Eqs. 3-5, the force at the half-drift
 * positions), COLATUS_KDK or COLATUS_KDK_CANONICAL (Sec. II).  A change
 * synchronises, drops the captured step graphs and re-opens the next step
 * from the state.  Errors: COLATUS_E_ARG. */
colatus_status colatus_ensemble_set_scheme(colatus_ens_t e, colatus_scheme scheme);
colatus_status colatus_ensemble_synchronize(colatus_ens_t e);
/* Tracers of the ensemble (Sec. I: the velocities of single bodies at every
 * step), as colatus_record_tracers for one system: record (x, v) of ntr
 * bodies idx[0..ntr) (host int64 indices into the dense N_tot rows,
 * distinct) after every subsequent step, graph replays included, into a
 * device ring of capacity_steps records; ntr = 0 stops recording.  Replaces
 * any earlier recording and drops the captured step graphs (recaptured at
 * the next step).  Synchronises.  Errors: COLATUS_E_ARG. */
colatus_status colatus_ensemble_record_tracers(colatus_ens_t e, const int64_t *idx, int ntr,
                                               int64_t capacity_steps);
/* The recorded tracers, oldest first, to host xv_out [nrec][ntr][6] floats
 * (x, y, z, vx, vy, vz); *nrec_out = records copied (<= capacity); xv_out
 * may be NULL to query *nrec_out.  Synchronises and reports device flags. */
colatus_status colatus_ensemble_read_tracers(colatus_ens_t e, float *xv_out, int64_t *nrec_out);
/* Synchronises; out[0] kernel launches (a 16-step graph counts its 33),
 * out[1] interactions enqueued, out[2] steps, out[3] interactions per step,
 * out[4]/out[5] milliseconds/number of force launches timed outside graphs
 * since the last call; profile_on switches that timing on or off. */
colatus_status colatus_ensemble_stats(colatus_ens_t e, int profile_on, double out[6]);
/* Ensemble force-kernel tuning.  The kernel exists in four CTA shapes: three
 * with the same 256-body tiles (0: 128 threads x 2 bodies, 4 CTAs per SM;
 * 1: 256 x 1, 4 per SM; 2: 64 x 4, 8 per SM) and 3: 128 x 4 on 512-body
 * tiles of each realisation with every pair evaluated once and applied to
 * both bodies (Newton's third law), usable while its partial sums take at
 * most an eighth of the device memory; shape 3 is the built-in choice where
 * it is usable, else shape 2.
 * colatus_ensemble_autotune times reps force evaluations of every usable
 * shape at the current state (state required; one untimed launch first),
 * writes the milliseconds per evaluation to out_ms[k] (0 for a shape that is
 * not usable; out_ms may be NULL), keeps the fastest and returns its index
 * in *chosen (may be NULL).  colatus_ensemble_set_tuning applies a known
 * choice (-1: the built-in one; COLATUS_E_ARG for a shape that is not usable).
 * Either call synchronises the stream, drops the captured step graphs and
 * recomputes the step opening at the next colatus_ensemble_step; results
 * then follow the new shape's summation order (deterministic per shape). */
colatus_status colatus_ensemble_autotune(colatus_ens_t e, int reps, double out_ms[4], int *chosen);
colatus_status colatus_ensemble_set_tuning(colatus_ens_t e, int shape);
const char *colatus_ensemble_last_error(colatus_ens_t e);
void colatus_ensemble_destroy(colatus_ens_t e);

/* Tangent-linear model for finite-time Lyapunov growth of single tracers
 * (FP32; any of the three schemes).  Tangent b starts as a unit position
 * perturbation `dir` (host double[3]; NULL: x axis) on body seeds[b] only,
 * with zero velocity perturbation; the whole system's linear response is
 * then propagated:
 *     dF_k = G sum_{j != k} m_j J(d_kj) (dx_j - dx_k),  J(d) = I/s^3 - 3 d d^T/s^5,
 * through the same steps as the state (the linearisation of Eqs. 3-5 for
 * DKD, with the JVP at the half-drift positions).  After every step the norm
 * |(dx, dv)| of the seed body of each tangent is recorded (ring of
 * capacity_steps records); ln(norm)/t is the finite-time Lyapunov exponent.
 * Initialising replaces any previous tangents. */
colatus_status colatus_tangent_init(colatus_t ctx, const int64_t *seeds, int B, const double *dir,
                                    int64_t capacity_steps);
/* Advance the state and its tangents (the derivative of Eqs. 3-5 and of the
 * Eq. 1 force, Sec. I's tracer trajectories) by nsteps steps of size dt of the
 * configured scheme (FP32 precision only; the step size and the scheme may
 * change between calls).  COLATUS_E_STATE if the state was stepped without
 * them. */
colatus_status colatus_tangent_step(colatus_t ctx, double dt, int64_t nsteps);
/* Recorded growth, oldest first, host [nrec][B] floats; growth may be NULL
 * to query *nrec_out.  Synchronises. */
colatus_status colatus_tangent_read(colatus_t ctx, float *growth, int64_t *nrec_out);

/* Microbenchmark of the pipes the force roofline assumes, on the current
 * device: out[0] scalar FFMA lane-ops, out[1] packed FFMA2 (f32x2) lane-ops,
 * out[2] MUFU.RSQ results, each per SM per SM clock (independent chains, so
 * throughput-bound); out[3] SMs; out[4] blocks per SM used. */
colatus_status colatus_probe_pipes(double out[6]);

/* Release every device and host resource of ctx (NULL is a no-op). */
void colatus_destroy(colatus_t ctx);

#ifdef __cplusplus
}
#endif
#endif /* COLATUS_H */
