/*
 * coil.h -- C ABI of the B300 coupled electromagnetic-thermal coil stepper.
 *
 * The library advances the per-time-step coupled update of arXiv:2403.07666
 * (Numerical Algorithm section and Fig. 2b; Methods, heat-diffusion and E-J
 * paragraphs) over every conductor element of an axisymmetric coil:
 *
 *   1. the field on every element from the currents of all other elements
 *      plus the applied field (the dense coaxial-loop mutual-inductance
 *      operator M, complete elliptic integrals K and E);
 *   2. the E-J law E = rho(J) J with Jc(B, T, eps) and Joule heating E.J;
 *   3. the transport-current constraint of every turn (the A-V formulation:
 *      one loop-voltage unknown per wire) solved with the circuit equations
 *      (M + dt G) Idot - P u = -R,  P^T Idot = c  (linearly-implicit Euler);
 *   4. heat diffusion c dT/dt = div(kappa grad T) + E.J with T^3 laws and the
 *      bath sink -kappa grad T . n = h (T - T0) on the four borders, by ADI.
 *
 * Every step runs in hand-written CUDA kernels for sm_103a; there is no CPU
 * fallback.  The library owns all device memory of a coil; the caller owns
 * every host buffer passed in or out.  Arrays of per-element values are in
 * the element order
 *
 *     e = (t * n_layers + l) * n_sub^2 + b * n_sub + a
 *
 * (wire of layer l and turn t, element column a and row b inside the wire).
 * All functions return a coil_status by value; no C++ exception crosses the
 * ABI.  One handle must not be used by two host threads at once.
 */
#ifndef COIL_H
#define COIL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct coil coil_t;

typedef enum {
    COIL_OK = 0,
    COIL_ERR_INVALID = -1,        /* bad argument; nothing was changed */
    COIL_ERR_OOM = -2,            /* a device allocation failed */
    COIL_ERR_CUDA = -3,           /* a CUDA call failed; text in coil_last_error */
    COIL_ERR_NOT_CONVERGED = -4,  /* the per-step solve hit its iteration cap */
    COIL_ERR_NONFINITE = -5       /* NaN/Inf or a non-positive pivot appeared */
} coil_status;

enum { COIL_GEOM_SOLENOID = 0, COIL_GEOM_LIST = 1 };

/* Storage precision of the dense far part of M (row a3).  Near/self blocks,
 * the per-wire constraint solve and the accumulation of flux and temperature
 * are FP64 in every mode. */
enum { COIL_PREC_FP64 = 0, COIL_PREC_FP32 = 1, COIL_PREC_BF16 = 2 };

/*
 * Geometry (Numerical Algorithm section, Fig. 2a: axisymmetric cross-section,
 * square array of N_x x N_y turns, N_sub pieces per wire).
 *
 * COIL_GEOM_SOLENOID: n_layers x n_turns square wires of side wire_d on a
 *   pitch (epoxy gap pitch - wire_d, centred), first wire's inner face at
 *   r_in + gap/2, coil centred on z = 0, n_sub x n_sub square elements per
 *   wire.  transport = 1: every wire is a series turn carrying I_t(t);
 *   transport = 0: every element is a free loop.
 * COIL_GEOM_LIST: n_elem explicit square elements (centres r, z; side h)
 *   grouped in blocks of `block` consecutive elements; block_transport[w] = 1
 *   makes block w a turn carrying I_t(t), 0 leaves its loops free.  A list has
 *   no element grid: the stencil field (B = 0) and the thermal update are
 *   unavailable, so the material must use jc_model = 1 and thermal = 0.
 * Blocks (wires) hold at most 64 elements (n_sub <= 8).
 *
 * Subelements (Numerical Algorithm section: J = J_H + J_I, the field-driven
 * part J_H with zero net current in every subelement, the transport part J_I
 * spread over the whole wire with coupled subelements by the A-V
 * formulation).  n_groups > 1 with group[k] in [0, n_groups) for each of the
 * `block` element positions k of a turn (the same layout in every turn)
 * splits every transport turn into subelements: each step first solves J_I
 * on the turn alone (its own block of M + dt G, the resistive voltage
 * 2 pi r rho J_I of the transport part, the transport constraint), then the
 * coupled step with the net current rate of every subelement fixed to its
 * J_I share; J_I is kept as state.  Free loops are unaffected.  Limits:
 * every group non-empty, at most 6 subelements for blocks of up to 16
 * elements and COIL_MAX_GROUPS for larger blocks; coil_adjoint is unavailable
 * with subelements.
 * n_groups <= 1 (group may be NULL): one group, the plain turn constraint.
 */
#define COIL_MAX_GROUPS 16
typedef struct {
    int kind;
    int n_layers, n_turns, n_sub;
    double r_in, pitch, wire_d;
    int transport;
    int n_elem, block;
    const double *r, *z, *h;
    const int *block_transport;
    int n_groups;
    const int *group;
} coil_geometry;

/*
 * Material (Methods: E-J law, Kramer-type Jc, T^3 thermal laws).
 *   Jc = f Jc0 (1-T/Tc)^1.5 (1-|B|/Bc2(T))^2 / sqrt(|B|+B_reg)
 *        * max(0, 1 - C_eps |eps|^p_eps),  Bc2(T) = Bc2_0 (1 - (T/Tc)^2),
 *   (jc_model = 1: Jc = f Jc0);  filament elements follow E0 (J/Jc)^n in
 *   parallel with rho_n, Cu elements are ohmic (rho_n).
 *   c = c0 T^3 [J/kg/K] at density rho_m, kappa = kappa_{cu,ep} (T/T_ref)^3,
 *   bath coefficient h0 (T/T_ref)^3, bath temperature T_bath.
 * jc_factor (f), strain (eps) and mat (1 = filament, 0 = Cu) are per-element
 * host arrays of length N, copied at coil_create.
 * Y_eff [Pa] > 0 adds the Lorentz-force hoop strain of the winding (Flux
 * Jumps Propagation section: the electromagnetic strain produced by the
 * Lorentz force, to which Jc of Nb3Sn is sensitive): the strain of element e is
 *   eps_e = strain_e + r_e J_e B_z,e / Y_eff
 * from the start-of-step current density and axial field (hoop stress r J B_z
 * of a loop carrying J in the axial field B_z, over an effective Young's
 * modulus of the winding).  Y_eff = 0: the static strain only.
 */
typedef struct {
    double E0, n, Jc0, Tc, Bc2_0, B_reg, C_eps, p_eps;
    double rho_n, rho_m, c0, kappa_cu, kappa_ep, h0, T_ref, T_bath;
    int jc_model;
    int thermal;
    const double *jc_factor;
    const double *strain;
    const int *mat;
    double Y_eff;       /* > 0: Lorentz hoop strain on; 0: off */
} coil_material;

/*
 * Options.  rtol: the per-step projected PCG stops when the preconditioned
 * residual norm falls below rtol times the preconditioned norm of the step's
 * right-hand side.  maxit: iteration cap (then COIL_ERR_NOT_CONVERGED).
 * stream: a cudaStream_t to launch on (NULL: the library creates one).
 * diag_capacity: per-step diagnostic records kept on the device (ring).
 * profile: record a CUDA event pair around every operator launch on the coil's
 * stream (coil_info reports their summed duration; in the tensor-core format
 * the pair brackets the tensor-core product kernel, not the input split); the
 * step's kernels are then launched one by one, the convergence test read
 * after every PCG iteration.  Without it a step runs as one CUDA graph.
 */
typedef struct {
    int precision;
    double rtol;
    int maxit;
    int device;
    void *stream;
    long diag_capacity;
    int profile;        /* 1: time every operator apply with CUDA events */
    int format;         /* COIL_FORMAT_DENSE, _TOEPLITZ or _TOEPLITZ_TC */
} coil_options;

/* Storage format of the far operator.  DENSE: N x N rows in `precision`.
 * TOEPLITZ (regular solenoids, FP32 only): the coaxial-loop inductance depends
 * on r, r' and z - z' only, so between turn rows t and t' the operator is one
 * C x C block of offset t - t' (C = n_layers n_sub^2); the 2 n_turns - 1
 * distinct blocks are stored (C^2 (2 n_turns - 1) entries instead of N^2, the
 * same FP32 values as the dense form) and applied as a Toeplitz-structured
 * FP32 matrix product.
 * TOEPLITZ_TC (regular solenoids with n_turns <= 112, FP32 precision only):
 * the blocks of offsets >= 0 (the others are their transposes), each entry
 * stored as two FP16 numbers hi + lo after a power-of-two scaling (about 22
 * significant bits, 4 bytes per entry: half the bytes of the FP32 Toeplitz
 * table), applied on the tensor cores to an equally split input with three
 * products hi*hi, hi*lo and lo*hi (lo*lo, below 2^-22 of the result, is
 * left out), FP32 accumulation per stage and compensated sums across stages.  Unsupported shapes get COIL_ERR_INVALID.
 * A bounded wait inside the apply kernel that runs out makes the step return
 * COIL_ERR_CUDA ("tensor-core apply timed out"). */
enum { COIL_FORMAT_DENSE = 0, COIL_FORMAT_TOEPLITZ = 1, COIL_FORMAT_TOEPLITZ_TC = 2 };

/*
 * Drive (Numerical Algorithm section: ramping transport current I_a and
 * ramping external field H_a).  I_t(t) = min(ramp_rate t, I_max).
 * Ba_waveform 0: no applied field; 1: B_a = min(Ba_rate t, Ba_max);
 * 2: triangle 0 -> +Ba_max -> -Ba_max -> 0 with slope Ba_rate, repeated.
 */
typedef struct {
    double dt, ramp_rate, I_max, Ba_rate, Ba_max;
    int Ba_waveform;
} coil_drive;

/* Number of doubles in one diagnostic record and their order:
 * t, I_t, V_term (sum of loop voltages), moment sum(pi r^2 I), Joule power
 * sum(q 2 pi r a) of the step's start state, T_max after the step,
 * max |J|/Jc over filament elements (flux-jump criterion |J/Jc| > 1,
 * Flux Jumps Propagation section), max over wires of the mean rho/rho_n of
 * their filament elements (quench criterion rho > 0.95 rho_n, Quenches
 * Propagation section), PCG iterations, final relative residual. */
#define COIL_DIAG_WIDTH 10

typedef struct {
    long n_elem, n_blocks, block, grid_r, grid_z;
    int precision;
    size_t operator_bytes;        /* bytes of the stored far operator */
    size_t device_bytes;          /* all device memory held by the handle */
    long steps;                   /* completed steps */
    double t;                     /* simulated time after the last step */
    double setup_ms;              /* operator assembly + upload */
    long long kernel_launches;    /* kernels launched by coil_step so far */
    long long operator_launches;  /* dense-operator (GEMV) launches so far */
    double operator_ms;           /* their summed duration (profile = 1) */
    long long pcg_iterations;     /* summed over all steps */
    size_t descriptor_bytes;      /* host-to-device bytes uploaded per coil_step call */
    int step_graph;               /* 1: each step runs as one CUDA graph (its PCG loop a
                                     device-controlled while node); profile = 1 launches
                                     the kernels one by one to time every operator apply */
} coil_info_t;

/* Zero the launch / timing counters of coil_info. */
coil_status coil_reset_counters(coil_t *c);

/* Create a coil: validate, upload, assemble M on the device (far part in the
 * chosen precision, intra-wire blocks in FP64).  State: I = 0, T = T_bath,
 * t = 0.  On failure *out is NULL and nothing is leaked. */
coil_status coil_create(const coil_geometry *geom, const coil_material *mat,
                        const coil_options *opt, coil_t **out);

/* Advance n_steps time steps with the drive.  Runs entirely on the device;
 * returns after the stream has finished.  A non-OK status leaves the state
 * at the end of the last completed step (see coil_info.steps). */
coil_status coil_step(coil_t *c, long n_steps, const coil_drive *drive);

/* Advance n_steps of n_coils coils together (batched sweep of coil variants
 * and ramp rates of uneven size): every kernel of the step is launched once
 * for the whole batch, one grid row (blockIdx.y) per coil, each coil with
 * its own drive drives[i] and its own convergence test.  All coils must live
 * on the same device and use the same operator precision; the launches go to
 * the first coil's stream.  A coil whose solve fails stops advancing; the
 * call returns the first failure after the others completed the step. */
/* With the tensor-core format the coils' applies run side by side on side
 * streams, each with the two-fill schedule and its floor of schedule steps
 * per CTA (a small coil's apply on a few SMs) in place of its autotuned one;
 * a coil stepped alone afterwards returns to its autotuned schedule, and a
 * coil stepped alone with that batch schedule (coil_set_tc_schedule(c, 0, 0,
 * 0)) gets bit for bit what the batch gives it. */
coil_status coil_batch_step(coil_t *const *coils, int n_coils, long n_steps,
                            const coil_drive *drives);

/* Replace the calibration parameters of the E-J / Jc laws (Methods: the laws
 * are fitted to a measured magnetization loop): the per-element Jc factor
 * (host array of N doubles, NULL = keep), the creep exponent n (>= 1) and the
 * strain coefficient C_eps. */
coil_status coil_set_params(coil_t *c, const double *jc_factor, double n, double C_eps);

/* Discrete adjoint of n_steps coupled steps starting from the current state
 * (gradients for calibrating the E-J / Jc laws against a magnetization loop).
 * dL_dm[k] is the derivative of the caller's loss with respect to the moment
 * sum(pi r^2 I) after step k+1 (host array of n_steps doubles).  The call runs
 * the n_steps forward, keeping the state every ckpt_every steps, then sweeps
 * backwards: each reverse step recomputes its segment's forward states from
 * the last checkpoint and applies the hand-written reverse of every kernel of
 * the step (transposed per-step solve with the same projected PCG, E-J and Jc
 * Jacobians including the dependence of the solve's matrix on G, stencil
 * transpose, one operator apply for M^T = M, reverse ADI).  Outputs (host,
 * NULL = skip): g_jc_factor[N] = dL/d(jc_factor), *g_n = dL/dn,
 * *g_C_eps = dL/dC_eps.  On return the state is the one after the n_steps
 * forward steps.  Scratch device memory is allocated for the call and freed
 * before it returns. */
coil_status coil_adjoint(coil_t *c, long n_steps, const coil_drive *drive, int ckpt_every,
                         const double *dL_dm, double *g_jc_factor, double *g_n,
                         double *g_C_eps);

/* The adjoint of coil_adjoint for a loss on two per-step series: dL_dm[k]
 * as above (the moment after step k+1) and dL_dP[k], the derivative of the
 * loss with respect to the Joule power P_k = sum q 2 pi r a of the start
 * state of step k (column 4 of the diagnostic records; it rises steeply when
 * filaments go normal, so a soft maximum of P over the steps is a smooth
 * quench-onset loss: Quenches Propagation section, the Joule heat released
 * from the onset of the rise of rho to the quench).  Either array may be
 * NULL (not both); everything else as coil_adjoint. */
coil_status coil_adjoint_losses(coil_t *c, long n_steps, const coil_drive *drive, int ckpt_every,
                                const double *dL_dm, const double *dL_dP, double *g_jc_factor,
                                double *g_n, double *g_C_eps);

/* Copy the current state to host buffers of N doubles (NULL = skip): current
 * density J [A/m^2], B_r, B_z [T] from the stencil of the loop flux, T [K];
 * and the moment sum(pi r^2 I) [A m^2].  `Ba` is the applied field at the
 * current time, needed for B (pass the drive used by coil_step, or NULL for
 * B_a = 0). */
coil_status coil_read(coil_t *c, const coil_drive *Ba, double *J, double *Br,
                      double *Bz, double *T, double *moment);

/* Same as coil_read but into DEVICE buffers of N doubles (NULL = skip). */
coil_status coil_read_device(coil_t *c, const coil_drive *Ba, double *dJ,
                             double *dBr, double *dBz, double *dT);

/* Diagnostic records of steps [first, first + count) into out[count][10]. */
coil_status coil_read_diag(coil_t *c, long first, long count, double *out);

/* Per wire: first step index whose start state met the flux-jump criterion
 * (max |J|/Jc > 1) and the quench criterion (mean rho/rho_n > 0.95); -1 if
 * never.  Host arrays of n_blocks longs. */
coil_status coil_read_onsets(coil_t *c, long *first_jump, long *first_quench);

/* Per-wire statistics of the forward steps taken so far (Flux Jumps
 * Propagation and Quenches Propagation sections), into the host array
 * out[7][n_blocks] (row-major, a row per quantity):
 *   0  Q_total: Joule heat per unit of time integrated by the rectangle rule,
 *      sum over steps of dt * P_w, P_w = sum_e q_e 2 pi r_e a_e [J]
 *   1  T_max: maximum element temperature over the start-of-step states [K]
 *   2  P_max: maximum Joule power density q = rho J^2 over them [W/m^3]
 *   3  Q_at_jump, 4 Q_at_rise, 5 Q_at_quench: Q_total before the step whose
 *      start state first met max |J|/Jc > 1, mean rho/rho_n > 0.05 and mean
 *      rho/rho_n > 0.95 respectively; -1 while not met
 *   6  first_rise: index of that step for the resistivity rise, -1 if never.
 * The adjoint's recomputations do not count; coil_save_state/coil_load_state
 * carry these statistics. */
coil_status coil_read_wire_stats(coil_t *c, double *out);

/* Start a new observation window: the statistics above back to 0 / -1 and the
 * onsets of coil_read_onsets back to -1. */
coil_status coil_reset_wire_stats(coil_t *c);

/* Element currents I [A] (host, N doubles) and set them (state injection for
 * tests; also resets the accumulated flux to M I). */
coil_status coil_get_currents(coil_t *c, double *I);
coil_status coil_set_currents(coil_t *c, const double *I);

/* Apply the assembled operator: y = M p (far part in the stored precision
 * plus the FP64 intra-wire blocks), host vectors of N doubles. */
coil_status coil_apply_operator(coil_t *c, const double *p, double *y);

/* Same product as coil_apply_operator, y = M p, for callers that must not
 * allocate device memory after set-up: code running while a stream is being
 * captured into a CUDA graph, real-time control loops that fix their memory
 * at start-up, or processes whose device memory is capped by a scheduler.
 * The paper has no counterpart; this is an interface convenience.
 *
 * d_p (input) and d_y (output) are DEVICE arrays of n_elem doubles owned by
 * the caller.  Nothing is allocated or freed: the zero-padded copy of p that
 * the operator kernels read lives in one file-scope device array of
 * 1,048,576 doubles (8 MiB), which every device that loads the library holds
 * until the process exits.  Coils whose operator pitch (n_elem rounded up to
 * 64) exceeds 1,048,576 get COIL_ERR_INVALID, and so do coils whose far
 * operator is not in the dense format (COIL_FORMAT_TOEPLITZ and
 * COIL_FORMAT_TOEPLITZ_TC are not accepted here).  The first call on a device
 * looks up that array's device address (one cudaGetSymbolAddress); make that
 * first call before any stream capture.  Launches go to `stream` (a
 * cudaStream_t, NULL = default stream) and the call returns without waiting;
 * d_y is ready when the stream reaches that point.  Every call shares the
 * array and it keeps the last call's contents: two calls that overlap on the
 * GPU (different streams or threads at the same time) race on it and give
 * wrong results.  The looked-up address is kept for the life of the process:
 * after a cudaDeviceReset (or anything else that destroys the device's
 * primary context) it is stale, and this entry point must not be called
 * again in that process. */
coil_status coil_apply_operator_static(coil_t *c, const double *d_p, double *d_y,
                                       void *stream);

/* Read the dense operator row by row into a host N x N FP64 array
 * (far part converted from its storage precision, near blocks added). */
coil_status coil_read_operator(coil_t *c, double *M);

/* Serialise / restore the FP64 state (I, flux, T^4, t, step, the last three
 * steps' Idot that start the next PCG,
 * onsets and per-wire statistics).
 * With buf == NULL, *bytes receives the required size. */
coil_status coil_save_state(coil_t *c, void *buf, size_t *bytes);
coil_status coil_load_state(coil_t *c, const void *buf, size_t bytes);

/* Test hook of the failure path of the tensor-core apply (COIL_FORMAT_
 * TOEPLITZ_TC): the bounded waits inside its kernel that raise the kernel's
 * abort flag give up after `cycles` SM clock cycles instead of their default
 * (cycles = 0 restores it: 2^31 cycles, about a second).  A limit of a few
 * cycles makes the next apply stop early on purpose: the CTA that gave up
 * raises the flag, the others stop issuing, the copies and products already
 * in flight are waited for (with the default limit), the tensor memory is
 * freed and the step returns COIL_ERR_CUDA ("tensor-core apply timed out")
 * with I, flux, T and t of the last completed step (the warm start of the
 * next solve and the per-wire statistics may include the stopped attempt).
 * The GPU context stays usable, and the coil steps normally once the limit
 * is back at 0.  Other formats ignore the limit.  COIL_ERR_INVALID for
 * cycles < 0. */
coil_status coil_set_wait_limit(coil_t *c, long long cycles);

/* Schedule of the tensor-core apply (COIL_FORMAT_TOEPLITZ_TC).  coil_create
 * picks it with an autotuner: a few candidate schedules are timed on the
 * coil's own table (CUDA events around four applies each) and the fastest is
 * kept; the choice is remembered for later coils of the same shape (channels,
 * turns, SM count, device) in the process.  mode 0: every stored tile is
 * loaded by the CTAs of both of its products (the tile and its transpose);
 * mode 1: one load serves both products (a 128-row and a 64-row MMA per
 * tile).  n_cta: CTAs of the apply; stages: table tiles in flight per CTA;
 * us: measured duration of one apply [microseconds].  COIL_ERR_INVALID for
 * other formats. */
coil_status coil_tc_schedule(const coil_t *c, int *mode, int *n_cta, int *stages, double *us);

/* The autotuner's candidates of the last tuning run: on entry *count is the
 * capacity of out (rows), on return the number of candidates; out[i][4] =
 * (mode, n_cta, stages, us).  out may be NULL to query the count. */
coil_status coil_tc_candidates(const coil_t *c, int *count, double *out);

/* Pin the schedule: mode 0 or 1 with n_cta <= 0 and stages <= 0 for that
 * mode's defaults (mode 0 takes no CTA count), or mode -1 to run the
 * autotuner again.  The new schedule is timed; COIL_ERR_INVALID when the
 * coil's shape does not admit it. */
coil_status coil_set_tc_schedule(coil_t *c, int mode, int n_cta, int stages);

coil_status coil_info(const coil_t *c, coil_info_t *info);
const char *coil_last_error(const coil_t *c);
void coil_destroy(coil_t *c);

#ifdef __cplusplus
}
#endif
#endif /* COIL_H */
