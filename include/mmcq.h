/*
 * mmcq.h -- C ABI of the GB300 (sm_103a) library for the LLG + cavity-QED hot
 * path of Mumax3-cQED (arXiv 2410.00966).
 *
 * One handle holds `batch` independent instances that share a grid, a cell
 * size, the material constants, the per-cell Ms map and the coupling-profile
 * shape; each instance has its own magnetisation, bias field, cavity
 * (omega_c, kappa, g, x0, p0) and integrator state (time, step size,
 * accept/reject counters).  Every step runs on the GPU: the zero-padded FFT
 * demag convolution, exchange, anisotropy, Zeeman, the cavity field
 * B_rms * Gamma(t) from an FP64 reduction of the coupling-weighted
 * magnetisation, the LLG torque and the RK4 / Dormand-Prince update with |m|
 * renormalisation.  Nothing of the step runs on the host.
 *
 * Conventions for every call:
 *   - Return 0 (MMCQ_OK) or a negative MMCQ_ERR_* code; no exception crosses
 *     the ABI.  mmcq_last_error() gives a one-line message for the handle.
 *   - Arrays are row-major with x fastest: cell i = (z * ny + y) * nx + x.
 *     Vector arrays are N x 3 float (x, y, z components interleaved).
 *   - `where` = MMCQ_HOST (host pointer, caller-owned, copied before the call
 *     returns) or MMCQ_DEVICE (device pointer on the handle's device; the copy
 *     is ordered on the handle's stream and has completed when the call returns).
 *   - `inst` selects one instance (0 <= inst < batch); -1 means all instances
 *     where the call says so.
 *   - Stepping is enqueued on the handle's stream and returns without waiting;
 *     errors detected on the device (non-finite values, step-size underflow)
 *     are reported by the next call that synchronises (mmcq_sync, mmcq_get_*).
 *   - A handle is not thread-safe; distinct handles are independent.
 *   - Units are SI: m, s, T, A/m, J/m, J/m^3, rad/s.
 */
#ifndef MMCQ_H
#define MMCQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mmcq mmcq_t;

enum {
    MMCQ_OK = 0,
    MMCQ_ERR_ARG = -1,         /* invalid argument (sizes, pointers, indices) */
    MMCQ_ERR_UNSUPPORTED = -2, /* valid request this build does not handle (e.g. padded size > 4096) */
    MMCQ_ERR_CUDA = -3,        /* a CUDA runtime call failed; see mmcq_last_error */
    MMCQ_ERR_NUMERIC = -4,     /* non-finite m / field (RK4), or adaptive step underflow (DP45: a
                                  non-finite trial attempt is rejected and the step shrunk) */
    MMCQ_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
    MMCQ_ERR_STATE = -6        /* call not valid in the current state */
};

enum { MMCQ_HOST = 0, MMCQ_DEVICE = 1 };
enum { MMCQ_RK4 = 0, MMCQ_DP45 = 1 };
enum { MMCQ_CAVITY_E = 0, MMCQ_CAVITY_P = 1 };

/* field-term selection for mmcq_eval_field */
enum {
    MMCQ_TERM_DEMAG = 1,
    MMCQ_TERM_EXCHANGE = 2,
    MMCQ_TERM_ANIS = 4,
    MMCQ_TERM_ZEEMAN = 8,
    MMCQ_TERM_CAVITY = 16,
    MMCQ_TERM_ALL = 31
};

typedef struct {
    int nx, ny, nz;        /* cells per axis, >= 1 */
    double dx, dy, dz;     /* cell size (m), > 0 */
    int batch;             /* instances sharing this grid, >= 1 */
} mmcq_grid;

/* Device-memory hooks: when alloc is non-NULL every device buffer of the
 * handle is obtained from alloc(bytes, ctx) (256-byte aligned) and released
 * with free(ptr, ctx) at mmcq_destroy; otherwise cudaMalloc / cudaFree. */
typedef void* (*mmcq_alloc_fn)(size_t bytes, void* ctx);
typedef void (*mmcq_free_fn)(void* ptr, void* ctx);

typedef struct {
    double gamma;          /* gyromagnetic ratio rad/(s T); 0 -> 1.7595e11 */
    double mu0;            /* vacuum permeability; 0 -> 4 pi 1e-7 */
    double hbar;           /* 0 -> 1.05457182e-34 (the paper's HBAR default, Sec. 3.2) */
    int device;            /* CUDA device ordinal */
    void* stream;          /* cudaStream_t to enqueue on; NULL -> a stream owned by the handle */
    mmcq_alloc_fn alloc;   /* optional device allocator */
    mmcq_free_fn free;
    void* alloc_ctx;
} mmcq_opts;

typedef struct {
    double t;              /* simulated time of the instance (s) */
    double t_cav;          /* time since the cavity was set or reset (s) */
    double re_alpha, im_alpha; /* photon amplitude alpha = <a> (Sec. 2.2) */
    double n_photon;       /* |alpha|^2 */
    double Gamma;          /* memory factor Gamma(t_cav), Eq. (gammafinal) */
    double S, C;           /* P-mode accumulators (J s, include V_c), Eq. (Sdiscrete, Cdiscrete) */
    double X;              /* V_c sum_i Ms_i m_i . B_rms,i at the current m (J) */
    double dt;             /* next trial step (DP45) or last step (RK4) */
    int64_t accepted, rejected;
    double err;            /* DP45: error estimate max_i |m5_i - m4_i| of the last attempt, the value
                              the step controller used (FP32 on the device, widened); 0 for RK4 */
} mmcq_cavity;

typedef struct {
    int px, py, pz;            /* padded FFT sizes */
    int tile;                  /* kx columns per spectrum tile */
    size_t device_bytes;       /* device memory held by the handle */
    double setup_ms;           /* demag-tensor set-up time */
    int64_t launches_per_step; /* kernels launched by one RK4 step / one DP45 attempt */
} mmcq_info;

/* Create a handle: allocate device state and compute the demag kernel.
 * The demag tensor is the Newell, Williams & Dunlop (1993) cell-averaged
 * tensor within 16 largest-cell-edges and the point dipole beyond, evaluated
 * in FP64 on the device and transformed with an FP64 FFT on the padded grid;
 * the paper lists B_demag among the field terms (Sec. 2.1) without giving a
 * method.  Ms (A/m), Aex (J/m), alpha (Gilbert damping, Eq. llg), Ku (J/m^3)
 * and axis (normalised here) are shared by all instances.  Initial state:
 * m = +x, uniform Ms, zero bias, cavity off, RK4, E-mode.
 * Padding: each axis is zero-padded to the smallest power of two >= 2n - 1.
 * Errors: MMCQ_ERR_ARG (null/invalid), MMCQ_ERR_UNSUPPORTED (nx > 1024, or
 * ny or nz > 2048), MMCQ_ERR_CUDA. On error *h is set to NULL. */
int mmcq_create(mmcq_t** h, const mmcq_grid* g, double Ms, double Aex, double alpha, double Ku,
                const double axis[3], const mmcq_opts* opts);
void mmcq_destroy(mmcq_t* h);
const char* mmcq_last_error(const mmcq_t* h);
int mmcq_info_get(mmcq_t* h, mmcq_info* out);

/* Per-cell saturation magnetisation (A/m), shared by all instances; 0 marks
 * empty cells (geometry mask).  Ms enters the cavity sum as M_{s,i}
 * (Eq. gammafinal).  N floats.  Cells that become empty get m = 0. */
int mmcq_set_ms_map(mmcq_t* h, const float* ms, int where);

/* Uniform Zeeman field B_ext (T) of one instance or all (inst = -1), Sec. 2.1. */
int mmcq_set_bias(mmcq_t* h, int inst, const double B[3]);

/* Magnetisation of one instance or of all (inst = -1: the same N x 3 array
 * for every instance).  Normalised on entry (FP64), zero in empty cells.
 * A non-finite direction is stored as zero and reported as MMCQ_ERR_NUMERIC
 * by the next call that synchronises (mmcq_sync, mmcq_get_*).
 * Invalidates the first-same-as-last stage of the adaptive integrator. */
int mmcq_set_m(mmcq_t* h, int inst, const float* m, int where);
int mmcq_get_m(mmcq_t* h, int inst, float* out, int where);

/* Single-mode cavity of one instance or all (inst = -1): Sec. 3.2 built-ins
 * Wc (omega_c, rad/s), Kappa (kappa, rad/s) and B_rms.  The cavity field is
 * B_cav,i = B_rms,i Gamma(t) (Eq. bcav).
 *   profile: N x 3 host floats shared by the whole batch, or NULL to keep the
 *            current shape (initially the uniform unit vector +y).
 *   profile_is_brms = 1: profile is B_rms in tesla, g is ignored.
 *   profile_is_brms = 0: profile is a dimensionless shape p_i and
 *            B_rms,i = g sqrt(2 hbar / (gamma V_c sum_i Ms_i)) p_i, the
 *            macrospin relation g = B_rms sqrt(gamma Ms V / (2 hbar)) obtained
 *            by matching the linearised equations of motion to the normal-phase
 *            polariton formula (Eq. dickepolaritons, Sec. 4).
 * Sets t_cav = 0, S = C = 0, alpha = alpha0 and enables the cavity
 * (CavityFeatureStatus = 1 in the paper's terms). */
int mmcq_set_cavity(mmcq_t* h, int inst, double omega_c, double kappa, double g, const float* profile,
                    int profile_is_brms);
/* Cavity mode `mode` (0 .. 3) of one instance or all: the same arguments as
 * mmcq_set_cavity, which sets mode 0.  Every enabled mode k adds
 * B_rms,k Gamma_k to the field and follows its own amplitude equation driven
 * by X_k = V_c sum_i Ms_i m_i . B_rms,k,i (the paper keeps one mode and notes
 * that more modes follow the same equations, Sec. 4).  Each mode has its own
 * profile map, shared by the instances.  Configuring any mode restarts the
 * cavity memory of every mode of the selected instances (t_cav = 0,
 * S = C = 0, alpha_k = alpha_k(0)).  MMCQ_ERR_ARG for a mode outside 0..3. */
int mmcq_set_cavity_mode(mmcq_t* h, int inst, int mode, double omega_c, double kappa, double g,
                         const float* profile, int profile_is_brms);
/* x0 = 2 Re alpha0, p0 = -2 Im alpha0 (Sec. 3.2 built-ins X0, P0; the paper's
 * wording after Eq. gammadiscretefinal is read with alpha0). Resets alpha. */
int mmcq_set_cavity_init(mmcq_t* h, int inst, double x0, double p0);
int mmcq_set_cavity_init_mode(mmcq_t* h, int inst, int mode, double x0, double p0);
/* ResetMemoryTerm() (Sec. 3.2): t_cav := 0, S = C = 0, alpha := alpha0, every mode. */
int mmcq_reset_cavity(mmcq_t* h, int inst);
int mmcq_disable_cavity(mmcq_t* h, int inst);

/* kind: MMCQ_RK4 (classic, fixed step) or MMCQ_DP45 (Dormand-Prince 5(4),
 * adaptive: error = max_i |m5_i - m4_i|, accept if <= tol, next step
 * dt * clamp(0.9 (tol/err)^(1/5), 0.2, 5)); m is renormalised after each
 * accepted step.  cavity_mode: MMCQ_CAVITY_E integrates alpha with the same
 * tableau (exact memory integral, Appendix A); MMCQ_CAVITY_P uses the paper's
 * recursive accumulators S_n, C_n (Eq. Sdiscrete, Cdiscrete) folded in after
 * each accepted step and Gamma from Eq. (gammadiscretefinal) at every stage. */
int mmcq_set_integrator(mmcq_t* h, int kind, double tol, int cavity_mode);

/* Optional end time per instance (or all, inst = -1) for the adaptive
 * integrator: steps are clipped to land on t_end and further attempts are
 * skipped.  t_end <= 0 removes the limit. */
int mmcq_set_horizon(mmcq_t* h, int inst, double t_end);

/* Advance every instance.  RK4: n steps of dt.  DP45: n attempts; dt > 0
 * sets the next trial step of every instance.  Asynchronous on the stream. */
int mmcq_step(mmcq_t* h, int64_t n, double dt);

/* Wait for the stream; report device-side errors raised since the last sync. */
int mmcq_sync(mmcq_t* h);

/* FP64 cavity / integrator read-out (Sec. 2.2 a-posteriori photon amplitude;
 * in P-mode alpha is rebuilt from S and C).  inst = -1 fills out[0..batch-1]
 * for every instance in one call; otherwise out is one struct. */
int mmcq_get_cavity(mmcq_t* h, int inst, mmcq_cavity* out);
/* The same read-out for cavity mode `mode` (mmcq_get_cavity reads mode 0). */
int mmcq_get_cavity_mode(mmcq_t* h, int inst, int mode, mmcq_cavity* out);

/* Pipelined read-out (mode 0, every instance), for a loop that reads each
 * step's result without draining the GPU between steps:
 *   mmcq_post_cavity enqueues on the handle's stream the read-out as of the
 *   work enqueued so far (the coupling sums, then a copy of the instance
 *   states, the sums and the error flags into one of MMCQ_POST_SLOTS pinned
 *   host buffers owned by the handle) and returns without waiting.
 *   mmcq_take_cavity waits for the oldest posted read-out and fills
 *   out[0..batch-1] with what mmcq_get_cavity(h, -1, out) would have returned
 *   at that point (converted with the instance parameters current at take).
 * Steps enqueued between a post and its take run while the host waits.
 * Errors: MMCQ_ERR_STATE when every slot is taken (post) or nothing is posted
 * (take); MMCQ_ERR_NUMERIC from take when the device raised a non-finite or
 * step-underflow flag before the posted point (the flag is then cleared, as by
 * mmcq_sync); MMCQ_ERR_CUDA on a failed copy or allocation (the slots are
 * allocated by the first post). */
#define MMCQ_POST_SLOTS 4
int mmcq_post_cavity(mmcq_t* h);
int mmcq_take_cavity(mmcq_t* h, mmcq_cavity* out);

/* Accepted step lengths of one instance in order (at most max are copied;
 * *n receives the total count).  Used to replay adaptive runs. */
int mmcq_get_dt_history(mmcq_t* h, int inst, double* out, int64_t max, int64_t* n);

/* ---- excitation and spectra (Appendix C) --------------------------------
 * mmcq_set_drive: the excitation of the paper's example script, added to the
 *   external field of one instance or all (inst = -1):
 *     B_ext,i(t) += amp * B_rms,i * sinc(omega_cut * (t - t0)),  sinc(0) = 1,
 *   with B_rms,i the instance's coupling map (mmcq_set_cavity; it stays in
 *   use after mmcq_disable_cavity), t the simulation time at each Runge-Kutta
 *   stage, omega_cut in rad/s.  amp = 0 turns it off.  Part of the Zeeman term
 *   of mmcq_eval_field.
 * mmcq_set_recording: every > 0 records (t, <mx>, <my>, <mz>) of every
 *   instance after every `every`-th accepted step, <m> the mean of m over the
 *   magnetised cells (FP64 sums); 0 stops.  Capacity 65536 samples per
 *   instance (then MMCQ_ERR_STATE from the read-out).  First use allocates
 *   32 bytes x 65536 per instance.
 * mmcq_get_mavg_history: copies up to max samples of one instance into out
 *   (host, caller owned, max x 4 doubles: t, <mx>, <my>, <mz>); *n = samples.
 * mmcq_spectrum: on the device, the Fourier transform of one component
 *   (comp 0..2) of an instance's recorded <m>:
 *     S(w) = sum_n c_n (y_n - ybar) exp(-i w t_n),
 *   c_n the trapezoid weights of the sample times (any spacing), ybar their
 *   time average, at the nw angular frequencies omega (host, rad/s); out
 *   (host, 2 nw doubles) receives Re, Im.  MMCQ_ERR_STATE if recording was
 *   never on. */
int mmcq_set_drive(mmcq_t* h, int inst, double amp, double omega_cut, double t0);
int mmcq_set_recording(mmcq_t* h, int every);
int mmcq_get_mavg_history(mmcq_t* h, int inst, double* out, int64_t max, int64_t* n);
int mmcq_spectrum(mmcq_t* h, int inst, int comp, const double* omega, int nw, double* out);

/* ---- gradients: discrete adjoint of the RK4 path ------------------------
 * Objective per instance b (mode 0 amplitude alpha, <m> the mean over the
 * magnetised cells, alpha_n the amplitude after step n of N):
 *   J_b = w . <m>(T) + wn |alpha_N|^2 + wavg (1/W) sum_{n = N-W+1}^{N} |alpha_n|^2,
 * the last term the photon number averaged over the final W = window steps
 * (times hbar omega_c: the photon energy).
 *
 * mmcq_adjoint_rk4 runs nsteps RK4 steps of dt from the current state of
 * every instance (E-mode, cavity mode 0 only, no drive), keeping a
 * checkpoint (m and the FP64 instance state) every ckpt_every steps on the
 * device (0 or 1: every step; memory 16 B x cells x instances per checkpoint
 * plus ckpt_every states for the segment being replayed), then sweeps back
 * through the discrete adjoint of each step: the states of a segment are
 * recomputed from its checkpoint, the four stages of each step from its
 * state, and the renormalisation is included.
 *   J (host, B doubles, may be NULL): J_b.
 *   grad (host, B x 6 doubles): dJ_b/d(B_ext x, y, z; eta; omega_c; kappa), eta
 *     the scale of the instance's B_rms map at eta = 1 (dJ/dg = grad[3] / g
 *     when B_rms comes from g).
 *   grad_ms (host, B x N floats, may be NULL): dJ_b/dMs_i per cell with the
 *     magnetic mask and the B_rms map held fixed (0 on empty cells).
 * The demag convolution of the adjoint field reuses the forward passes (the
 * tensor is symmetric).  The state is left at step nsteps and the integrator
 * setting is restored.  MMCQ_ERR_UNSUPPORTED in P-mode, with more than one
 * mode or with the drive on; MMCQ_ERR_ARG for nsteps < 1, dt <= 0,
 * ckpt_every < 0 or a NULL obj / grad. */
typedef struct {
    double w[3];      /* weights of <m>(T) */
    double wn;        /* weight of |alpha(T)|^2 */
    double wavg;      /* weight of the photon number averaged over the last `window` steps */
    int64_t window;
} mmcq_objective;
int mmcq_adjoint_rk4(mmcq_t* h, int64_t nsteps, double dt, const mmcq_objective* obj, int64_t ckpt_every,
                     double* J, double* grad, float* grad_ms);

/* ---- checkpoint / resume -----------------------------------------------
 * A snapshot holds everything that evolves in time or was set per instance:
 * for every instance the accepted m, the first Dormand-Prince stage kept for
 * first-same-as-last reuse, the integrator and cavity state (t, t_cav, dt,
 * alpha, S, C, counters) and the instance parameters (bias, omega_c, kappa,
 * g, x0, p0), plus the integrator choice.  Configuration that is shared by
 * all instances (grid, material, Ms map, coupling profile) is not stored: the
 * handle that restores must have been created and configured the same way.
 * Resuming from a snapshot continues bit-for-bit as the original run.  The
 * dt history restarts empty.
 *
 * mmcq_get_state: synchronises; writes the snapshot (host memory, caller
 *   owned) when buf is non-NULL and cap >= its size; *size = its size.
 *   buf == NULL only reports the size.  MMCQ_ERR_ARG if cap is too small.
 * mmcq_set_state: MMCQ_ERR_ARG if the snapshot is truncated, is not one, or
 *   was taken on a handle of another grid or batch size; nothing changes then. */
int mmcq_get_state(mmcq_t* h, void* buf, int64_t cap, int64_t* size);
int mmcq_set_state(mmcq_t* h, const void* buf, int64_t size);

/* Effective field (T) of one instance at its current m, with the selected
 * MMCQ_TERM_* terms (cavity term uses the current Gamma); N x 3 floats. */
int mmcq_eval_field(mmcq_t* h, int inst, int terms, float* out, int where);

/* ---- allocation-free coupling sum ---------------------------------------
 * The paper has no counterpart to this call.  It computes
 * X = vc * sum_i ms[i] * (m_i . brms_i) in FP64 (the same sum that drives the
 * cavity, reported as X by mmcq_get_cavity) for callers that cannot allocate
 * device memory: code running inside a host framework whose own memory pool
 * owns the device and forbids allocations behind its back, or a latency-bound
 * loop that cannot afford cudaMalloc's implicit device synchronisation.  No
 * handle is needed and nothing is allocated: the kernel's scratch is a fixed
 * 32.8 KB array in the library's static device memory, which every GPU that
 * loads the library keeps until the process exits.
 *   m, brms: device arrays of n x 3 floats; ms: device array of n floats;
 *   vc: cell volume (m^3); out: host pointer receiving X (J).
 *   stream: cudaStream_t to run on (NULL = the default stream); the call
 *   waits for its own work on that stream and copies X to the host before
 *   returning, so it must not be made while that stream is capturing.
 * Limits and behaviour:
 *   - n <= 16,777,216 cells (4096 chunks of 4096); larger n returns
 *     MMCQ_ERR_UNSUPPORTED without touching the GPU.
 *   - The first call on each device looks up the array's device address
 *     (with that device current).
 *   - Every call shares the one array, so calls whose work overlaps on the GPU
 *     (different streams, threads or processes sharing the context) race and
 *     may return wrong sums; serialise them.
 *   - Errors: MMCQ_ERR_ARG (null pointer, n < 1, vc <= 0), MMCQ_ERR_CUDA. */
int mmcq_coupling_sum_noalloc(const float* m, const float* ms, const float* brms, int64_t n, double vc, double* out,
                              void* stream);

/* ---- groups: several handles stepped as one CUDA graph -----------------
 * A group advances handles of different grids (a sweep over mixed grid
 * sizes) or settings together.  The kernels of every handle for `chunk`
 * steps are captured once into a CUDA graph, each handle on its own branch so
 * that independent handles run concurrently, and the graph is replayed
 * n / chunk times (the remainder is enqueued directly).
 *
 * mmcq_group_step(g, n, dt) has the effect of mmcq_step(h, n, dt) on every
 * handle h of the group: work already queued on a handle's stream comes
 * first, and later calls on that stream see the result.  A handle whose
 * integrator (kind, tolerance, cavity mode) changed since the capture is
 * captured again; while any handle is profiling the group steps the handles
 * one by one without a graph.  MMCQ_ERR_ARG for an empty list, a NULL or
 * repeated handle, handles on different devices, chunk < 1, or RK4 with
 * dt <= 0.  The handles must outlive the group; the group owns its streams,
 * events and graph. */
typedef struct mmcq_group mmcq_group_t;
int mmcq_group_create(mmcq_group_t** g, mmcq_t* const* handles, int n, int chunk);
int mmcq_group_step(mmcq_group_t* g, int64_t n, double dt);
/* graph replays since creation (0 when every step ran without a graph) */
int64_t mmcq_group_replays(const mmcq_group_t* g);
void mmcq_group_destroy(mmcq_group_t* g);
const char* mmcq_group_last_error(const mmcq_group_t* g);

/* ---- autotuning of the launch parameters --------------------------------
 * The paper runs Mumax3's fixed kernels; here the launch shape of each pass of
 * the field evaluation is chosen per grid by timing.  The knobs change no data
 * layout and no arithmetic, so every plan computes the same field:
 *   x_rows         cells rows per block of the x passes (1 .. the rule's count);
 *   col_groups[k]  kx tiles (y passes) or ky columns (z pass) per block of the
 *                  column passes: k = 0 the 2-D convolution, 1 the forward y,
 *                  2 the z pass, 3 the inverse y (0: not launched for this
 *                  grid); a power of two up to the rule's (largest) count;
 *   z_split        pz = 16 or 32: 1 the split z kernel (two threads per
 *                  column), 0 one thread per column (the rule: split for 32,
 *                  one thread for 16); -1: no choice for this grid;
 *   x_pipe         rows of L = 1024 points: 1 the persistent x inverse fed by
 *                  bulk tensor copies, 0 one row per block; -1: no choice;
 *   y_split[k]     y padding 2048 with tiles of 8 columns (k = 0 the forward,
 *                  1 the inverse y pass): 1 each half of the split transform
 *                  in a block of its own (the inverse's two blocks a cluster
 *                  exchanging terms through shared memory), 0 both halves in
 *                  one block; -1: no choice.
 * mmcq_autotune times one middle Runge-Kutta stage of the whole batch (stage
 *   input, transforms, field, torque, coupling sums, per-instance finish) at
 *   the current state under the fixed rules and under each candidate, one knob
 *   at a time with the others at their best so far, with events around every
 *   pass: a candidate is kept when the passes its knob changes (both x passes
 *   for x_rows, the column part for col_groups, the z pass for z_split, the x
 *   inverse for x_pipe, the y pass for y_split) take less time, by the median of `reps` stages.  The
 *   fastest plan stays in use for the later steps of the handle.  Only that stage's scratch buffers are written and the
 *   instance states are restored, so the integration is unchanged.  The choice
 *   is also cached for the process (per device, grid and batch size): a later
 *   handle of the same shape gets it without timing (out->candidates = 0).
 *   Synchronises.
 * mmcq_set_tuning applies a plan (MMCQ_ERR_ARG, nothing changed, if it is not
 *   one of this grid's choices); NULL restores the fixed rules.  A group
 *   holding the handle captures its graph again at its next step. 
 * mmcq_get_tuning reports the plan in use (eval_ms, rule_ms, candidates 0). */
typedef struct {
    int x_rows;
    int col_groups[4];
    int z_split;
    int x_pipe;
    int y_split[2];
    double eval_ms;        /* one stage of the batch with this plan: sum of the passes' median times */
    double rule_ms;        /* the same with the fixed rules */
    int candidates;        /* plans timed (0: taken from the cache) */
} mmcq_tuning;
int mmcq_autotune(mmcq_t* h, int reps, mmcq_tuning* out);
int mmcq_set_tuning(mmcq_t* h, const mmcq_tuning* t);
int mmcq_get_tuning(mmcq_t* h, mmcq_tuning* out);

/* ---- measurement -------------------------------------------------------
 * Per-kernel-class timing of the launches mmcq_step enqueues.  While enabled,
 * each launch is bracketed by two CUDA events on the handle's stream; the
 * record also carries the launch's algorithmic bytes: the compulsory HBM
 * traffic of that pass (every value the pass must read or write once: m,
 * stage torques, spectra rows, one copy of the demag kernel per launch). */
typedef struct {
    char name[24];         /* "x_forward", "conv_2d", "y_forward", "z_convolve", "y_inverse", "x_inverse" */
    int64_t launches;
    double total_ms;       /* summed event-timed durations */
    double bytes;          /* summed algorithmic bytes */
} mmcq_kernel_stat;

/* enable = 1 clears the records and starts recording; 0 stops. */
int mmcq_profile(mmcq_t* h, int enable);
/* Synchronises, then writes up to max per-class totals; *n = classes written. */
int mmcq_profile_read(mmcq_t* h, mmcq_kernel_stat* out, int max, int* n);
/* Kernels launched by mmcq_step since the handle was created (or -1 for a null handle). */
int64_t mmcq_launch_count(const mmcq_t* h);

#ifdef __cplusplus
}
#endif
#endif /* MMCQ_H */
