/*
 * lbm_d2v16.h -- C ABI of the GB300 (sm_103a) library for the D2V16-FFT-TLB thermal
 * liquid-vapour lattice Boltzmann kinetic model of Gan, Xu, Zhang, Wang, Yu and Yang
 * ("Lattice Boltzmann kinetic modeling and simulation of thermal liquid-vapor system").
 *
 * The library advances the 16 discrete distributions f_i of the Kataoka-Tsutahara
 * D2V16 velocity model on a doubly periodic nx x ny grid by the two-stage Runge-Kutta
 * scheme of Sec. 2.3 applied to Eq. (1), with the forcing term I_i of Eq. (2) and
 * spatial derivatives by FFT with the 16th-order modified wavenumber of Eq. (3).
 * All device memory of a simulation is owned by its handle; every host buffer
 * passed in or out is owned by the caller.
 *
 * Layouts. A scalar field is row-major [ny][nx] (x fastest), float64. The 16 distributions
 * are [16][ny][nx]. Velocity i (0-based) is: 0..3 -> (1,0),(0,1),(-1,0),(0,-1);
 * 4..7 -> 6x the same; 8..11 -> (s,s),(-s,s),(-s,-s),(s,-s) with s = 1 (speed sqrt2);
 * 12..15 -> the same with s = 1.5 (speed 3/sqrt2): the Kataoka-Tsutahara speeds 1, 6, sqrt2,
 * 3/sqrt2. eta_i = eta0 on 0..3 and 0 elsewhere (Sec. 2.1).
 *
 * Errors. Every int-returning call returns LBM_OK (0) or a negative LBM_ERR_* code;
 * lbm_strerror() gives a message, lbm_last_error() a detailed one for the calling thread.
 * A call that fails leaves the handle usable unless it returns LBM_ERR_CUDA, after which
 * the CUDA context may be unusable (sticky errors).
 *
 * Streams. All device work of a handle is issued on the stream given to lbm_create
 * (NULL = the legacy default stream). Calls with host buffers synchronise that stream;
 * calls with device buffers are asynchronous on it.
 */
#ifndef LBM_D2V16_H
#define LBM_D2V16_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_ERR_ARG (-1)       /* invalid argument (sizes, params, NULL pointers) */
#define LBM_ERR_NOMEM (-2)     /* device allocation failed */
#define LBM_ERR_CUDA (-3)      /* a CUDA runtime call or kernel launch failed */
#define LBM_ERR_NONFINITE (-4) /* a NaN or Inf was found in the state */
#define LBM_ERR_TIMEOUT (-5)   /* a bounded device-side wait gave up */
#define LBM_ERR_STATE (-6)     /* call out of order (e.g. lbm_step before lbm_init) */
#define LBM_ERR_UNSUPPORTED (-7) /* size or precision not supported by the library */

/* precision of the hot path */
#define LBM_FP64 0   /* every step in float64 (the plain method) */
#define LBM_MIXED 1  /* f storage, all transforms and the update in float32; float64 tables; moment
                        sums of the stored values exact up to one rounding; collision in moment
                        space */
#define LBM_MIXED_RHO64 2 /* LBM_MIXED with the density chain in float64: rho as the float64 sum of
                             the stored distributions, its first and second derivatives by float64
                             transforms, and the van der Waals pressure and the Lambda terms of the
                             macroscopic pass evaluated in float64 */

/* test hooks: switch terms of Eq. (1) off */
#define LBM_FLAG_NO_ADVECTION 1 /* drop v_i . grad f_i */
#define LBM_FLAG_NO_COLLISION 2 /* drop -(f_i - f_i^eq)/tau */
#define LBM_FLAG_NO_FORCE 4     /* drop I_i (and skip the macroscopic derivative chain) */
/* variants */
#define LBM_FLAG_EULER 8        /* forward Euler f^{n+1} = f^n + dt R(f^n) instead of the two-stage
                                   Runge-Kutta scheme (the D2V33 runs' scheme of Sec. 3.2) */
#define LBM_FLAG_ISOTHERMAL 16  /* T = T_iso in f^eq and I_i at every node instead of the temperature
                                   moment (thermostat; mass and momentum stay conserved) */

typedef struct lbm_params {
    double tau;   /* relaxation time (Eq. (1)) */
    double dt;    /* time step of the Runge-Kutta scheme (Sec. 2.3) */
    double dx;    /* grid spacing along x (Eq. (3)) */
    double dy;    /* grid spacing along y */
    double K;     /* surface-tension coefficient (Lambda, C) */
    double H;     /* M = K + H T (Sec. 2.2) */
    double q;     /* heat-flux coefficient of C_q */
    double zeta;  /* bulk viscosity in B and C */
    double b;     /* total degrees of freedom (Sec. 2.1) */
    double eta0;  /* extra-degree-of-freedom parameter of velocities 0..3 (Sec. 2.1: 2.5) */
    double win_alpha; /* window of the windowed FFT: W(m) = exp(-win_alpha (|m|/(N/2))^win_p) */
    double win_p;     /* along each derivative's axis; win_alpha = 0 (default): W = 1, Eq. (3) */
    int precision; /* LBM_FP64, LBM_MIXED or LBM_MIXED_RHO64 */
    int flags;     /* LBM_FLAG_* bits, 0 for the full model */
    double T_iso;  /* temperature of LBM_FLAG_ISOTHERMAL (> 0 when the flag is set) */
    int keff_terms; /* terms of the series of Eq. (3), 1..8: 8 = 16th order (default), 4 = 8th order */
    int reserved;   /* 0 */
    double filter_alpha; /* window of the solution: after every step, f_i <- the inverse transform of */
    double filter_p;     /* W(m_x) W(m_y) times its spectrum, W(m) = exp(-filter_alpha (|m|/(N/2))^filter_p);
                            filter_alpha = 0 (default): no filter */
} lbm_params;

typedef struct lbm_ctx *lbm_handle;

/* Fills *p with the phase-separation set of Sec. 3.2 (tau = dt = 1e-4, dx = dy = 1/256,
 * K = 5e-6, H = 0, zeta = 0) with q = -0.004 and b = 2 (Sec. 3.1), eta0 = 2.5, no window
 * (win_alpha = 0, win_p = 36), FP64, no flags, T_iso = 0, keff_terms = 8, no solution filter
 * (filter_alpha = 0, filter_p = 36). */
void lbm_default_params(lbm_params *p);

/* Creates a simulation on the current CUDA device. nx, ny: powers of two, 2 <= n <= 4096
 * (LBM_ERR_ARG otherwise; LBM_ERR_UNSUPPORTED when the row kernels' shared memory cannot
 * hold a row, e.g. nx = 4096 in LBM_FP64). params is copied. stream: a cudaStream_t or NULL.
 * On success *out owns all device memory of the simulation. */
int lbm_create(int nx, int ny, const lbm_params *params, void *stream, lbm_handle *out);

/* Sets f_i := f_i^eq(rho, u, T) at every node (the initial state of Sec. 3's runs) and
 * resets the step counter. Host buffers, [ny][nx] float64 each; T > 0 and 0 < rho < 3.
 * With LBM_FLAG_ISOTHERMAL the T buffer is checked but T_iso is used. */
int lbm_init(lbm_handle h, const double *rho, const double *ux, const double *uy, const double *T);

/* Same as lbm_init with device buffers (asynchronous on the handle's stream). */
int lbm_init_device(lbm_handle h, const double *rho, const double *ux, const double *uy,
                    const double *T);

/* Advances n >= 0 full Runge-Kutta steps (Sec. 2.3; forward Euler steps with
 * LBM_FLAG_EULER), asynchronously on the stream. */
int lbm_step(lbm_handle h, int n);

/* Moments rho, u_x, u_y, T of the current f (Sec. 2.1) into host buffers [ny][nx].
 * Synchronises the stream. Any pointer may be NULL to skip that field. */
int lbm_moments(lbm_handle h, double *rho, double *ux, double *uy, double *T);

/* Same into device buffers (asynchronous). */
int lbm_moments_device(lbm_handle h, double *rho, double *ux, double *uy, double *T);

/* Copies the 16 distributions to / from host memory, [16][ny][nx] float64. lbm_set_f
 * replaces the state (LBM_MIXED rounds to float32) and resets nothing else. */
int lbm_get_f(lbm_handle h, double *f16);
int lbm_set_f(lbm_handle h, const double *f16);

/* ---- checkpoint and resume ---------------------------------------------------------
 * A state blob holds everything a step reads from the previous one, bit for bit: the 16
 * distributions and the 4 moment fields in the handle's storage precision and device layout,
 * the step counter, and a hash of the parameters, so that k steps, lbm_get_state, then k more
 * steps from lbm_set_state (on the same or another handle of the same size and parameters)
 * give exactly the state of 2k uninterrupted steps. Layout: a 64-byte header
 * {char magic[8] = "LBMSTATE"; uint32 version = 1; int32 nx, ny, precision; int64 steps;
 * uint64 params_hash; uint64 payload_bytes; uint32 element_size; uint32 reserved[3]},
 * then the payload: rows y = 0..ny-1, each the 16 distributions then the moments rho, u_x,
 * u_y, T of that row (nx values each, element_size bytes per value, host byte order). The
 * paper has no counterpart (a library service). */

/* Bytes of the blob of an nx x ny simulation in `precision` (host only; 0 for bad sizes). */
size_t lbm_state_bytes(int nx, int ny, int precision);
/* 64-bit FNV-1a hash of the parameters (every field of lbm_params in order, doubles by their
 * bit patterns; host only, 0 for NULL). */
unsigned long long lbm_params_hash(const lbm_params *params);
/* Writes the current state into the caller's host buffer of `bytes` >= lbm_state_bytes(...)
 * (LBM_ERR_ARG if smaller). Synchronises the stream. */
int lbm_get_state(lbm_handle h, void *blob, size_t bytes);
/* Replaces the state (distributions, moments, step counter) by a blob from lbm_get_state.
 * LBM_ERR_ARG if the blob is short, its header is not a version-1 state, or its size,
 * precision or parameter hash differ from the handle's; nothing is changed then.
 * LBM_ERR_NONFINITE if a value of the payload is not finite. Synchronises the stream. */
int lbm_set_state(lbm_handle h, const void *blob, size_t bytes);

/* Global diagnostics (host out[6]): total mass, x and y momentum, total energy
 * sum(e_T) dx dy with e_T = rho T - 9 rho^2/8 + K |grad rho|^2 / 2 + rho u^2 / 2 (Sec. 2.2),
 * max |u|, and the number of steps taken. Synchronises the stream. */
int lbm_diagnostics(lbm_handle h, double out[6]);

/* lbm_diagnostics in two halves, so that a caller reading the diagnostics of every step does
 * not stall the stream (no counterpart in the paper: a library service). lbm_diagnostics_begin
 * requests the diagnostics of the current state and returns at once; lbm_diagnostics_end
 * waits for the oldest pending request only and reduces it into out[6] (as lbm_diagnostics;
 * out[5] = the step count when it was issued). A request's per-block partial sums come back by
 * an asynchronous copy into a pinned host slot the handle owns (allocated at the first call).
 * For LBM_MIXED handles with the forcing chain on, a request is fused into the next lbm_step:
 * that step's first macroscopic pass, which holds the state's moments and density derivatives,
 * also sums the diagnostics (no launch of their own; their copy runs on a side stream the handle
 * owns, after an event recorded on the handle's stream right after that pass, so the end returns
 * while the rest of the step runs); if no step comes before the end, or the
 * state is replaced first (lbm_init, lbm_set_f, lbm_set_state, lbm_autotune), it is computed
 * on its own then, from the same state. The fused form agrees with lbm_diagnostics to rounding
 * (its d_x rho comes from the pass's own transform: the energy to ~1e-9). Other handles issue
 * the computation at the begin (as lbm_diagnostics, bit for bit). At most two requests may be
 * pending (LBM_ERR_STATE otherwise; also for an end without a request). Typical use: step,
 * begin, end of the previous step's request. An end reports LBM_ERR_TIMEOUT if a bounded device
 * wait gave up before its request. */
int lbm_diagnostics_begin(lbm_handle h);
int lbm_diagnostics_end(lbm_handle h, double out[6]);

/* Circularly averaged structure factor of the density (the domain-growth measure of the
 * phase-separation runs, Sec. 3.2), computed on the device in float64 from the current
 * density: S[b] = mean over shell b of |rho_hat(m)|^2 / (nx ny) for b < nbins (1..8192),
 * rho_hat the unnormalised 2D DFT of rho, shell b = round(|q|) with q = (m_x N/nx, m_y N/ny),
 * N = max(nx, ny), m the signed DFT indices; S[0] (the mean) is reported as 0. count[b]
 * (optional, may be NULL) receives the number of indices in shell b. Host arrays of nbins
 * doubles. Uses the half-step buffer as scratch and a temporary device buffer of
 * (nx + ny) ints + nbins doubles; synchronises the stream. */
int lbm_structure_factor(lbm_handle h, int nbins, double *S, double *count);

/* Waits for all work of the handle; returns LBM_ERR_CUDA if a kernel failed. */
int lbm_synchronize(lbm_handle h);

/* Frees all device memory of the handle (synchronises first). NULL is ignored. */
void lbm_destroy(lbm_handle h);

/* Static message of an error code; lbm_last_error(): last detailed message of this thread. */
const char *lbm_strerror(int code);
const char *lbm_last_error(void);

/* Maxwell construction of the van der Waals fluid P = 3 rho T/(3 - rho) - 9 rho^2/8
 * (Sec. 3.1): coexisting liquid and vapour densities at 0 < T < 1 (host only). */
int lbm_maxwell(double T, double *rho_l, double *rho_v);

/* Per-kernel timing with CUDA events recorded on the handle's stream around every launch
 * while enabled. lbm_timing_read returns, for kernel class k (LBM_K_*), the summed device
 * time in ms and the launch count since the last lbm_timing(h, 1). Reading synchronises. */
#define LBM_K_COL 0    /* column-pass derivative kernels (f and macroscopic fields) */
#define LBM_K_MACRO 1  /* row pass of the macroscopic chain (fluxes, x-derivatives) */
#define LBM_K_FLUX 2   /* column pass of the flux divergences */
#define LBM_K_UPDATE 3 /* fused row pass: x-derivatives of f, f^eq, I_i, BGK, RK stage, moments */
#define LBM_K_RHO64 4  /* LBM_MIXED_RHO64: the float64 density sum and its float64 derivatives */
#define LBM_K_COUNT 5
int lbm_timing(lbm_handle h, int enable);
int lbm_timing_read(lbm_handle h, int kernel, double *ms, long long *launches);

/* Device bytes held by the handle. */
size_t lbm_device_bytes(lbm_handle h);

/* Launch shapes (no counterpart in the paper: a performance service). geometry[0]: width in
 * columns of the column-pass tiles; geometry[1], geometry[2]: rows per CTA of the macro and
 * update row passes; geometry[3]: width of the flux column-pass tiles. lbm_autotune times
 * every legal candidate of each (column tiles with at most 100 KB of line buffers; row CTAs
 * of at most 4096 nodes whose line buffers fit the 227 KB of shared memory a CTA can have)
 * on the handle's own buffers by the time of a whole Runge-Kutta stage, each timed run after
 * an L2 flush (the cold cache a step starts from), one pass's shape at a time, keeps the
 * fastest, and reports the chosen shapes and the stage time with each pass's chosen shape (ms:
 * column, macro, update, flux tuning; either pointer may be NULL). The state is unchanged (the moment fields the
 * update pass rewrites are saved and restored) and results do not depend on the shapes. If it
 * fails midway, the previous shapes and the saved moment fields are put back before it
 * returns the error. Needs an initialised state; allocates temporary device buffers of 4
 * fields and of twice the L2 size (the flush; without it the timings are taken warm);
 * synchronises the stream. */
int lbm_geometry(lbm_handle h, int geometry[4]);
/* The default launch plan of an nx x ny grid in the given precision, computed on the host
 * (no device, no handle): what lbm_create will choose before any tuning, and what each pass
 * needs. out[18] (caller-owned): [0] column tile width, [1] its CTA threads, [2] its shared
 * memory (bytes); [3] macro rows per CTA, [4] macro CTA threads, [5] macro shared memory,
 * [6] 1 if the macro pass transforms a row's two lines in turn; [7] update rows per CTA,
 * [8] update shared memory, [9] 1 if the update takes d_x f from a separate row pass (then
 * [8] is 0); [10] rows per CTA, [11] CTA threads and [12] shared memory of the row-derivative
 * pass; limits: [13] CTA threads of the column and update passes, [14] CTA threads of the
 * macro pass, [15] shared memory per CTA; [16] CTAs per row of the update pass (a cluster of four
 * splits float32 rows of 4096), [17] CTAs per cluster of the column pass. LBM_ERR_ARG for sizes or precision outside the
 * library's range; LBM_ERR_UNSUPPORTED (out filled) if a pass would exceed [15]. */
int lbm_launch_plan(int nx, int ny, int precision, int out[18]);
/* Sets the launch shapes (same meaning as lbm_geometry) to any of the autotuner's legal
 * candidates (LBM_ERR_ARG otherwise); results do not depend on them. Synchronises. */
int lbm_set_geometry(lbm_handle h, const int geometry[4]);
int lbm_autotune(lbm_handle h, int geometry[4], double ms[4]);

/* Form of the passes (no counterpart in the paper: performance choices that do not change any
 * result). kinds[0]: the column pass, kinds[1]: the flux column pass; LBM_COL_DIRECT: each CTA
 * loads its column tile straight from global memory, transforms and stores it (tiles wider
 * than one CTA's threads split every line over a thread-block cluster of 2 or 4 CTAs that
 * exchange points through distributed shared memory); LBM_COL_TMA: a persistent grid whose CTAs
 * stage the next tile in shared memory with tiled bulk tensor copies (TMA) while they transform
 * the current one; LBM_COL_TMA1: the same with one staging buffer per CTA (half the shared
 * memory, so two CTAs per SM where two buffers leave one; a CTA's copy overlaps the other
 * CTAs' transforms instead of its own); LBM_COL_LOOKAHEAD: the direct form, each CTA first issuing bulk L2
 * prefetches of the input rows of the CTA about one wave of resident CTAs after it, so that
 * DRAM streams while the resident CTAs transform. kinds[2]: CTAs per row of the update pass, 1,
 * 2 or 4 (a cluster of two or four splits each row's transforms and node loop; float32 rows of
 * 2048 or more for two, of 4096 for four, one row per cluster). Defaults: LBM_COL_TMA1 for both column passes of LBM_MIXED and
 * LBM_MIXED_RHO64 handles whose columns have 2048 or more points (where the shape allows it),
 * LBM_COL_DIRECT otherwise; 4 CTAs per update row for float32 rows of 4096, 1 otherwise.
 * lbm_autotune chooses them together with the tile widths and rows
 * per CTA. lbm_set_pass_kinds returns LBM_ERR_ARG for a choice the current shapes cannot take
 * (TMA forms and lookahead: rows of fewer than 16 bytes or cluster-split widths; TMA forms:
 * staging buffers beyond a CTA's shared memory); where a launch still cannot use TMA, the
 * direct form runs. */
#define LBM_COL_DIRECT 0
#define LBM_COL_TMA 1
#define LBM_COL_LOOKAHEAD 2
#define LBM_COL_TMA1 3
int lbm_pass_kinds(lbm_handle h, int kinds[3]);
int lbm_set_pass_kinds(lbm_handle h, const int kinds[3]);

/* Fault injection for tests (no counterpart in the paper). Every device-side wait of the
 * library (the TMA column pass waiting for its copies) is bounded by `wait_cycles` clock
 * cycles (<= 0: the default, about one second); a wait that runs out makes its kernel record
 * the failure in the handle's device error word and return, and the next synchronising call
 * (lbm_synchronize, lbm_moments, lbm_get_f, lbm_get_state, lbm_diagnostics) returns
 * LBM_ERR_TIMEOUT once. LBM_FAULT_STARVE_COPIES makes the TMA column pass arm its barriers
 * without issuing the copies, so that its first wait runs out (nothing is copied, nothing
 * faults); LBM_FAULT_NONE restores normal operation. */
#define LBM_FAULT_NONE 0
#define LBM_FAULT_STARVE_COPIES 1
int lbm_fault_inject(lbm_handle h, int what, long long wait_cycles);

/* lbm_diagnostics for callers that cannot allocate device memory. The paper has no
 * counterpart: this is a library service. Examples: host applications or plugins whose GPU
 * memory belongs to another allocator or is budgeted at start-up, and services that must not
 * grow their footprint later. It computes out[5] = total mass, x and y momentum, total energy
 * and max |u| (the quantities of lbm_diagnostics out[0..4]) from the moment fields rho, u_x,
 * u_y, T given as caller-owned float64 device arrays [ny][nx] on the grid nx x ny with
 * spacings dx, dy, surface-tension coefficient K, window (win_alpha, win_p; win_alpha = 0 for
 * none) and keff_terms terms of the series of Eq. (3) (1..8, as lbm_params.keff_terms). out is
 * a caller-owned host array. For a handle's state taken with lbm_moments_device and the
 * handle's own parameters, the result equals lbm_diagnostics to about 1e-12 (relative) for
 * LBM_FP64; for LBM_MIXED, lbm_diagnostics differentiates the float32 density instead, and the
 * energy agrees to about 1e-6 (relative), the other values to about 1e-12.
 * It calls no cudaMalloc, cudaFree or allocating library routine: its scratch (d_x rho,
 * d_y rho, per-block partial sums, derivative tables) is one file-scope device array of
 * about 16.3 MiB, which every GPU that loads this library holds until the process exits; its
 * device address is looked up (cudaGetSymbolAddress) on every call, in the current device's
 * context. Limits: nx, ny powers of two in [2, 4096] and nx * ny <= 1048576 (e.g. 1024 x 1024);
 * larger sizes return LBM_ERR_ARG with the reason in lbm_last_error(). Work is issued on
 * `stream` (a cudaStream_t, NULL = legacy default stream), which the call synchronises before
 * it returns; it also copies its tables from host memory. It therefore must not be called on a
 * stream that is being captured into a CUDA graph: there it returns LBM_ERR_STATE without
 * issuing work (the capture stays valid). Every call rewrites the whole scratch it reads
 * (nothing needs to start at zero), but all calls share the one array: calls that overlap on
 * the GPU (other streams, other host threads) race. */
int lbm_diagnostics_noalloc(int nx, int ny, double dx, double dy, double K, double win_alpha, double win_p,
                            int keff_terms, const double *rho, const double *ux, const double *uy,
                            const double *T, void *stream, double out[5]);

/* ---- batches of independent simulations ------------------------------------------------
 * Many independent runs of Eq. (1) (parameter scans, ensembles over initial states, the
 * coexistence curve of Sec. 3.1 at several temperatures need one run per temperature) are
 * advanced together. Instances of equal grid size are stacked along y in one set of device
 * buffers and advanced by the same launches (the row passes see one nx x (count ny) grid,
 * the column passes take the instance from the grid's z index); groups of different sizes
 * run as parallel branches of one CUDA graph per step. All instances share one lbm_params;
 * every instance is its own doubly periodic domain, bit for bit the run a separate handle
 * of the same size and params would make. */
typedef struct lbm_batch_ctx *lbm_batch;

/* Creates count >= 1 instances, instance k of size nx[k] x ny[k] (powers of two in
 * [2, 4096]; at most 65535 instances of one size and count * ny <= 2^24 per size: else
 * LBM_ERR_ARG). params is copied; stream as in lbm_create. *out owns all device memory. */
int lbm_batch_create(int count, const int *nx, const int *ny, const lbm_params *params, void *stream,
                     lbm_batch *out);

/* Number of instances (0 for NULL). */
int lbm_batch_count(lbm_batch b);

/* lbm_init of instance k (host buffers [ny[k]][nx[k]]); resets that instance's step count. */
int lbm_batch_init(lbm_batch b, int k, const double *rho, const double *ux, const double *uy, const double *T);

/* Advances every instance by n >= 0 Runge-Kutta steps, asynchronously on the stream (one
 * graph launch per step). LBM_ERR_STATE until every instance has been initialised. */
int lbm_batch_step(lbm_batch b, int n);

/* lbm_moments, lbm_get_f and lbm_diagnostics of instance k (host buffers of its size;
 * out[5] of the diagnostics counts the steps since lbm_batch_init(b, k, ...)). Each
 * synchronises the stream. */
int lbm_batch_moments(lbm_batch b, int k, double *rho, double *ux, double *uy, double *T);
int lbm_batch_get_f(lbm_batch b, int k, double *f16);
int lbm_batch_diagnostics(lbm_batch b, int k, double out[6]);

/* lbm_get_state / lbm_set_state of instance k (its own step count). */
int lbm_batch_get_state(lbm_batch b, int k, void *blob, size_t bytes);
int lbm_batch_set_state(lbm_batch b, int k, const void *blob, size_t bytes);

/* lbm_autotune for every size group of the batch (all instances initialised); the launch
 * shapes of instance k's group via lbm_batch_geometry. */
int lbm_batch_autotune(lbm_batch b);
/* lbm_structure_factor of instance k. */
int lbm_batch_structure_factor(lbm_batch b, int k, int nbins, double *S, double *count);
int lbm_batch_geometry(lbm_batch b, int k, int geometry[4]);

/* How lbm_batch_step advances the batch (no counterpart in the paper: a performance choice that
 * does not change any result). LBM_BATCH_GRAPH (the default): one CUDA graph per step whose
 * size groups run as parallel branches of the per-pass kernels. LBM_BATCH_PERSISTENT: one
 * persistent kernel launch per step (captured in a CUDA graph after a reset of its control
 * words) whose CTAs take work items (stage, pass, size group, instance, tile) from a global
 * queue; each item waits, bounded, until every tile of the previous pass of its own instance
 * has completed (per-instance counters), so instances move through the passes independently.
 * The persistent form takes LBM_MIXED batches of at most 4 sizes with nx and ny in 128..1024
 * and flags 0 or LBM_FLAG_ISOTHERMAL (LBM_ERR_UNSUPPORTED otherwise); it allocates its control
 * words (a few ints per instance) on its first step. A wait that runs out (budget: the
 * wait_cycles of lbm_batch_fault_inject, about a second by default) makes every CTA leave the
 * launch; the next lbm_batch_synchronize / lbm_batch_moments / lbm_batch_get_f /
 * lbm_batch_diagnostics / lbm_batch_get_state returns LBM_ERR_TIMEOUT once and the states must be
 * re-initialised. */
#define LBM_BATCH_GRAPH 0
#define LBM_BATCH_PERSISTENT 1
int lbm_batch_set_form(lbm_batch b, int form);
int lbm_batch_form(lbm_batch b); /* -1 for NULL */
/* Waits for all work of the batch; LBM_ERR_TIMEOUT if a bounded device wait gave up. */
int lbm_batch_synchronize(lbm_batch b);
/* Fault injection for tests (no counterpart in the paper): LBM_FAULT_WITHHOLD_COMPLETION makes
 * the persistent kernel's first work item never report its completion, so the items that wait
 * for it run out their budget of wait_cycles clock cycles (<= 0: the default); nothing faults.
 * LBM_FAULT_NONE restores normal operation. */
#define LBM_FAULT_WITHHOLD_COMPLETION 2
int lbm_batch_fault_inject(lbm_batch b, int what, long long wait_cycles);

/* Frees all device memory of the batch (synchronises first). NULL is ignored. */
void lbm_batch_destroy(lbm_batch b);

#ifdef __cplusplus
}
#endif
#endif /* LBM_D2V16_H */
