/*
 * fdlb.h - C ABI of the GB300 (sm_103a) finite-difference lattice Boltzmann (FDLB) solver
 * for the simplified Enskog equation in cylindrical and spherical geometry
 * (S. Busuioc, "Mesoscopic Lattice Boltzmann modeling of dense gas flows in curvilinear
 * geometries", arXiv 2403.15051).
 *
 * The library advances the weighted populations f(R, p_ijk) over all radial cells and all
 * momenta of the mixed half-range x full-range Gauss-Hermite quadrature (Sec. III.A) with
 * the three-stage SSP Runge-Kutta scheme (Sec. III).  Each right-hand-side evaluation is
 *   L(f) = - radial advection (Sec. II.B/C, conservative form, WENO5)
 *          - curvature force in momentum space (Sec. II.B/C with the matrices of Sec. III.B)
 *          - (f - f^S)/tau + J1[f^MB]  (Eqs. j0, j1; Shakhov f^S, Carnahan-Starling chi, Eq. chi,
 *                                       with the Fischer-Methfessel average of Eq. fm)
 * with diffuse-reflection walls on the half-range radial axis at R_L + sigma/2 and
 * R_R - sigma/2 (Sec. IV).
 *
 * Conventions
 *  - Units: m = k_B = 1; momenta in units of sqrt(T_ref), T_ref = 1.
 *  - Every call returns FDLB_OK (0) or an error code; no exception crosses the ABI.
 *  - Device state is owned by the library (or carved from a caller workspace, see
 *    fdlb_create_in).  Output buffers are owned by the caller.
 *  - Population layout seen through the ABI (fdlb_get_f / fdlb_set_f / fdlb_eval_rhs):
 *    host FP64 array [cell][i][j][k], i over the 2 Q_R radial momenta (positive half first,
 *    each half in ascending |p|), j over the Q_2 nodes of the second axis (ascending), k over
 *    the Q_3 nodes of the third axis (ascending).  Axes: cylinder (R, phi, z), sphere
 *    (r, theta, phi).  The values are weighted populations f_ijk = w_i w_j w_k f(p)/omega^3
 *    (Sec. III.A), so plain sums give moments.
 *  - Moments are always returned in FP64, in both precision modes.
 *  - All device work is issued on the stream given at creation; calls that return host data
 *    synchronise that stream.
 */
#ifndef FDLB_H
#define FDLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------------- status codes */
#define FDLB_OK 0
#define FDLB_EINVAL 1          /* invalid argument or parameter set                     */
#define FDLB_ECUDA 2           /* a CUDA runtime call failed                            */
#define FDLB_ENOMEM 3          /* device or host allocation failed / workspace too small */
#define FDLB_ENOTCONVERGED 4   /* run_to_steady hit max_steps                           */
#define FDLB_ETIMEOUT 5        /* run_to_steady hit max_seconds, or a device wait gave up */
#define FDLB_ENAN 6            /* non-finite moments detected                           */
#define FDLB_EIO 7             /* checkpoint file could not be read or written          */
#define FDLB_ENOGPU 8          /* no usable CUDA device                                 */

/* ----------------------------------------------------------------------- enumerations */
#define FDLB_CYL 0             /* coaxial cylinders, axes (R, phi, z)  (Sec. II.B)        */
#define FDLB_SPH 1             /* concentric spheres, axes (r, theta, phi)  (Sec. II.C)   */
#define FDLB_CYL_Z 2           /* coaxial cylinders with p_z integrated out (the trivial axis of
                                  Sec. III.A's remark on Couette flow): per (p_R, p_phi) node the
                                  pair phi = int f dp_z, chi = int p_z^2 f dp_z, stored as k = 0, 1
                                  of the third index (Q_3 must be 0; n_momenta = 2 x 2Q_R x Q_2);
                                  for states even in p_z it evolves the p_z-projection of FDLB_CYL */
#define FDLB_FP64 0            /* populations and arithmetic in FP64                      */
#define FDLB_FP32 1            /* FP32 populations and streaming, FP64 moment sums         */
#define FDLB_CHI_RET_FM 0      /* chi_SET at the Fischer-Methfessel density (Eqs. chi_ret, fm) */
#define FDLB_CHI_SET_LOCAL 1   /* chi_SET at the local density (Eq. chi)                   */

#define FDLB_QUAD_FULL 0       /* full-range Gauss-Hermite, Q nodes (Sec. III.A)           */
#define FDLB_QUAD_HALF 1       /* half-range Gauss-Hermite, 2Q nodes (Sec. III.A)          */

#define FDLB_NMOM 9            /* per-cell moments: n, u_1, u_2, u_3, T, q_1, q_2, q_3, P_12 */

/* ----------------------------------------------------------------------- parameters */
typedef struct fdlb_params {
    int geometry;          /* FDLB_CYL, FDLB_SPH or FDLB_CYL_Z                             */
    double R_in, R_out;    /* physical wall radii, R_out > R_in > 0 (Sec. IV)              */
    int n_cells;           /* radial cells on [R_in + sigma/2, R_out - sigma/2], >= 8       */
    double stretch_beta;   /* 0: uniform cells; > 0: tanh map with this beta (finer at walls) */
    int Q_R, Q_2, Q_3;     /* half-range order on the radial axis (2 Q_R nodes), 1 <= Q_R <= 100
                              (the paper's runs use 20, 60 and 100, Sec. IV); full-range
                              orders on the two homogeneous axes, 1 <= Q_2, Q_3 <= 24       */
    int N_R, N_2, N_3;     /* equilibrium expansion orders (Sec. III.C), 0 <= N < Q;
                              negative: min(Q - 1, 7)                                      */
    double eta0;           /* mean reduced density eta0 = pi sigma^3 n0 / 6, in (0, 0.5)    */
    double Kn;             /* Knudsen number; sets C by Kn = 1/(6 sqrt2 eta0 chi(eta0) C)
                              (Sec. II) when sigma <= 0                                    */
    double sigma;          /* molecular diameter; > 0 overrides Kn                         */
    int chi_model;         /* FDLB_CHI_RET_FM or FDLB_CHI_SET_LOCAL                         */
    int precision;         /* FDLB_FP64 or FDLB_FP32                                       */
    double dt;             /* > 0: fixed time step; <= 0: min(cfl dR_min/(max|p_R| sqrt(T_max)),
                              tau_min/2) at the mean state                                 */
    double cfl;            /* CFL number when dt <= 0; <= 0 selects 0.4                    */
    double T_wall[2];      /* wall temperatures, inner [0] and outer [1], > 0              */
    double u_wall[2];      /* tangential wall speeds along the second axis (cylinder only) */
} fdlb_params;

/* Read-only facts about one instance, filled by fdlb_get_info. */
typedef struct fdlb_info {
    double C;              /* confinement ratio L / sigma                                  */
    double sigma, n0;      /* molecular diameter and mean number density                   */
    double dt;             /* time step in use                                             */
    double R_first, R_last;/* computational domain [R_L^c, R_R^c]                          */
    int n_cells;
    int n_momenta;         /* 2 Q_R Q_2 Q_3                                                */
    int fm_band;           /* width of the stored Fischer-Methfessel band (cells)          */
    int precision;
    int64_t step;          /* RK3 steps taken since the last init                          */
} fdlb_info;

typedef struct fdlb_solver* fdlb_handle;

/* ----------------------------------------------------------------------- lifecycle */

/* Build one solver instance: quadrature, derivative matrices, equilibrium tables, grid and
 * FM weights on the host (Secs. III.A-C, App. A), then device state.  `cuda_stream` is a
 * cudaStream_t; NULL makes the handle create (and later destroy) a private blocking stream, so
 * that the step can be captured into a CUDA graph.  The state is left at the uniform equilibrium
 * (fdlb_init_uniform with defaults).  Errors: FDLB_EINVAL for a parameter outside the ranges
 * above, C = L/sigma < 3, or a Fischer-Methfessel band (cells x stored band width) of more than
 * 2^31 - 1 entries; FDLB_ENOMEM when the host set-up runs out of memory; FDLB_ENOGPU /
 * FDLB_ECUDA / FDLB_ENOMEM from the device. */
int fdlb_create(const fdlb_params* p, void* cuda_stream, fdlb_handle* out);

/* Many independent instances advanced together by one set of launches (the batched sweep):
 * all instances share the geometry kind, Q_R, Q_2, Q_3, the expansion orders and the
 * precision; everything else (size, radii, Kn, eta0, walls, dt) may differ.  Instance ids are
 * 0..n_instances-1 in the order given.  Errors as fdlb_create, and FDLB_EINVAL when the batch's
 * total cells, work items or stored FM band entries exceed 2^31 - 1 (the device tables index
 * them with 32-bit integers; about 5000 instances of 1024 stretched cells reach the band limit). */
int fdlb_batch_create(const fdlb_params* ps, int n_instances, void* cuda_stream, fdlb_handle* out);

/* Device bytes needed by fdlb_create_in for these instances. */
int fdlb_workspace_bytes(const fdlb_params* ps, int n_instances, size_t* bytes);

/* As fdlb_batch_create, but all device state lives in the caller's device buffer
 * `workspace` (at least fdlb_workspace_bytes, 256-byte aligned); the library allocates
 * no device memory of its own and the buffer must outlive the handle. */
int fdlb_create_in(const fdlb_params* ps, int n_instances, void* cuda_stream, void* workspace,
                   size_t workspace_bytes, fdlb_handle* out);

void fdlb_destroy(fdlb_handle h);

/* ----------------------------------------------------------------------- set-up calls */

/* Diffuse-reflection wall (Sec. IV): side 0 = inner, 1 = outer; temperature T_w > 0 and
 * tangential speed along the second axis (must be 0 for the sphere).  Takes effect at the
 * next step. */
int fdlb_set_wall(fdlb_handle h, int instance, int side, double T_w, double u_tangential);

/* Uniform equilibrium n0 g_R(0,T0) g_2(0,T0) g_3(0,T0) (Sec. III.C); n0 <= 0 selects the
 * instance's mean density, T0 <= 0 the mean wall temperature.  instance < 0: all. */
int fdlb_init_uniform(fdlb_handle h, int instance, double n0, double T0);

/* Warm start from moment profiles given at n_points >= 2 equally spaced points of the
 * normalised radius x = (R - R_L^c)/(R_R^c - R_L^c) in [0, 1] (host arrays): n, u_2 (second
 * axis velocity), T and the radial heat flux q_R, linearly interpolated onto the cells.
 * f = n g_R(0,T) g_2(u_2,T) g_3(0,T) [1 + (xi^2/(5T) - 1) xi_R q_R/(n T^2)]  (the Shakhov
 * factor of Sec. II with 1 - Pr set to 1). */
int fdlb_init_from_moments(fdlb_handle h, int instance, const double* n, const double* u2,
                           const double* T, const double* qR, int n_points);

/* Replace / read the populations of one instance: host FP64 [cell][i][j][k] (see layout). */
int fdlb_set_f(fdlb_handle h, int instance, const double* f_host);
int fdlb_get_f(fdlb_handle h, int instance, double* f_host);

/* ----------------------------------------------------------------------- time stepping */

/* Advance all active instances by n_steps SSP-RK3 steps (asynchronous on the stream;
 * repeated blocks of steps are replayed from a captured CUDA graph). */
int fdlb_step(fdlb_handle h, int64_t n_steps);

/* Step until the moment residual r <= tol for every instance (checked every `check_every`
 * steps; r = max over n, u_2, T, q_R of max_cells |M(t+K dt) - M(t)| / (K max(max|M(t)|,
 * scale)), scales n0, 1, T0, n0 T0^1.5), or max_steps / max_seconds is reached.  In a batch,
 * converged instances stop stepping; so do instances whose moments become non-finite (residual
 * +inf; the others run on) and, with fdlb_set_stall_checks, instances whose residual has stopped
 * falling.  steps_taken (per instance, may be NULL) and residual (per instance, may be NULL) are
 * host arrays of length n_instances.  Returns FDLB_OK (every instance converged), else FDLB_ENAN
 * if an instance became non-finite, else FDLB_ETIMEOUT or FDLB_ENOTCONVERGED. */
int fdlb_run_to_steady(fdlb_handle h, double tol, int64_t max_steps, double max_seconds,
                       int check_every, int64_t* steps_taken, double* residual);

/* Stall rule of fdlb_run_to_steady (and of both phases of fdlb_run_to_steady_mixed): an instance
 * whose residual has not fallen below half of its lowest value for `checks` consecutive checks
 * stops stepping, unconverged (it has settled on a small self-sustained oscillation of the
 * residual instead of a steady state, as some instances of the discretised problem do; in a batch
 * it would otherwise keep the whole run going to max_steps).  0 (default): never.  FDLB_EINVAL
 * for checks < 0. */
int fdlb_set_stall_checks(fdlb_handle h, int checks);

/* Steady state at the FP64 level of accuracy for an FP32 handle: the FP32 form runs to the
 * residual tolerance (as fdlb_run_to_steady; its steady state sits on the FP32 rounding floor,
 * ~1e-5 to 1e-4 of the moment scales from the FP64 one for dense, small-Kn instances), then an FP64
 * copy of the handle (the same instances, walls and time step) continues from that state, scaled
 * per instance to the total mass the call started with (the walls conserve mass and the steady
 * state depends on it; FP32 rounding walks it by up to ~1e-9 per step), to the tolerance, and
 * the polished state, rounded to FP32, replaces the handle's populations (its
 * moments are the FP64 steady state's to FP32 rounding; stepping on in FP32 drifts back to the
 * floor).  The FP64 copy lives in `fp64_workspace` (fdlb_polish_workspace_bytes bytes, 256-byte
 * aligned) when given, else in device memory the call allocates and frees.  steps_fp32 /
 * steps_fp64 / residual: per-instance host arrays (may be NULL); residual is the FP64 phase's.
 * The step counts of the handle grow by the FP64 steps.  For an FP64 handle it is
 * fdlb_run_to_steady.  Returns as fdlb_run_to_steady for the FP64 phase, FDLB_ENAN if either
 * phase met non-finite moments (an error of the FP32 phase other than ENOTCONVERGED / ETIMEOUT /
 * ENAN is returned at once).  The paper's method is
 * precision-agnostic; this two-precision schedule is a library service. */
int fdlb_run_to_steady_mixed(fdlb_handle h, double tol, int64_t max_steps, double max_seconds, int check_every,
                             void* fp64_workspace, size_t fp64_workspace_bytes, int64_t* steps_fp32,
                             int64_t* steps_fp64, double* residual);
int fdlb_polish_workspace_bytes(fdlb_handle h, size_t* bytes);

/* Evaluate L(f) of the current state of one instance without advancing it (Secs. II-III);
 * host FP64 [cell][i][j][k]. */
int fdlb_eval_rhs(fdlb_handle h, int instance, double* L_host);

/* ----------------------------------------------------------------------- outputs */

/* Per-cell moments of one instance (Eq. macro_def from the quadrature sums of Eq. mom_quad):
 * out[cell][FDLB_NMOM] = n, u_1, u_2, u_3, T, q_1, q_2, q_3, P_12 (P_12 = shear stress between
 * the radial and second axis), FP64.  instance -1: every instance at once, [total cells][FDLB_NMOM]
 * with the cells of instance q after those of instances 0..q-1.  on_device != 0: `out` is a device
 * pointer, written asynchronously on the stream; else a host pointer (the call synchronises). */
int fdlb_get_moments(fdlb_handle h, int instance, double* out, int on_device);

/* Closure diagnostics of the current state of one instance, host FP64 arrays of n_cells
 * (any may be NULL): the Fischer-Methfessel density nbar (Eq. fm), chi (Eq. chi), tau
 * (Eq. tau); and the two wall densities n_w (inner, outer) of the diffuse walls. */
int fdlb_get_closure(fdlb_handle h, int instance, double* nbar, double* chi, double* tau,
                     double* n_wall2);

/* One SSP-RK3 step of every active instance, reporting per instance the relative L2 change of the
 * populations, rel_change[q] = ||f^{n+1} - f^n||_2 / ||f^n||_2 summed in FP64 (a host array of
 * n_instances; inactive instances report 0): the per-step change of f itself, beside the moment
 * residual of fdlb_run_to_steady.  Keeps a copy of the state in device memory it allocates and frees
 * (the size of the populations); synchronises the stream.  Returns FDLB_OK, FDLB_EINVAL, FDLB_ENOMEM
 * or FDLB_ECUDA. */
int fdlb_step_change(fdlb_handle h, double* rel_change);

/* Total mass sum_c V_c n_c (FP64), the last residual and the step count of one instance. */
int fdlb_get_diagnostics(fdlb_handle h, int instance, double* total_mass, double* residual,
                         int64_t* step);

int fdlb_get_info(fdlb_handle h, int instance, fdlb_info* out);

/* Checkpoint: step count, parameters, populations (native precision) and their FP64 raw
 * moment sums of all instances; restoring it continues the run bit for bit. */
int fdlb_save(fdlb_handle h, const char* path);
/* Restore a checkpoint written by fdlb_save for a handle created with the same parameters;
 * FDLB_EINVAL if they differ, FDLB_EIO on a read error.  Under another momentum slicing
 * (fdlb_set_tiling) the sums are recomputed instead: the same moments up to rounding order. */
int fdlb_load(fdlb_handle h, const char* path);

const char* fdlb_error_string(int code);

/* Kernel-tuning knobs of the streaming kernel (cells per tile, p_3 values per momentum slice,
 * threads per block); 0 keeps the current value.  A change of the cells per tile alone regroups
 * cells without changing any result; the slice width and the block size change the order of the
 * moment sums (results then agree to rounding).  For the 16 x 8 x 8 FP32 cylinder a block of at
 * most 128 threads selects the row kernel (a whole p_2 row of 8 momenta per thread), the default
 * for handles of more than 64 cells per SM.
 *
 * fdlb_autotune times candidate tile shapes on the device and keeps the fastest: the cells per
 * stream tile (2 .. 32) under each register bound of the stage kernel that is built for the shape
 * (the compiled arithmetic is the same), then the closure's form and its own cells per item (2, 4,
 * 8, 16), each candidate over three stages written to the stage-1 scratch buffers (the state, its
 * sums and the step count are not touched).  Only these regrouping knobs are searched, so a tuned
 * handle produces the same results bit for bit as an untuned one.  The choice is cached per process for the momentum set,
 * precision, block size, slice width and size class (log2 of the handle's cells and instances);
 * fdlb_autotune always measures and refreshes that cache.  fdlb_set_autotune selects automatic
 * tuning at the first fdlb_step / fdlb_run_to_steady of a handle, from the cache when it holds
 * the handle's key: 0 off, 1 batches of two or more instances (default), 2 every handle.
 * fdlb_get_tiling reports the tiling in use (any pointer may be NULL). */
int fdlb_set_tiling(fdlb_handle h, int cells_per_tile, int slice_k, int threads);
int fdlb_autotune(fdlb_handle h, int* cells_per_tile, int* slice_k, int* threads);
int fdlb_set_autotune(fdlb_handle h, int mode);
int fdlb_get_tiling(fdlb_handle h, int* cells_per_tile, int* slice_k, int* threads, int* closure_cells);

/* The stage kernel in use: momenta per thread vector (vector_width), vectors per thread, and the
 * blocks per SM its register allocation is bounded for (1: none beyond the 512-thread bound).  Any
 * pointer may be NULL. */
int fdlb_get_stage_kernel(fdlb_handle h, int* vector_width, int* vectors_per_thread, int* min_blocks);

/* Pins the register bound of the stage kernel (the choice fdlb_autotune makes among the variants
 * built for the shape): min_blocks 1 (none beyond the 512-thread bound), or 2, 3, 5 where built
 * (the 16 x 8 x 8 FP32 cylinder: 3 for blocks of up to 256 threads, 2, 3 and 5 for the row
 * kernel).  The arithmetic and its order are the same in all, so results do not change by a bit.
 * min_blocks -1 changes nothing.  *in_use (may be NULL) = the bound in use.  FDLB_EINVAL for a
 * bound not built for the handle's shape (the handle keeps its previous one). */
int fdlb_set_stage_min_blocks(fdlb_handle h, int min_blocks, int* in_use);

/* The K^h contraction of the curvature force on the tensor cores (default off): an
 * nR x nR by nR x (n2 KS) product per cell in split TF32 (K = Kh + Kl, f = fh + fl; three
 * TF32 products with FP32 accumulation, FP32-level accuracy) with mma.sync m16n8k8, for FP32
 * populations on the 16 x 8 x 8 and 24 x 12 x 12 quadratures; elsewhere the CUDA-core path
 * stays.  *in_use (may be NULL) tells whether it applies to this handle.  On GB300 these
 * contractions are too small to pay for the splitting: the default is the CUDA-core path. */
int fdlb_set_tensor_contraction(fdlb_handle h, int enable, int* in_use);

/* Whole SSP-RK3 steps in one persistent launch (default off): each block owns tiles of cells
 * for the launch and runs, per stage, the closure of its own cells into shared memory and the
 * stage, with a grid-wide barrier between stages (cooperative launch, every wait bounded: a
 * barrier that does not complete within 1 s sets the error flag, reported as FDLB_ETIMEOUT by
 * fdlb_get_diagnostics).  The results are those of the closure and stage kernels, bit for bit.
 * It applies to the 16 x 8 x 8 and 24 x 12 x 12 quadratures with one momentum slice when the
 * grid fits on the device at once; elsewhere, and in kernel-timing mode, the two launches per
 * stage stay.  enable < 0 only reports; *in_use (may be NULL) tells whether it applies to this
 * handle.  This scheduling is an implementation choice of this library; the paper describes the
 * method, not launches. */
int fdlb_set_persistent_step(fdlb_handle h, int enable, int* in_use);

/* Test hooks of the bounded device waits (both 0 in use).  tx_extra_bytes (0..65536): every
 * staged copy of the stage kernel waits for that many bytes more than it copies, so its bounded
 * wait on the copy barrier runs out; barrier_extra (0..65536): every grid barrier of the
 * persistent step kernel waits for that many arrivals more than the grid makes, so its 1 s wait
 * runs out.  In both cases the blocks set the error flag and leave without faulting: the next
 * fdlb_get_diagnostics returns FDLB_ETIMEOUT and the state of the interrupted step is
 * undefined.  fdlb_clear_error clears the flag (the handle stays usable; set a state again).
 * The same holds after a wait that runs out in use (FDLB_ETIMEOUT from fdlb_get_diagnostics
 * without a test hook): a block that gives up leaves while a copy into its shared memory may
 * still be in flight, so the populations, sums and records of the interrupted step are
 * undefined; restore a checkpoint (fdlb_load) or set a new state before stepping on. */
int fdlb_set_wait_test(fdlb_handle h, int tx_extra_bytes, int barrier_extra);
int fdlb_clear_error(fdlb_handle h);

/* Programmatic dependent launch of the closure and stage kernels (default on): each may start
 * while its predecessor in the stream finishes, loading its constant tables, and waits for the
 * predecessor's completion before it reads anything the predecessor writes.  Results are the same
 * bit for bit either way; 0 turns it off (ordinary stream-ordered launches). */
int fdlb_set_programmatic_launch(fdlb_handle h, int enable);

/* Own cells per closure work item of the chain form (1..28; default 2 on the cylinder, 4 on the
 * sphere, 8 where items outnumber the co-resident blocks several times over).  A closure item also
 * recomputes the macroscopic fields of two stencil cells on each side, so larger items repeat less
 * work and smaller items spread the latency-bound closure over more SMs.  Selects the chain form.
 * FDLB_EINVAL outside the range. */
int fdlb_set_closure_cells(fdlb_handle h, int cells);

/* Form of the closure (Eqs. fm, chi, j1, tau, prandtl and the equilibria of Sec. III.C, once per
 * stage).  form 0, the chain: one launch, each block runs an item of a few cells through the whole
 * closure (short, latency-bound: one instance).  form 1, the batch form: two launches over items
 * of 28 cells, the first giving every FM band row a warp of its own (the band sum, chi), the
 * second forming the records of each item from the raw sums of its reach and the band results
 * (throughput-bound: batches and long instances; the default when the items of 28 cells are more
 * than four times the SM count).  The records are the same bit for bit either way.
 * form -1 changes nothing.  *in_use (may be NULL) = the form in use.  FDLB_EINVAL for another
 * form. */
int fdlb_set_closure_form(fdlb_handle h, int form, int* in_use);

/* Number of kernel launches issued by the last fdlb_step call (for launch accounting). */
int64_t fdlb_launch_count(fdlb_handle h);

/* SSP-RK3 steps per captured CUDA graph replayed by fdlb_step (1..1000, default 20). */
int fdlb_set_graph_steps(fdlb_handle h, int steps);

/* Per-kernel timing.  When on, fdlb_step launches the kernels directly (no graph) and brackets
 * every closure and streaming launch with CUDA events on the solver's stream; fdlb_kernel_times
 * returns the accumulated durations (ms) and launch counts since the last call and clears them.
 * Where the persistent step kernel is in use (fdlb_set_persistent_step), its launches are timed
 * instead and fdlb_step_kernel_times returns their accumulated duration (ms), the number of
 * launches and the steps they ran.  Any output pointer may be NULL. */
int fdlb_set_kernel_timing(fdlb_handle h, int on);
int fdlb_step_kernel_times(fdlb_handle h, double* ms, int64_t* launches, int64_t* steps);
int fdlb_kernel_times(fdlb_handle h, double* stream_ms, int64_t* n_stream, double* closure_ms,
                      int64_t* n_closure);

/* The cudaStream_t the solver issues its work on (the one given at creation, or a private
 * blocking stream when NULL was given). */
int fdlb_get_stream(fdlb_handle h, void** stream);

/* Populations of one instance in the library's own layout and precision: [cell][k][i][j]
 * (k outermost inside a cell), n_cells * n_momenta elements of FP32 (FDLB_FP32) or FP64.
 * instance -1: the whole batch as the library stores it, fdlb_state_bytes bytes (each instance's
 * populations start on a 256-byte boundary, the gaps between them carry no data), in one copy.
 * on_device != 0: `src`/`dst` is a device pointer; else host (pinned memory gives the fastest
 * copies).  fdlb_set_state_raw also recomputes the quadrature sums of the new state (one pass
 * over every instance) and resets the step counts of the instances it sets. */
int fdlb_set_state_raw(fdlb_handle h, int instance, const void* src, int on_device);
int fdlb_get_state_raw(fdlb_handle h, int instance, void* dst, int on_device);
int fdlb_state_bytes(fdlb_handle h, size_t* bytes);

/* ----------------------------------------------------------------------- learned warm start
 * A one-dimensional Fourier neural operator that maps the five parameters of a cylindrical
 * instance (Kn, eta0, radius ratio R_out/R_in, inner wall speed, wall temperature ratio
 * T_out/T_in) to its steady moment profiles on n_points equally spaced points of the normalised
 * radius x = (R - R_L^c)/(R_R^c - R_L^c); the profiles seed a Shakhov-type warm start
 * (fdlb_init_from_moments).  The paper has no network: this is a library service, trained on the
 * solver's own steady states.  Architecture: input channels = 5 normalised parameters + x; lift
 * to `width`; `layers` Fourier layers v <- GELU(v W + b + G R F v) keeping `modes` modes; GELU
 * hidden layer of `hidden`; 4 outputs.  BF16 weights in every product, FP32 accumulation and
 * activations, FP32 master weights with Adam (beta1 0.9, beta2 0.999).
 * Output channels (normalised): o0 = n/n0 - 1, o1 = u_2/0.1, o2 = (T/T_in - 1)/0.1,
 * o3 = q_R/(0.01 n0 T_in^1.5).  Raw parameters are float[batch][5] in the order above; targets
 * and outputs float[batch][n_points][4].  The parameter vector is float[n] in the layout
 * lift W [6][width], lift b; per layer R_re [modes][width][width], R_im, W [width][width], b;
 * P1 [width][hidden], c1; P2 [hidden][4], c2. */
typedef struct fdlb_nn* fdlb_nn_handle;
int fdlb_nn_create(int width, int modes, int layers, int hidden, int n_points, int max_batch, void* cuda_stream,
                   fdlb_nn_handle* out);
void fdlb_nn_destroy(fdlb_nn_handle h);
int fdlb_nn_num_params(fdlb_nn_handle h, int64_t* count);
int fdlb_nn_set_params(fdlb_nn_handle h, const float* theta_host);   /* also resets Adam */
/* Seeded initialisation: weight matrices U(-1, 1)/sqrt(fan_in), spectral weights U(0, 1)/width^2,
 * biases 0 (splitmix64 stream); also resets Adam. */
int fdlb_nn_init_params(fdlb_nn_handle h, uint64_t seed);
int fdlb_nn_get_params(fdlb_nn_handle h, float* theta_host);
int fdlb_nn_forward(fdlb_nn_handle h, const float* raw_params_host, int batch, float* out_host);
/* MSE loss mean((out - target)^2) and its gradient with respect to every parameter. */
int fdlb_nn_loss_grad(fdlb_nn_handle h, const float* raw_params_host, const float* targets_host, int batch,
                      float* loss, float* grad_host);
/* One Adam step on one batch (forward, backward, update); returns the batch loss. */
int fdlb_nn_train_step(fdlb_nn_handle h, const float* raw_params_host, const float* targets_host, int batch,
                       float lr, float* loss);
/* Predict the profiles of one instance of `solver` from its parameters and seed its state with
 * them (decode the outputs as above, then fdlb_init_from_moments).  The density and heat-flux
 * profiles are rescaled together so that the seed carries the instance's total mass (that of its
 * uniform start): the walls conserve mass, so the steady state depends on it.  The solver's
 * stream is synchronised (two mass reads). */
int fdlb_nn_warm_start(fdlb_nn_handle h, fdlb_handle solver, int instance, const float* raw_params_host);

/* ----------------------------------------------------------------------- no device allocation
 * Per-cell moments of populations the caller already holds on the device, for callers that
 * cannot allocate device memory: plugins inside an application that owns the whole device
 * budget, and latency-critical loops that cannot afford cudaMalloc's implicit synchronisation.
 * The paper has no counterpart: this is a library service.
 *
 * f_dev: device array of n_cells * 2Q_R * Q_2 * Q_3 populations in the library's own layout
 * ([cell][k][i][j], as fdlb_get_state_raw writes it), FP32 or FP64 per `precision`.
 * nodes_host: host array [2Q_R radial nodes | Q_2 nodes | Q_3 nodes] as fdlb_quadrature returns
 * them; it is copied to the device with cudaMemcpyAsync on `cuda_stream`, in stream order: from
 * pageable memory the call returns once the copy has been staged (the buffer may be reused at
 * once), from pinned memory the buffer must stay valid until the copy has run on the stream.
 * moments_dev: device array [n_cells][FDLB_NMOM] (n, u_1..3, T, q_1..3, P_12), FP64.
 * Work is issued on `cuda_stream` (a cudaStream_t; NULL = legacy stream), asynchronously.
 *
 * Allocates no device memory: the partial sums live in a fixed scratch array of this library
 * (3.4 MB, held by every GPU that loads the library until the process exits), so n_cells is
 * limited to 32768 (FDLB_EINVAL beyond).  The first call on a device looks up the scratch
 * address (cudaGetSymbolAddress, once per device, serialised across host threads); make that
 * first call before any stream capture on that device.  Every call shares the one scratch
 * array, which keeps the last call's contents; calls that overlap on the GPU (different streams,
 * no ordering) race on it and must be serialised by the caller.  A launch error of this call is
 * reported as FDLB_ECUDA; errors left by earlier, unrelated work are neither reported nor
 * cleared.  Returns FDLB_OK, FDLB_EINVAL, FDLB_ENOGPU or FDLB_ECUDA. */
int fdlb_moments_noalloc(int precision, int Q_R, int Q_2, int Q_3, const double* nodes_host, int n_cells,
                         const void* f_dev, double* moments_dev, void* cuda_stream);

/* ----------------------------------------------------------------------- device probe
 * Measured FP32 fused multiply-add rate of the current device, the denominator of the fused stage
 * kernel's arithmetic roofline (the paper has no counterpart: a measurement service).  A kernel of
 * independent FMA chains fills every SM; one warm-up launch, then `repeats` launches timed with
 * CUDA events on `cuda_stream` (a cudaStream_t; NULL = legacy stream).  *tflops = the best rate
 * (an FMA counted as two flops), *ms = that launch's duration.  Synchronises the stream.  Returns
 * FDLB_OK, FDLB_EINVAL (repeats < 1, null outputs), FDLB_ENOGPU or FDLB_ECUDA. */
int fdlb_fp32_fma_peak(void* cuda_stream, int repeats, double* tflops, double* ms);

/* ----------------------------------------------------------------------- host-only set-up
 * These run on the host only (no GPU needed). */

/* Quadrature rule of Sec. III.A.  kind FDLB_QUAD_FULL: Q nodes ascending, weights summing
 * to 1.  FDLB_QUAD_HALF: 2Q nodes, positive half first in ascending order, then their mirror
 * images; weights sum to 1 (1/2 per half).  nodes/weights: host arrays of Q or 2Q. */
int fdlb_quadrature(int kind, int Q, double* nodes, double* weights);

/* Momentum-derivative matrix of Sec. III.B acting on weighted populations, row-major:
 * FDLB_QUAD_HALF: (d f/dp) on the half-range axis, 2Q x 2Q (Eq. force1, half range);
 * FDLB_QUAD_FULL: (d (f p)/dp) on a full-range axis, Q x Q (Eq. force2, full range). */
int fdlb_derivative_matrix(int kind, int Q, double* K);

/* Confinement ratio, molecular diameter and mean density from (Kn, eta0, L) (Sec. II). */
int fdlb_physical_parameters(double Kn, double eta0, double L, double* C, double* sigma, double* n0);

/* Grid of the computational domain (Sec. IV): cell-centre radii R_c[n_cells], face radii
 * R_f[n_cells+1], cell volumes V[n_cells] and curvature factors kappa[n_cells] (any may be NULL). */
int fdlb_grid(int geometry, double R_in, double R_out, double sigma, int n_cells, double beta,
              double* R_c, double* R_f, double* V, double* kappa);

/* Fischer-Methfessel weights (Eq. fm, App. A) as a dense row-major n_cells x n_cells matrix:
 * nbar_i = sum_j W[i][j] n_j with n = 0 outside the computational domain.  FDLB_EINVAL for the
 * arguments fdlb_grid rejects or a band of more than 2^31 - 1 entries, as fdlb_create. */
int fdlb_fm_weights(int geometry, double R_in, double R_out, double sigma, int n_cells,
                    double beta, double* W);

#ifdef __cplusplus
}
#endif
#endif /* FDLB_H */
