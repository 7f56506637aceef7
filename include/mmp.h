/*
 * mmp.h -- C-ABI of the GB300 micromagnetic field/torque library (libmmp.so).
 *
 * One context (`mmp_ctx`) holds one magnet on a regular grid of nx*ny*nz
 * cuboid cells of size cx*cy*cz (metres) with one or two sublattices, its
 * material parameters, its state and its solver.  This follows the problem
 * statement of arXiv 2411.18194, Methods: the unit magnetisation of each
 * magnet evolves as dm/dt = tau (Eq. magnetic-dynamic-equation), with the LLG torque of
 * Eq. (LLG_torque), the effective-field terms listed after it (external,
 * uniaxial anisotropy, exchange, demagnetising, DMI, magnetoelastic), the
 * antiferromagnetic exchange of Eq. (AFM_exchange_field), the elastodynamics
 * of Eq. (elasticity) and the embedded Runge-Kutta solvers of the solver
 * table (Dormand-Prince RK45 here).
 *
 * Conventions shared by every call
 *   - Units: SI.  Fields in tesla, magnetisation in A/m, time in seconds.
 *   - Vector fields are SoA float32 [3][nz][ny][nx] (x fastest); cell index
 *     c = x + nx*(y + ny*z).
 *   - Pointers to vector fields may be host or device pointers (the library
 *     copies with cudaMemcpyDefault on the context's stream).  The caller
 *     owns every pointer it passes; the library owns everything it
 *     allocates.  The library allocates device memory through the caller's
 *     allocator when one is given at creation, else with cudaMalloc.
 *   - All device work is enqueued on the context's stream.  Calls that
 *     return host values, or read/write host buffers, synchronise that
 *     stream before returning.
 *   - Errors: a negative status; mmp_last_error() gives a message (thread
 *     local).  After MMP_E_CUDA the context is poisoned and later calls
 *     return MMP_E_STATE.  Unsupported requests fail with MMP_E_INVAL; the
 *     library never falls back to another code path.
 *   - One context must be used by one host thread at a time.
 *   - The demag kernel spectrum (the FFT of -mu0 N, FP32, about 4 * 6 *
 *     (nz + 1) / nz bytes per cell) is built on the first evaluation and
 *     shared by every context of the process with the same extents and
 *     cell size on the same device: it is library-owned cudaMalloc memory
 *     (not taken through the context allocator), freed with the last such
 *     context.
 */
#ifndef MMP_H
#define MMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MMP_VERSION 2

typedef struct mmp_ctx mmp_ctx;

enum mmp_status {
    MMP_OK = 0,
    MMP_E_INVAL = -1,      /* bad argument or unsupported configuration */
    MMP_E_OOM = -2,        /* device allocation failed */
    MMP_E_CUDA = -3,       /* a CUDA call failed; the context is poisoned */
    MMP_E_NONFINITE = -4,  /* a NaN/Inf appeared; the step was rolled back */
    MMP_E_TIMEOUT = -5,    /* a host-side deadline passed */
    MMP_E_STATE = -6,      /* context poisoned or call out of order */
    MMP_E_BOUNDS = -7      /* bounds-checked build only (compiled with -DMMP_CHECK_BOUNDS, loaded
                            * by the binding when MMP_CHECK_BOUNDS=1): a kernel's index check
                            * found an access outside its buffer (the access was skipped); the
                            * context is poisoned */
};

/* Per-sublattice, per-region scalar parameters (mmp_set_param). */
enum mmp_param {
    MMP_MS = 0,     /* saturation magnetisation Ms (A/m); Ms = 0 marks an empty cell */
    MMP_AEX = 1,    /* ferromagnetic exchange stiffness A11 (J/m) */
    MMP_ALPHA = 2,  /* Gilbert damping */
    MMP_KU1 = 3,    /* first uniaxial anisotropy constant along ANIS_U (J/m^3) */
    MMP_KU2 = 4,    /* second-order uniaxial constant along ANIS_U (J/m^3) */
    MMP_KB1 = 5,    /* second uniaxial constant along ANIS_UB (J/m^3) */
    MMP_DIND = 6,   /* interfacial DMI strength D (J/m^2) */
    MMP_B1 = 7,     /* first magnetoelastic coupling constant (J/m^3) */
    MMP_B2 = 8,     /* second magnetoelastic coupling constant (J/m^3) */
    MMP_KC1 = 9,    /* cubic anisotropy constant (J/m^3) along the axes ANIS_C1, ANIS_C2 */
    MMP_NPARAM = 10
};

/* Per-sublattice, per-region vector parameters (mmp_set_param3). */
enum mmp_param3 {
    MMP_ANIS_U = 0,   /* uniaxial axis of KU1/KU2 (normalised by the library) */
    MMP_ANIS_UB = 1,  /* uniaxial axis of KB1 (normalised by the library) */
    MMP_B_EXT = 2,    /* external field (T) */
    MMP_ANIS_C1 = 3,  /* first cubic axis (normalised; default x) */
    MMP_ANIS_C2 = 4,  /* second cubic axis (made orthogonal to C1 and normalised; default y);
                         the third is C1 x C2 */
    MMP_NPARAM3 = 5
};

/* Global constants (mmp_set_global). */
enum mmp_global {
    MMP_A0 = 0,         /* homogeneous AFM exchange A0 (J/m), Eq. AFM_exchange_field */
    MMP_A12 = 1,        /* inhomogeneous AFM exchange A12 (J/m) */
    MMP_LATTICE_A = 2,  /* lattice parameter a (m) */
    MMP_C11 = 3,        /* cubic stiffness c11 (Pa) */
    MMP_C12 = 4,        /* cubic stiffness c12 (Pa) */
    MMP_C44 = 5,        /* cubic stiffness c44 (Pa) */
    MMP_RHO = 6,        /* mass density (kg/m^3) */
    MMP_ETA = 7,        /* viscous (Rayleigh stiffness) damping time (s) */
    MMP_NGLOBAL = 8
};

/* Field terms (mmp_enable_terms bitmask). */
enum mmp_term {
    MMP_T_DEMAG = 1,     /* FFT demag of M = sum_s Ms m (Methods, Magnetostatic field) */
    MMP_T_EXCH = 2,      /* 6-neighbour exchange (first term of Eq. AFM_exchange_field) */
    MMP_T_ANIS = 4,      /* uniaxial anisotropy (KU1, KU2 along ANIS_U; KB1 along ANIS_UB) */
    MMP_T_DMI = 8,       /* interfacial DMI (Eq. dmi, interfacial tensor) with the boundary
                            condition of mmp_set_boundary */
    MMP_T_ZEEMAN = 16,   /* external field B_EXT */
    MMP_T_AFM = 32,      /* A12 and A0 terms of Eq. AFM_exchange_field (2 sublattices) */
    MMP_T_MEL = 64,      /* magnetoelastic field/force (Eqs. magnetoelastic-field/-force) */
    MMP_T_ELASTIC = 128, /* elastodynamics rho u'' = f_tot (Eq. elasticity) */
    MMP_T_CUBIC = 256    /* cubic anisotropy: energy Kc1 (a^2 b^2 + a^2 c^2 + b^2 c^2), a, b, c the
                            components of m on the cubic axes (the paper's "uniaxial or cubic"
                            anisotropy, as in mumax3) */
};

/* Boundary condition of the exchange and DMI stencils at the magnet's surface
 * (grid edges and faces towards empty cells); Methods, DMI and boundary
 * conditions, which names Neumann (default), open and periodic conditions. */
enum mmp_bc {
    MMP_BC_NEUMANN = 0,  /* a missing neighbour takes the ghost value m + Delta_n d_n m with
                            d_n m = -(D/2A)(z x n) x m (Eq. AFM_Neumann_BC, A12 = 0); zero-Neumann
                            without DMI */
    MMP_BC_OPEN = 1      /* a missing neighbour drops out of the exchange and DMI sums (no
                            boundary twist): the field is the exact negative gradient of the
                            pair energy.  Without DMI it equals the Neumann field. */
};

/* Embedded Runge-Kutta solvers of the paper's table (Methods): convergence
 * order / error-estimate order.  The higher-order solution is propagated;
 * every step ends with an evaluation at the renormalised solution, which is
 * the next step's first stage (free for the FSAL methods DP45 and BS23). */
enum mmp_method {
    MMP_DP45 = 0,      /* Dormand-Prince 5 / 4, 6 evaluations per step */
    MMP_HEUN = 1,      /* Heun 2 / Euler 1, 2 evaluations per step */
    MMP_BS23 = 2,      /* Bogacki-Shampine 3 / 2, 3 evaluations per step */
    MMP_CASHKARP = 3,  /* Cash-Karp 5 / 4, 6 evaluations per step */
    MMP_RKF45 = 4      /* Fehlberg 5 / 4, 6 evaluations per step */
};

typedef void* (*mmp_alloc_fn)(size_t bytes, void* user);
typedef void (*mmp_free_fn)(void* ptr, void* user);

/* Create a context.  nx, ny, nz >= 1 (padded FFT lengths are at most 4096
 * per axis; nz <= 16 when the demag term is on); cx, cy, cz > 0 (m);
 * n_sublattices 1 or 2; `stream` is a cudaStream_t (NULL = legacy default
 * stream); `alloc`/`dealloc`/`user` an optional device allocator (both or
 * neither).  On success *out owns the context.  Errors: MMP_E_INVAL,
 * MMP_E_OOM, MMP_E_CUDA (e.g. no GPU). */
int mmp_create(mmp_ctx** out, int nx, int ny, int nz, double cx, double cy, double cz,
               int n_sublattices, void* stream, mmp_alloc_fn alloc, mmp_free_fn dealloc,
               void* user);

/* Destroy a context and free everything it allocated (NULL is allowed). */
int mmp_destroy(mmp_ctx* ctx);

/* Region map: nx*ny*nz uint8 (host or device pointer), region r selects
 * row r of every parameter table.  Default: all cells in region 0. */
int mmp_set_region_map(mmp_ctx* ctx, const uint8_t* regions);

/* Set a scalar (mmp_set_param) or vector (mmp_set_param3) parameter of
 * sublattice `sub` (-1 = all) in `region` (0..255, -1 = all). */
int mmp_set_param(mmp_ctx* ctx, int sub, int param, int region, double value);
int mmp_set_param3(mmp_ctx* ctx, int sub, int param, int region, double x, double y, double z);
int mmp_set_global(mmp_ctx* ctx, int param, double value);

/* Select the boundary condition (mmp_bc; default MMP_BC_NEUMANN).  Periodic
 * conditions are not supported (MMP_E_INVAL). */
int mmp_set_boundary(mmp_ctx* ctx, int bc);

/* Select the field terms (bitmask of mmp_term).  Two-sublattice contexts
 * with DMI, the magnetoelastic term without the elastic term, and the
 * elastic/magnetoelastic terms with empty cells are rejected (MMP_E_INVAL
 * at the next evaluation). */
int mmp_enable_terms(mmp_ctx* ctx, unsigned terms);

/* State.  m: [3][nz][ny][nx] float32 of sublattice `sub`; with normalize != 0
 * each vector is scaled to unit length on the device.  u, v: elastic
 * displacement (m) and velocity (m/s), same layout.  Setting the state
 * invalidates the cached first Runge-Kutta stage. */
int mmp_set_m(mmp_ctx* ctx, int sub, const float* m, int normalize);
int mmp_get_m(mmp_ctx* ctx, int sub, float* m);
int mmp_set_elastic(mmp_ctx* ctx, const float* u, const float* v);
int mmp_get_elastic(mmp_ctx* ctx, float* u, float* v);

/* Solver.  method: an mmp_method.  adaptive = 0: fixed step dt.  adaptive =
 * 1: dt is the initial step, tol the absolute max-norm tolerance on the
 * error estimate dt*max|sum_i (b_i - b*_i) k_i| of m, dt in [dt_min,
 * dt_max], step factor 0.9 (tol/err)^(1/(q+1)) in [0.2, 5] with q the
 * method's error-estimate order. */
int mmp_set_solver(mmp_ctx* ctx, int method, int adaptive, double dt, double tol,
                   double dt_min, double dt_max);

/* Evaluate B_eff and the LLG torque of sublattice `sub` at the current state
 * (one field evaluation).  B (T) and tau = dm/dt (1/s) are
 * [3][nz][ny][nx] float32, host or device, either may be NULL. */
int mmp_eval_field(mmp_ctx* ctx, int sub, float* B, float* tau);

/* Advance nsteps steps (fixed or adaptive; an adaptive step reads the
 * 4-byte error estimate back once per attempt).  Fixed steps run in pairs
 * from a CUDA graph captured on a private stream (ordered with the
 * context's stream by events; re-captured after any change it depends on),
 * bitwise equal to single steps.  Returns MMP_E_NONFINITE (state rolled back
 * to the last accepted step) if the error is NaN/Inf. */
int mmp_step(mmp_ctx* ctx, int nsteps);

/* Advance by `duration` seconds (the last step is shortened to land on time). */
int mmp_run(mmp_ctx* ctx, double duration);

/* Relax: damping-only torque -gamma alpha/(1+alpha^2) m x (m x B), adaptive
 * DP45, until max|m x B| <= torque_tol_T (tesla), or simulated time
 * max_time, or host wall time timeout_s (then MMP_E_TIMEOUT). */
int mmp_relax(mmp_ctx* ctx, double torque_tol_T, double max_time, double timeout_s);

/* Time, step size and counters (field evaluations, accepted and rejected
 * steps) since creation. */
int mmp_get_time(mmp_ctx* ctx, double* t, double* dt, long long* steps,
                 long long* rejected, long long* evals);

/* Energy of every field term at the current state, in J:
 * e_terms[i] for the term with bit (1 << i) of mmp_term (0 for terms that
 * are off), MMP_NTERMS entries.  Exchange, DMI and the intersublattice
 * exchange over pairs of neighbouring magnetic cells; demag -1/2 sum M.B dV;
 * anisotropy, cubic, Zeeman and magnetoelastic densities; elastic strain plus
 * kinetic energy.  (The fields are minus the gradients of these energies,
 * Methods, Micromagnetism.)  One extra demag-only evaluation when the demag
 * term is on (not counted as a solver evaluation).  Synchronises. */
#define MMP_NTERMS 9
int mmp_energy(mmp_ctx* ctx, double* e_terms);

/* Checkpoint: serialise (size query with blob = NULL) / restore the state
 * (m of every sublattice, u, v, t, dt, counters) to/from a host blob.  A
 * restored run continues bitwise identically on the same device. */
int mmp_get_state(mmp_ctx* ctx, void* blob, size_t* size);
int mmp_set_state(mmp_ctx* ctx, const void* blob, size_t size);

/* Tracing: with enable != 0, every kernel launch of the context is bracketed
 * by CUDA events on the context's stream (counters reset); enable = 0 stops
 * recording.  mmp_profile_read synchronises the stream and returns, for
 * kernel `kernel` (an mmp_kernel), the number of launches and their summed
 * device time since the last reset. */
enum mmp_kernel {
    MMP_K_PASS_A = 0,     /* stage assembly + forward x FFT */
    MMP_K_PASS_B = 1,     /* y FFT, z transform, kernel multiply, inverse y/z */
    MMP_K_FIELD = 2,      /* inverse x FFT + local field + LLG torque (+ error) */
    MMP_K_ASSEMBLE = 3,   /* stage assembly without demag */
    MMP_K_STRAIN = 4,     /* strain and stress */
    MMP_K_ELASTIC = 5,    /* elastic + magnetoelastic force */
    MMP_NKERNEL = 6
};
int mmp_profile(mmp_ctx* ctx, int enable);
int mmp_profile_read(mmp_ctx* ctx, int kernel, long long* launches, double* total_ms);

/* Demagnetising field without any device allocation (the paper has no
 * counterpart; it exists for callers that cannot call cudaMalloc, e.g. code
 * whose device memory is owned by a host framework, or a loop that must not
 * allocate once running).
 *   B = -mu0 N * M on an nx*ny*nz grid of cx*cy*cz cells (same tensor, FFT
 *   passes and kernels as the context path), M in A/m and B in tesla, both
 *   caller-owned device float32 [3][nz][ny][nx]; work is enqueued on
 *   `stream` (cudaStream_t, NULL = legacy default stream).
 * All working memory is one file-scope static device array of
 * MMP_NOALLOC_SCRATCH_BYTES (32 MiB) that every GPU loading the library holds
 * until exit.  Grids needing more (roughly above 2e5 cells) are rejected with
 * MMP_E_INVAL and a message giving the size.  The first call on a device,
 * and the first call after the geometry (extents or cell size) changes,
 * sets the array up: it looks up the array's device address, copies tables
 * from the host, builds the demag kernel and synchronises the stream -- make
 * that first call before any stream capture.  All calls share the array and
 * it keeps the last call's contents (the kernel of the last geometry); calls
 * that overlap on the GPU, or run concurrently on two host threads with
 * different geometries, race on it. */
#define MMP_NOALLOC_SCRATCH_BYTES (32 * 1024 * 1024)
int mmp_demag_noalloc(int nx, int ny, int nz, double cx, double cy, double cz, const float* M, float* B,
                      void* stream);

/* ---------------------------------------------------------------------
 * Launch shape and autotuning (no counterpart in the paper: how the FFT
 * passes of Methods, Magnetostatic field are laid out on the GPU).
 * --------------------------------------------------------------------- */
typedef struct mmp_shape {
    int ty;            /* rows (y) per tile of pass A (stage assembly + forward x FFT): 2, 4 or 8 */
    int radix_x;       /* x FFT plan: 0 = radix-16 passes first, 1 = radix-8 passes */
    int radix_y;       /* plan of the y FFT of pass B (length Py/R), same choices */
    int R;             /* ky residue classes = CTAs per pass-B cluster: 1, 2, 4 or 8 */
    int stage_kernel;  /* 1: pass B stages its slice of the kernel octant in shared memory */
    int tyc;           /* rows per tile of pass C (inverse x FFT + field): 2, 4, 8, or 0 = the
                          default (ty, fewer when a block cannot hold its row pairs) */
    int engine;        /* FFT engine, bit mask (0 = the block-wide Stockham passes, any
                          supported grid):
                          MMP_ENGINE_WARP_B: pass B on warp-level transforms (one warp
                          per column, in-register DFTs and one shared-memory transpose;
                          folded y length Py/R of 256, 512 or 1024, ny <= Py/R, R of 1
                          or 2, nz of 1, 2, 4 or 8); radix_y and stage_kernel do not
                          apply to it;
                          MMP_ENGINE_WARP_X: passes A and C on warp-level transforms in
                          tiles of one row pair (Px = 2048, i.e. nx of 769 .. 1024);
                          ty, tyc and radix_x do not apply to them;
                          MMP_ENGINE_TC_Y (with MMP_ENGINE_WARP_B): the final length-32
                          DFT of every y transform of pass B as a dense GEMM on the
                          tensor cores in split TF32 (each product as three TF32
                          products, FP32 accumulation in tensor memory).  A device-side
                          wait of it that runs past its limit makes the next
                          synchronising call return MMP_E_TIMEOUT. */
} mmp_shape;
#define MMP_ENGINE_WARP_B 1
#define MMP_ENGINE_WARP_X 2
#define MMP_ENGINE_TC_Y 4

/* Current shape of the context (chosen at creation: ty from the grid, the
 * radix-16 plans; the warp passes where they apply (pass B with R = 2 when
 * Py = 2048 and R = 1 below), else the smallest R that fits the block pass
 * B with stage_kernel = 1). */
int mmp_get_shape(mmp_ctx* ctx, mmp_shape* out);

/* Set a shape.  MMP_E_INVAL (context unchanged) if it does not fit the grid
 * (shared memory above 227 KB, FFT capacity, R not dividing Py).  The plans
 * change the FP32 rounding order of the transforms, so the cached first
 * Runge-Kutta stage is dropped; results agree to FP32 rounding. */
int mmp_set_shape(mmp_ctx* ctx, const mmp_shape* shape);

#define MMP_TUNE_BATCH 1   /* only shapes a batch runs (R = 1, stage_kernel = 0, engine = 0), 8-row tiles */
#define MMP_TUNE_FORCE 2   /* time again even if this geometry was tuned before */
/* Time the valid shapes on the context's current state and keep the
 * fastest: after a warm-up of ~100 ms of evaluations (loaded clocks), the
 * candidates of passes A+C (tile rows, x plan) and of pass B (R, staging,
 * y plan, block or warp engine) are timed separately in two interleaved rounds (CUDA events per
 * pass on the context's stream, the better round counts); the combination
 * replaces the starting shape only if a longer interleaved measurement
 * finds it > 2 % faster per evaluation.  Returns the shape (chosen, may be
 * NULL) and its time per field evaluation in ms (eval_ms, may be NULL).
 * Results are cached per (grid, sublattices, flags) in the process; a
 * cached geometry is set without timing unless MMP_TUNE_FORCE.
 * Synchronises the stream. */
int mmp_autotune(mmp_ctx* ctx, int flags, mmp_shape* chosen, double* eval_ms);

/* ---------------------------------------------------------------------
 * Batches: independent contexts advanced together (no counterpart in the
 * paper, which runs one simulation at a time).  In every Dormand-Prince
 * stage each of the three demag passes of all active members is launched
 * once per (z group, block-size class) over a work list of (member, tile)
 * items, one block per item, longest first; the launches of a pass run
 * concurrently on side streams and stream order carries the dependencies
 * between passes (there is no device-side wait).  Lock steps of
 * fixed-step members are replayed from a CUDA graph.  A member runs
 * exactly the arithmetic of its own context
 * (same plans and coefficients), so its results are bitwise those of
 * mmp_step / mmp_run / mmp_relax on the same context with the same shape.
 *
 * Members: one sublattice, one region (no region map), the demag term on,
 * no AFM / magnetoelastic / elastic terms, and either the shape R = 1,
 * stage_kernel = 0, engine = 0 (mmp_set_shape or mmp_autotune with
 * MMP_TUNE_BATCH first; such members share work-list launches), or the warp
 * passes MMP_ENGINE_WARP_B | MMP_ENGINE_WARP_X with Py / R = 1024 and
 * stage_kernel = 0 (the creation default of grids with nx of 769 .. 1024 and
 * ny of 385 .. 512 or 769 .. 1024; such a member gets one launch per pass of
 * its own); otherwise MMP_E_INVAL.  The batch borrows its members: while a context is a member
 * it must not be used elsewhere, and it must be removed before it is
 * destroyed.  Between mmp_batch_advance calls every member's state sits in
 * its context as usual (mmp_get_m, mmp_get_time work).  All work runs on
 * the batch's stream; the calls synchronise it before returning.
 * --------------------------------------------------------------------- */
typedef struct mmp_batch mmp_batch;

enum mmp_goal {
    MMP_GOAL_STEPS = 0,  /* a = number of accepted steps (fixed or adaptive per the member's solver) */
    MMP_GOAL_RUN = 1,    /* a = duration (s); the last step lands on time */
    MMP_GOAL_RELAX = 2   /* a = torque tolerance (T), c = max simulated time (s); as mmp_relax */
};

/* `stream`: the cudaStream_t all batch work runs on; NULL (the legacy
 * default stream, on which graphs cannot be captured) makes the batch
 * create and own a non-blocking stream. */
int mmp_batch_create(mmp_batch** out, void* stream);
/* Destroys the batch, not its members. */
int mmp_batch_destroy(mmp_batch* b);
/* Add a member with its goal (counted from its current time / steps). */
int mmp_batch_add(mmp_batch* b, mmp_ctx* ctx, int goal, double a, double c);
int mmp_batch_remove(mmp_batch* b, mmp_ctx* ctx);
int mmp_batch_size(mmp_batch* b, int* n);
/* Run up to max_attempts lock-step attempts; a member stops taking part
 * once its goal is reached.  Adaptive or relaxing members read their
 * error estimates back once per lock step (one synchronisation for the
 * whole batch).  n_active (may be NULL) receives the members not done. */
int mmp_batch_advance(mmp_batch* b, int max_attempts, int* n_active);
/* done: goal reached (or failed); status: MMP_OK or the member's error
 * (MMP_E_NONFINITE: its state is the last accepted one). */
int mmp_batch_status(mmp_batch* b, mmp_ctx* ctx, int* done, int* status);
/* Kernel launches the batch has made (tracing). */
int mmp_batch_launches(mmp_batch* b, long long* n);
/* Tracing: with enable != 0 (counters reset) every pass launch is bracketed
 * by CUDA events and fixed-step lock steps launch directly instead of
 * through the graph; mmp_batch_profile_read returns, for pass 0 (A: stage
 * assembly + forward x FFT), 1 (B: y/z transforms + kernel multiply, all z
 * groups) or 2 (C: inverse x FFT + field + torque), the launches and their
 * summed device time since the reset.  Both synchronise the batch stream. */
int mmp_batch_profile(mmp_batch* b, int enable);
int mmp_batch_profile_read(mmp_batch* b, int pass, long long* launches, double* total_ms);

/* Wait for all work of the context. */
int mmp_sync(mmp_ctx* ctx);

/* Measured FP32 FMA throughput of the current device (no counterpart in the
 * paper: the arithmetic ceiling the passes' FP32 rate is reported against).
 * Runs `reps` launches of a kernel of eight independent FMA chains per
 * thread at full occupancy on `stream` (cudaStream_t as void*, NULL = the
 * default stream), each timed with CUDA events; returns the best launch as
 * GFLOP/s (2 flops per FMA) and its time in ms (may be NULL).  Allocates
 * and frees 1.2 MB of device memory; synchronises the stream. */
int mmp_fp32_peak(void* stream, int reps, double* gflops, double* ms_per_launch);

/* Message of the last error on this thread ("" if none). */
const char* mmp_last_error(void);

/* MMP_VERSION of the library. */
int mmp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MMP_H */
