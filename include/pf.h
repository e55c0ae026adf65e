/*
 * pf.h -- C ABI of libpf, a GB300 (sm_103a) engine for one explicit time step
 * of the obstacle-potential multi-phase-field model coupled to a KKS
 * concentration field, and for the explicit integrators compared by
 * M. Seiz and T. Takaki, "Numerical efficiency of explicit time integrators
 * for phase-field models", arXiv 2601.16522 (cited below as "the paper").
 *
 * Conventions for every entry point:
 *  - Every call returns an int status (pf_status).  Nothing throws or aborts
 *    across the ABI; pf_strerror() gives a short text.
 *  - The caller owns every pointer it passes; the library copies what it needs
 *    (set/get) and owns its device buffers, which live until pf_destroy().
 *  - Work is ordered on the CUDA stream given to pf_create (NULL: the legacy
 *    default stream).  A handle is not thread-safe; distinct handles are
 *    independent.  All device memory of a handle belongs to the device that
 *    was current at pf_create and that device must be current at every call.
 *  - Field layout at the ABI ("phase-major"): a state holds
 *    phi[a * V + i] for phases a = 0..N-1 and, when has_conc = 1, the
 *    concentration c[i], with i = (z * ny + y) * nx + x (x fastest),
 *    V = nx * ny * nz.  Values cross the ABI as double; in precision 32 the
 *    library converts on the way in and out.
 *  - ptr_is_device: 0 = host pointers (pageable or pinned; the call copies and
 *    synchronises the stream before returning), 1 = device pointers on the
 *    handle's device (stream-ordered, no synchronisation).
 */
#ifndef PF_H
#define PF_H
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum {
    PF_OK = 0,
    PF_EINVAL = 1,      /* invalid argument or unsupported combination            */
    PF_ENOMEM = 2,      /* device or host allocation failed                         */
    PF_EUNSTABLE = 3,   /* NaN/Inf error norm, non-positive simplex sum, or too
                           many rejected steps; the last accepted state is kept  */
    PF_ETIMEOUT = 4,    /* a bounded device wait gave up                            */
    PF_EDEVICE = 5,     /* a CUDA call failed (launch, copy, no device)             */
    PF_ESTATE = 6       /* no state has been set yet                                */
} pf_status;

/* Integrators of Sec. 3.2: forward Euler, SSP(s)2 and SSP(10)4 (Ketcheson
   2008, the low-storage forms with one extra buffer), and the
   Runge-Kutta-Legendre super-time-stepping schemes of order 1 and 2
   (Eq. sts with Legendre coefficients of Meyer et al. 2012/2014). */
typedef enum { PF_FEULER = 0, PF_SSP2 = 1, PF_SSP104 = 2, PF_RKL1 = 3, PF_RKL2 = 4 } pf_integrator;

/* Boundary conditions per face (Sec. 4: periodic by default; Sec. 5.2.2:
   zero-gradient phase field and Dirichlet concentration).  A periodic face
   requires its opposite face to be periodic for both phi and c. */
typedef enum { PF_BC_PERIODIC = 0, PF_BC_NEUMANN = 1, PF_BC_DIRICHLET = 2 } pf_bc;

/* Problem description (Sec. 2 model, Sec. 3 discretisation).  All arrays are
   read during pf_create only. */
typedef struct {
    int dim;                  /* 2 or 3 */
    int nx, ny, nz;           /* cells; nz = 1 when dim = 2 */
    double dx;                /* grid spacing */
    int n_phases;             /* N >= 2 phases stored densely.  Up to 12 nontrivial phases
                                 (the n(phi) filter of Eq. phieq) per cell take the fast
                                 per-cell list; a cell with more is recomputed on a slower
                                 path with a 64-entry list (same results); more than 64
                                 nontrivial phases in one cell is reported as PF_EINVAL by
                                 the call that meets it. */
    const int *phase_type;    /* N entries, chemical type 0 (alpha) or 1 (beta), Sec. 2 */
    const double *gamma;      /* N*N interface energies gamma_ab, symmetric (diag ignored) */
    const double *mobility;   /* N*N interface mobilities M_ab, symmetric (diag ignored) */
    double W;                 /* interface parameter, interface width pi*W (Eq. profile) */
    const double *L_override; /* NULL: L_ab = pi M_ab / (4 W) (Sec. 2); else N*N phase-field
                                 mobilities (e.g. Eq. thin-interface) */
    int has_conc;             /* K: 0 or 1 concentration field (Eq. ceq) */
    double k[2], c0[2], D[2]; /* per chemical type: k_t, c_{0,t} (Eq. gibbs-energy), D_t (Eq. ceq) */
    int bc_phi[6];            /* pf_bc per face x-, x+, y-, y+, z-, z+ (periodic or Neumann) */
    int bc_c[6];              /* pf_bc per face for c (periodic, Neumann or Dirichlet) */
    double c_dirichlet[6];    /* Dirichlet value of c per face */
    int precision;            /* 64: FP64 storage and arithmetic; 32: FP32 storage and stencil
                                 arithmetic, FP64 time, coefficients and reductions.  Every
                                 stage rounds each stored value once (combinations are affine,
                                 increments summed first), so sum c dV drifts by at most 2^-24
                                 of sum |c - c_ref| dV per stage */
    int options;              /* bit set of PF_OPT_* (0: defaults) */
    double c_ref;             /* FP32 storage only: c is kept as c - c_ref, so values near c_ref
                                 keep FP32's relative resolution and small per-stage changes are
                                 not rounded away (choose the concentration of the phase that fills
                                 most of the domain; 0 stores c itself).  Results are the same up to
                                 rounding; ignored for precision 64; must be finite. */
} pf_params;

/* pf_params.options: PF_OPT_TMA runs the FP32 3D passes (5..32 phases, nx a
   multiple of 32, ny a multiple of 8) through the warp-specialised kernel
   that streams phase planes into shared memory with TMA bulk tensor copies
   instead of the plain-load kernel.  Results are bit-identical; which is
   faster depends on the problem (on the 256^3, 32-phase grain workload the
   plain-load kernel is). */
/* PF_OPT_MASKED (FP32, at most 128 phases) selects masked storage, the
   GPU form of the per-cell phase lists of Sec. 3.1 (only the N_z local
   phases are loaded): the state keeps its dense phase-major layout and adds
   one 32-bit occupancy word per 32 phases and cell (bit b of word w set
   where phase 32 w + b may be nonzero; every entry whose bit is clear holds
   zero).  The FP32 fast passes
   skip the loads and the work of phases that are zero at a cell, its face
   neighbours and the pass's pointwise inputs; their RHS and stage values are
   exactly zero, so results equal the dense passes' up to the sign of zero.
   Every pass of every integrator has a masked form (SSP(10)4 included: its
   embedded accumulator and its mid-stage combination keep masks of their
   own); the pf_rhs pass runs dense.  The masks cost
   4 bytes per word, cell and state vector (pf_footprint counts them); TMA
   staging is not used.  PF_EINVAL for FP64. */
/* PF_OPT_ONE_CELL (FP32 dense storage) runs the passes through the kernel
   with one cell per thread and stage values held in registers (N <= 32; the
   chunked form for more phases) instead of the default kernel with two
   x-adjacent cells per thread (float2 loads and stores, stage values written
   through; used where nx is even).  Results agree to FP32 rounding; meant for
   comparison and tuning (pf_autotune picks per problem shape). */
/* PF_OPT_MOBILITY_SIMPLEX replaces the standard projection S after every
   stage (clamp, >= 1 rule, divide by the sum; Sec. 3.1) by a
   mobility-weighted one, a reading of the mobility-based simplex Sec. 3.1
   cites for the particle cases of Sec. 5.3 (the paper does not describe
   it): on the phases with a positive value at the cell, P, the point of the
   simplex face spanned by P nearest to the stage value in the metric
   sum (x_a - y_a)^2 / w_a, with w_a the mean phase-field mobility L_ab of
   phase a towards the other phases of P; so x_a = max(y_a - tau w_a, 0) with
   tau fixing the sum to 1, and a phase that moves slowly against its
   neighbours (an immobile particle) takes little of the correction.  With
   equal mobilities this is the Euclidean projection.  Runs on the generic
   passes (both precisions); PF_EINVAL with PF_OPT_MASKED, and pf_step
   returns PF_EINVAL for PF_STEP_REUSE_RHS and PF_STEP_DEVICE_LOOP; more than
   64 positive phases in one cell is PF_EINVAL from the call that meets it. */
/* PF_OPT_SLOTS (FP32, up to 32768 phases) selects slot storage, the per-cell
   phase records of Sec. 3.1: every cell holds at most N_p = 12 phase values
   with their phase ids (ascending, 16-bit), whatever the number of phases
   N, so a state vector costs 12 x 6 bytes (+ 4 for c) per cell: 256^3 cells
   with 2000 grains take 1.3 GB per vector instead of 134 GB dense.  The
   passes merge the sorted slot lists of the stencil and pointwise inputs
   and use the arithmetic of the masked one-cell passes, so results equal
   the dense ones bit for bit while no cell needs more than 12 slots.  A
   projected cell with more nonzero values keeps the 12 largest (equal
   values: the lower id) and divides them by their sum (the paper gives no
   rule; "S acted" for the RKL2 first-stage fix includes this step); the
   stored F(u^n) of RKL1/RKL2 keeps the 12 entries of largest magnitude
   (equal magnitudes: the lower id).  A state given with more than 12
   nonzero values in a cell is PF_EINVAL.  FE, SSP(s)2, RKL1 and
   RKL2 (fixed or adaptive); PF_EINVAL for SSP(10)4, PF_STEP_REUSE_RHS,
   PF_STEP_DEVICE_LOOP, pf_energy, and with PF_OPT_MASKED or
   PF_OPT_MOBILITY_SIMPLEX.  pf_set_state / pf_get_state / pf_rhs still take
   the dense layout (N x V values: for small N); pf_set_state_slots /
   pf_get_state_slots take the slot form.  pf_reduce's phase volumes are
   summed with atomics (their last bits depend on scheduling; the maxima,
   the grain count and the concentration total do not). */
enum { PF_OPT_TMA = 1, PF_OPT_MASKED = 2, PF_OPT_ONE_CELL = 4, PF_OPT_MOBILITY_SIMPLEX = 8, PF_OPT_SLOTS = 16 };
#define PF_N_SLOTS 12

/* Error tolerances of the weighted norm (Eq. error_norm): relative r and
   absolute a per field (phase field, concentration). */
typedef struct { double r_phi, a_phi, r_c, a_c; } pf_tol;

typedef struct {
    int ssp_stages;    /* s for PF_SSP2 (>= 2); ignored otherwise */
    double dt_mult;    /* > 0: fixed dt = dt_mult * dt_e; 0: adaptive (SSP104, RKL1, RKL2) */
    double dt0;        /* first adaptive step (0: 0.9 * dt_e); ignored if a previous adaptive
                          call left a proposal for the next step */
    int max_stages;    /* cap on RKL stages (0: 1001) */
    int max_attempts;  /* stop after this many attempted steps (0: no limit); the call then
                          returns PF_OK with t < t_end */
    /* Optional trace of attempted steps (NULL to skip): step size, stages,
       error norm and accepted flag, up to trace_cap entries. */
    int trace_cap;
    double *trace_dt;
    int *trace_s;
    double *trace_err;
    int *trace_acc;
    int *trace_len;
    int flags;         /* PF_STEP_* bit set (0: defaults) */
} pf_step_opts;

/* pf_step_opts.flags.  By default a fixed-step run on a non-default stream
   captures the smallest group of full steps after which the buffer rotation
   repeats into a CUDA graph (cached per handle) and replays it; results are
   identical to launching the passes one by one.  PF_STEP_NO_GRAPH disables
   that.
   PF_STEP_REUSE_RHS (adaptive RKL1/RKL2, dense storage) reuses F(u^{n+1}),
   which the error sweep of Sec. 3.3 evaluates anyway, as the next step's
   F(u^n) (the footnote on the Sommeijer estimate notes the paper's code
   does not): the error sweep also stores it, and after an accepted step the
   first stage is a pointwise pass u1 = S(u^n + mu~_1 dt F) (with the RKL2
   first-stage fix) instead of a stencil sweep.  One RHS evaluation fewer per
   accepted step; rhs_evals counts what was evaluated.  The trajectory is the
   one without reuse up to rounding.  The stored RHS belongs to the state it
   was computed from: pf_set_state, a rejected attempt or a step without the
   flag drop it.
   PF_STEP_DEVICE_LOOP (adaptive RKL1/RKL2 on a non-default stream; FP64, or
   FP32 dense storage with at most 32 phases; not with PF_STEP_REUSE_RHS or
   profiling; else PF_EINVAL) runs the adaptive loop device-driven: the
   output-time clip, stage count, stage coefficients and buffers, error
   norm, PID controller with bias and accept/reject of Sec. 3.2/3.3 are
   computed by GPU kernels inside one CUDA graph with conditional WHILE
   nodes, which carries up to 256 attempts per launch, so the host waits
   once per launch instead of once per attempt.  The controller's pow/atan
   then round as the GPU's math library does, which may differ from the
   host loop in the last bits of the step size. */
enum { PF_STEP_NO_GRAPH = 1, PF_STEP_REUSE_RHS = 2, PF_STEP_DEVICE_LOOP = 4 };

typedef struct {
    long long rhs_evals;       /* RHS sweeps, including rejected steps and STS error sweeps */
    long long steps_accepted;
    long long steps_rejected;
    double t;                  /* simulated time after the call */
    double dt_last;            /* size of the last attempted step */
    double err_last;           /* error norm of the last attempted step (0 for fixed steps) */
    double dt_e;               /* stable explicit Euler step used (Sec. 3.2) */
    double dt_next;            /* adaptive proposal for the next step */
    long long kernel_launches; /* CUDA kernels this call launched */
} pf_stats;

/* Create a handle for one simulation.  cuda_stream is a cudaStream_t (NULL:
   default stream).  Allocates the device buffers of every integrator
   (5 state vectors) plus reduction scratch.  PF_EINVAL on bad parameters,
   PF_ENOMEM when the device cannot hold the buffers. */
int pf_create(const pf_params *params, void *cuda_stream, struct pf_handle **out);

/* Set the state u (phase-major, (N + K) * V doubles; c may be NULL when
   K = 0 and is read from c otherwise) at time t.  Resets the step
   controller (Sec. 3.3).  PF_EINVAL on NULL phi. */
int pf_set_state(struct pf_handle *h, const double *phi, const double *c, double t, int ptr_is_device);

/* Semi-discrete RHS of the current state (Eq. phieq with the leading minus
   sign of the gradient flow, Eq. ceq; Sec. 3 second-order FD with face-flux
   differences), written phase-major: rhs_phi (N * V) and, when K = 1,
   rhs_c (V; may be NULL).  nz (V bytes, may be NULL) receives N_z, the
   number of nontrivial phases per cell (Sec. 3.1).  No state change. */
int pf_rhs(struct pf_handle *h, double *rhs_phi, double *rhs_c, unsigned char *nz, int ptr_is_device);
/* (pf_rhs synchronises the stream to read the kernel's status flags.) */

/* Advance to exactly t_end (Sec. 5: output at defined target times) with the
   given integrator.  Fixed steps (opts->dt_mult > 0): dt = dt_mult * dt_e, the
   last step shortened to land on t_end; RKL stage count from the rule of
   Sec. 3.2.  Adaptive (dt_mult = 0; PF_SSP104, PF_RKL1, PF_RKL2 only): the
   error estimate and norm of Sec. 3.3 and the PID controller with bias.  The
   simplex projection is applied to every stage.  tol may be NULL for fixed
   steps; opts may be NULL (defaults: s = 5, adaptive, dt0 = 0.9 dt_e).
   stats may be NULL.  PF_EUNSTABLE (a non-positive simplex sum, a non-finite
   concentration or error norm) and the other device-detected failures leave
   the state and time of the last accepted step: adaptive steps are checked
   after every attempt; in a run of fixed steps every pass after the failing
   one does nothing and the call returns the state after the last step that
   completed without a flag (stats->t and steps_accepted say which). */
int pf_step(struct pf_handle *h, pf_integrator integ, double t_end, const pf_tol *tol,
            const pf_step_opts *opts, pf_stats *stats);

/* Slot storage (PF_OPT_SLOTS; PF_EINVAL for other handles).  Set the state
   from its slot form: n_in planes of V values (vals[k * V + i]) and of
   phase ids (ids[k * V + i], 0..N-1, or -1 for an empty slot), in any order
   within a cell; entries whose value rounds to 0 in FP32 are dropped.  A
   cell with more than 12 nonzero values, an id out of range or a repeated
   id is PF_EINVAL.  c: V concentrations (K = 1).  Pointers as for
   pf_set_state; pageable host memory goes through temporary device copies
   freed before the call returns (Sec. 3.1: N_p values and ids per cell). */
int pf_set_state_slots(struct pf_handle *h, const double *vals, const int *ids, int n_in, const double *c,
                       double t, int ptr_is_device);

/* Copy a slot state out: 12 planes of V values and of ids (ascending ids
   first in every cell, then -1 with value 0), c (may be NULL) and t (may be
   NULL). */
int pf_get_state_slots(struct pf_handle *h, double *vals, int *ids, double *c, double *t, int ptr_is_device);

/* Copy the state out (phase-major doubles; c may be NULL), N_z of the
   current state (nz, V bytes, may be NULL) and the time (t, may be NULL). */
int pf_get_state(struct pf_handle *h, double *phi, double *c, unsigned char *nz, double *t,
                 int ptr_is_device);

/* Conserved totals (host outputs, FP64, deterministic): mass_c = sum c dV
   (0 when K = 0), vol_phi[a] = sum phi_a dV (N entries, may be NULL), and
   grains_alive = number of phases whose maximum is >= 0.5 (may be NULL). */
int pf_reduce(struct pf_handle *h, double *mass_c, double *vol_phi, int *grains_alive);

/* Energy functional F = int a + w + f dV of Eq. energy (Sec. 2) of the
   current state, evaluated in FP64 whatever the storage precision, written to
   the host double *F (deterministic for a given state and launch shape).
   a = -sum_{a>b} A_ab grad phi_a . grad phi_b with forward differences across
   the +x, +y, +z faces of each cell (a zero-gradient ghost across a
   non-periodic face), w = sum_{a>b} B_ab phi_a phi_b (the state is on the
   simplex), f = sum_a phi_a g_a(c_a) with the KKS phase concentrations
   (K = 1; absent when K = 0).  Phases that are zero at a cell and at its
   three forward neighbours contribute nothing; PF_EINVAL if more than 32
   phases are present around one cell.  Synchronises the handle's stream. */
int pf_energy(struct pf_handle *h, double *F);

/* Stable explicit Euler step dt_e = 2 / max(lambda_phi, lambda_c) from the
   Gershgorin reading of Sec. 3.2 (the estimates themselves are in the
   paper's supplement; the reading reproduces the three values printed in
   Sec. 5.3). */
int pf_dt_e(struct pf_handle *h, double *dt_e);

/* Self-test of the bounded device waits (failure detection without a GPU
   fault): launches one block on cuda_stream (NULL: default stream) whose
   thread waits on a shared-memory mbarrier that nothing arrives on, with the
   poll loop the TMA-staged kernels use and a limit of `polls` polls
   (1 .. 2^22, the kernels' own limit).  Returns PF_ETIMEOUT when the wait gave
   up, as it must; PF_OK if it completed (it cannot); PF_EINVAL for a limit out
   of range; PF_EDEVICE on a CUDA error.  The context stays usable.
   Synchronises cuda_stream. */
int pf_selftest_wait(void *cuda_stream, unsigned polls);

/* State of the adaptive step-size controller (Sec. 3.3: PID control with
   bias): the bias b (0.1..0.98; 0.9 after pf_set_state), the last two
   accepted biased error norms E1, E2 and step sizes dt1, dt2, how many of
   them are set (nhist 0..2), and the proposed next step dt_next (0: none,
   the next adaptive call starts from opts->dt0 or 0.9 dt_e).  A checkpoint
   of an adaptive run is pf_get_state + pf_get_controller; pf_set_state
   followed by pf_set_controller on any handle of the same problem resumes
   it so that the continued run takes the same steps as the uninterrupted
   one (with PF_STEP_REUSE_RHS the first resumed step re-evaluates F(u^n)).
   pf_set_controller returns PF_EINVAL for values outside those ranges or not
   finite, PF_ESTATE before pf_set_state. */
typedef struct {
    double b, E1, E2, dt1, dt2, dt_next;
    int nhist;
} pf_controller;
int pf_get_controller(struct pf_handle *h, pf_controller *out);
int pf_set_controller(struct pf_handle *h, const pf_controller *in);

/* Kinds of fused passes, for pf_profile. */
enum {
    PF_PASS_EULER = 0,       /* forward Euler stage */
    PF_PASS_SSP = 1,         /* SSP(s)2 / SSP(10)4 stages */
    PF_PASS_STS_FIRST = 2,   /* RKL stage 1 (stores F(u^n), RKL2 first-stage fix) */
    PF_PASS_RKL1 = 3,        /* RKL1 stages j >= 2 */
    PF_PASS_RKL2 = 4,        /* RKL2 stages j >= 2 */
    PF_PASS_STS_ERR = 5,     /* RKL error sweep: F(u^{n+1}), estimate and norm partials */
    PF_PASS_RHS = 6,         /* pf_rhs / N_z */
    PF_PASS_OTHER = 7,       /* reductions and layout conversion */
    PF_NPASS_KINDS = 8
};

/* Per-pass device timing with CUDA events recorded on the handle's stream
   around each fused pass (not part of the method; for measurement).  Reads
   the totals accumulated since the last reset into ms[PF_NPASS_KINDS] and
   launches[PF_NPASS_KINDS] (either may be NULL; synchronises), then
   enable = 1 resets and starts recording, enable = 0 resets and stops,
   enable = -1 keeps the totals and the current setting. */
int pf_profile(struct pf_handle *h, int enable, double *ms, long long *launches);

/* Kernel variants of the FP32 dense passes: two cells per thread (default
   where nx is even), one cell per thread, and one cell per thread with the
   phase planes staged into shared memory by TMA bulk tensor copies. */
enum { PF_KVAR_TWO_CELL = 0, PF_KVAR_ONE_CELL = 1, PF_KVAR_TMA = 2, PF_KVAR_COUNT = 3 };

/* Autotuner: times the RKL2 stage pass of this handle's current state with
   each kernel variant that applies (FP32 dense storage), switches the handle
   to the fastest and records the choice for the problem's shape (precision,
   dims, phases, K) in a process-wide table that later pf_create calls of the
   same shape apply (unless an option forces a variant).  *choice receives
   the PF_KVAR_* chosen (may be NULL); ms (may be NULL) receives
   PF_KVAR_COUNT average pass times in ms, -1 where a variant does not apply.
   FP64 and masked storage have one kernel: nothing is timed.  No state
   change.  PF_ESTATE without a state. */
int pf_autotune(struct pf_handle *h, int *choice, double *ms);

/* Number of CUDA kernels launched by this handle since pf_create (-1 on NULL). */
long long pf_launch_count(struct pf_handle *h);

/* Limits of pf_totals_noalloc: fields per call, and per-field partial slots
   of its fixed scratch (PF_NOALLOC_MAX_FIELDS * PF_NOALLOC_MAX_BLOCKS * 2
   doubles = 1.06 MB of device memory, reserved on every GPU that loads the
   library until the process exits). */
#define PF_NOALLOC_MAX_FIELDS 130
#define PF_NOALLOC_MAX_BLOCKS 512

/* pf_totals_noalloc -- the paper has no counterpart; this entry point exists
   for callers that must not allocate device memory.  cudaMalloc and cudaFree
   may synchronise the whole device, which a caller that keeps other streams
   busy or works under a latency budget cannot accept, and a caller whose
   device memory is entirely held by another allocator has none to give.
   It computes, for every field f < n_fields of a caller-owned FP64 state in
   the ABI layout (u_dev[f * n_cells + i], device memory of the current
   device), sum_dev[f] = dv * sum_i u_dev[f * n_cells + i] and max_dev[f] =
   max_i u_dev[f * n_cells + i] (either output may be NULL; both are device
   pointers).  It is the allocation-free form of the totals behind pf_reduce
   (mass = sum of the concentration field, volumes = sums of the phase
   fields, grains alive = phases whose max is >= 0.5).
   Scratch: a fixed device array inside the library; nothing is allocated and
   nothing is freed.  The first call on each device looks up that array's
   device address (once per device and context: after cudaDeviceReset the
   next call looks it up again); make that first call before any CUDA
   stream capture.  A NaN in a field makes that field's sum and maximum NaN.  Every call shares the array and writes every entry it
   later reads, so nothing needs clearing, but calls whose kernels overlap on
   the GPU (different streams without ordering) race on it and must be
   serialised by the caller.  The work is enqueued on cuda_stream (NULL: the
   default stream) and the call does not synchronise.
   Returns PF_EINVAL for NULL u_dev, n_cells < 1, n_fields < 1, both outputs
   NULL, or n_fields > PF_NOALLOC_MAX_FIELDS; PF_EDEVICE if a launch fails. */
int pf_totals_noalloc(const double *u_dev, int n_fields, long long n_cells, double dv, double *sum_dev,
                      double *max_dev, void *cuda_stream);

/* Device bytes a handle for these parameters holds once it has been
   created and a state has been set (state vectors, ABI staging buffer --
   none for slot storage, whose dense transfers allocate it on first use --,
   tables and reduction partials), without allocating anything.  Used to
   admit simulations by memory footprint. */
int pf_footprint(const pf_params *params, long long *bytes);

/* Caller-supplied device allocator (the paper has no counterpart: the
   library's device buffers may come from the caller, e.g. a framework's
   caching allocator).  alloc(bytes, cuda_stream, ctx) returns device memory
   of the current device usable on cuda_stream (the handle's stream), or NULL
   (pf_create then returns PF_ENOMEM); free(ptr, bytes, cuda_stream, ctx)
   takes back exactly what alloc returned, after the library has synchronised
   the stream.  pf_set_allocator sets the hook for the handles created after
   it (each handle keeps the hook it was created with until pf_destroy);
   alloc = free = NULL restores the default, CUDA's stream-ordered allocator.
   Process-wide, thread-safe.  PF_EINVAL when only one of the two is NULL. */
typedef void *(*pf_alloc_fn)(size_t bytes, void *cuda_stream, void *ctx);
typedef void (*pf_free_fn)(void *ptr, size_t bytes, void *cuda_stream, void *ctx);
int pf_set_allocator(pf_alloc_fn alloc, pf_free_fn free_fn, void *ctx);

/* Batched stepping for serving (continuous batching).  A batch advances
   many simulations together on its own CUDA stream: every round each
   admitted request takes one step (fixed steps) or one attempt (adaptive
   RKL1/RKL2, Sec. 3.3), and the passes of all requests are issued wave by
   wave, the passes of one kind (dimension, concentration field, pass
   signature) of FP32 dense problems with nx even in ONE packed launch whose
   blocks map to the problems (each block runs exactly what the problem's own
   launch would, so results equal those of pf_step on the handle alone).  The
   error norms and device flags of all requests come back in one transfer per
   round.  Requests that cannot be packed (FP64, masked or TMA storage, odd
   nx, SSP(10)4) launch their passes on their own handle's stream in the same
   round.  Every request keeps the bookkeeping of pf_step (fixed steps end at
   t0 + k dt, the controller state carries over), so its result equals that
   of pf_step on the handle alone (options of pf_step_opts other than
   ssp_stages, dt_mult, dt0 and max_stages are ignored).  Device memory: a request holds its handle's pf_footprint against
   the batch's budget max_bytes from admission until its result is taken.

   pf_batch_create: a batch with a budget of max_bytes (> 0) working on
   cuda_stream (NULL: the default stream).
   pf_batch_admit: add handle h (state set, not in another batch) to step to
   t_end with integ, tol and opts as pf_step would; *slot receives the
   request's slot.  PF_ENOMEM when the footprint does not fit the remaining
   budget (nothing changes: admit it later), PF_EINVAL for arguments pf_step
   would refuse.  The handle must not be used outside the batch until its
   result has been taken.
   pf_batch_run: up to `rounds` rounds (>= 1); *n_active (may be NULL)
   receives the number of requests still running.  Synchronises the batch's
   stream once per round.
   pf_batch_result: *done = 1 and the request's status and statistics
   (stats may be NULL) once it has finished or failed; its slot and budget
   are then released and the handle is free again (its stream ordered after
   the batch's work).  *done = 0 while it runs.
   pf_batch_destroy: drops every request (handles stay valid) and frees the
   batch.  NULL is accepted. */
typedef struct pf_batch pf_batch;
int pf_batch_create(long long max_bytes, void *cuda_stream, pf_batch **out);
int pf_batch_admit(pf_batch *b, struct pf_handle *h, pf_integrator integ, double t_end, const pf_tol *tol,
                   const pf_step_opts *opts, int *slot);
int pf_batch_run(pf_batch *b, int rounds, int *n_active);
int pf_batch_result(pf_batch *b, int slot, int *done, int *status, pf_stats *stats);
int pf_batch_destroy(pf_batch *b);

/* Release every device buffer of the handle.  NULL is accepted. */
int pf_destroy(struct pf_handle *h);

const char *pf_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif
