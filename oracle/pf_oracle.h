/*
 * pf_oracle.h -- plain, slow, FP64 CPU oracle for one explicit time step of the
 * obstacle-potential multi-phase-field + KKS concentration model of
 * Seiz & Takaki, "Numerical efficiency of explicit time integrators for
 * phase-field models" (arXiv 2601.16522).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this code; only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no header, helper, table
 * or constant with the CUDA engine.
 *
 * State layout (same as the public ABI): u = [phi_0[V], ..., phi_{N-1}[V],
 * c[V] (if K=1)], cell index i = (z*ny + y)*nx + x, x fastest.
 *
 * Pinning (see tests/test_oracle_*.py): every function here is pinned against
 * closed forms, invariants or numbers printed in the paper (the
 * mobility-weighted projection against the optimality conditions of its own
 * definition and the Euclidean simplex projection it reduces to), except
 *   - or_ssp104_embedded_weights (Sec. 3.3 cites external weights that the
 *     paper does not print; we use the minimum-norm order-3 embedding),
 *   - the chemical / diffusion parts of or_dt_e (Sec. 3.2: the Gershgorin
 *     estimates live in the missing supplement; our reading reproduces the
 *     three stable steps printed in Sec. 5.3 but is fitted, not derived),
 *   - the mobility-based simplex of Sec. 3.1/5.3 (cited, not described):
 *     or_project_cell_mobility is one reading of it (a projection in the
 *     metric the mobilities define), so the paper does not fix its values,
 *     and
 *   - the rule for a cell that needs more than N_p slots (Sec. 3.1 gives
 *     none): or_evict_cell / or_keep_rhs_cell are pinned against a sort of
 *     their own definition, not against the paper:
 *     parity unpinned for those four readings.
 */
#ifndef PF_ORACLE_H
#define PF_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

enum { OR_BC_PERIODIC = 0, OR_BC_NEUMANN = 1, OR_BC_DIRICHLET = 2 };
enum { OR_FEULER = 0, OR_SSP2 = 1, OR_SSP104 = 2, OR_RKL1 = 3, OR_RKL2 = 4 };
enum { OR_OK = 0, OR_EINVAL = 1, OR_EUNSTABLE = 3 };

typedef struct {
    int dim, nx, ny, nz;
    double dx;
    int N;                 /* number of phases (dense) */
    const int *ptype;      /* N entries: chemical type 0 (alpha) or 1 (beta) */
    const double *gamma;   /* N*N interface energies gamma_ab (symmetric) */
    const double *mob;     /* N*N interface mobilities M_ab (symmetric) */
    double W;              /* interface parameter, width pi*W (Sec. 2) */
    const double *Lover;   /* optional N*N phase-field mobility L_ab (Eq. thin-interface); NULL: pi*M/(4W) */
    int K;                 /* 0 or 1 concentration fields */
    double k[2], c0[2], D[2];   /* per chemical type (Eq. gibbs-energy, Eq. ceq) */
    int bc_phi[6], bc_c[6];     /* faces x-,x+,y-,y+,z-,z+ */
    double cdir[6];             /* Dirichlet concentration per face */
    int simplex;                /* projection S: 0 the standard one, 1 mobility-weighted */
    int n_slots;                /* > 0: per-cell phase slots, or_evict_cell after S */
} or_params;

typedef struct { double r_phi, a_phi, r_c, a_c; } or_tol;

typedef struct {
    double b;          /* controller bias (Sec. 3.3), starts at 0.9 */
    double E1, E2;     /* biased errors of the last two accepted steps */
    double dt1, dt2;   /* sizes of the last two accepted steps */
    int nhist;         /* accepted steps recorded (0,1,2) */
} or_ctrl;

typedef struct {
    long rhs_evals, accepted, rejected;
    double dt_last, err_last, dt_next;
} or_stats;

/* ---- model -------------------------------------------------------------- */
long or_ncells(const or_params *p);
/* A_ab = 4 W gamma/pi, B_ab = 4 gamma/(pi W), L_ab = pi M/(4W) (Sec. 2). */
void or_coeffs(const or_params *p, double *A, double *B, double *L);
/* Phase-field and concentration RHS (Eq. phieq, Eq. ceq, Sec. 3 FD), plus N_z. */
int or_rhs(const or_params *p, const double *u, double *r, unsigned char *nz);
/* Simplex projection S (Sec. 3.1); acted[i] (per cell, may be NULL) is set to
   1 where clamping or the >=1 rule changed a value.  Returns OR_EUNSTABLE if a
   cell sum is not positive.  With p->simplex = 1 the mobility-weighted
   projection (or_project_cell_mobility) replaces it. */
int or_project(const or_params *p, double *u, unsigned char *acted);
/* Mobility-weighted projection of one cell's N values y (in place), L the
   N*N phase-field mobilities: on P = {a : y_a > 0}, x_a = max(y_a - tau w_a, 0)
   with w_a the mean of L_ab over the other phases b of P and tau such that
   the x_a sum to 1; phases outside P become 0.  Returns 1 if a value changed
   (*acted), -1 if no value is positive (the cell cannot be projected), 0
   otherwise. */
int or_project_cell_mobility(int N, const double *L, double *y);
/* Per-cell phase slots (Sec. 3.1, N_p values and ids per cell): a cell with
   more than n_slots nonzero values keeps the n_slots largest (equal values:
   lower id first) and divides them by their sum (ascending ids); returns 1
   if it changed the cell.  or_project applies it after S when
   p->n_slots > 0 ("S acted" then includes it). */
int or_evict_cell(int N, int n_slots, double *y);
/* The stored RHS F(u^n) of the STS schemes in slots: a cell with more than
   n_slots nonzero entries keeps the n_slots largest in magnitude (equal
   magnitudes: lower id first), the others become 0 (reading, as above).
   Returns 1 if it changed the cell.  or_sys_pde applies it to F(u^n) after
   the first-stage fix when p->n_slots > 0. */
int or_keep_rhs_cell(int N, int n_slots, double *r);
/* Stable explicit Euler step from the Gershgorin reading (Sec. 3.2). */
double or_dt_e(const or_params *p);
/* Energy functional F = int a + w + f dV (Eq. energy) with forward
   differences across the +x, +y, +z faces of every cell for the gradients:
   a = -sum_{a>b} A_ab grad phi_a . grad phi_b, w = sum_{a>b} B_ab phi_a phi_b,
   f = sum_a phi_a g_a(c_a) = sum_a phi_a mu^2/(2 k_a) (K = 1).  The ghost
   value across a non-periodic face is the cell itself (zero gradient). */
double or_energy(const or_params *p, const double *u);
/* Totals (Sec. 5.2 area by integration): sum c dV, sum phi_a dV, #phases with max >= 0.5. */
void or_reduce(const or_params *p, const double *u, double *mass, double *vol, int *alive);

/* ---- integrators on a generic system (also used for Dahlquist tests) ---- */
typedef struct or_sys {
    long n;                 /* vector length = (N + K) * V */
    int N, K;               /* layout for projection / error filter / DoF count */
    long V;
    void *ctx;
    void (*rhs)(void *ctx, const double *u, double *r);
    int (*proj)(void *ctx, double *u, unsigned char *acted_cells); /* may be NULL */
    void (*keep_rhs)(void *ctx, double *r);   /* the stored F(u^n) of the STS schemes; may be NULL */
} or_sys;

void or_sys_pde(or_sys *s, const or_params *p);
/* u' = lam*u (V=1) or u' = (lr + i li) u stored as (re, im) (V=2) */
void or_sys_dahlquist(or_sys *s, double *lam2 /* [2] = {lr, li} */);

/* One step of size dt with s stages.  un is not modified.  Outputs unew,
   rn (effective rhs(u^n), NULL allowed) and for OR_SSP104 the embedded
   solution z (NULL allowed).  Returns #RHS evaluations or <0 on error. */
long or_step(const or_sys *S, int integ, double dt, int s, const double *un,
             double *unew, double *rn, double *z);
/* Stage-count rule (Sec. 3.2): smallest odd s whose RKL stability bound with
   0.9*dt_e covers dt. */
int or_sts_stages(int integ, double dt, double dt_e);
/* Local error estimate (Sec. 3.3) and weighted l2 norm (Eq. error_norm). */
double or_err_sts(const or_sys *S, const or_tol *tol, double dt, const double *un,
                  const double *unew, const double *rn, const double *rn1, long *ndof);
double or_err_embedded(const or_sys *S, const or_tol *tol, const double *un,
                       const double *unew, const double *z, long *ndof);
void or_ssp104_embedded_weights(double bh[10]);
void or_ctrl_init(or_ctrl *c);
/* PID + bias controller (Sec. 3.3).  Returns the next step size; *accept set. */
double or_ctrl_update(or_ctrl *c, double err, double dt, int P, int *accept);
int or_order(int integ);

/* ---- run to t_end (fixed: dt_mult > 0, adaptive: dt_mult == 0) ----------
   Exact output-time hitting (Sec. 5).  u is updated in place, *t advanced.
   Optional trace (cap entries): attempted dt, stages, error, accepted flag.
   Replay mode (replay_n > 0): instead of the controller, attempt i uses
   replay_dt[i], replay_s[i] and replay_acc[i]; the oracle's own error values
   are still written to the trace. */
int or_run(const or_params *p, int integ, double t_end, const or_tol *tol,
           double dt_mult, double dt0, int ssp_stages, int max_stages,
           double *u, double *t, or_ctrl *ctrl, or_stats *st,
           int cap, double *tr_dt, int *tr_s, double *tr_err, int *tr_acc, int *tr_len,
           int replay_n, const double *replay_dt, const int *replay_s, const int *replay_acc);

/* ---- controller-only run (Sec. 3.2-3.3) --------------------------------
   The decisions or_run takes in adaptive mode when the error norm of attempt
   k is errs[k]: the attempt's size (stretched onto t_end within 1e-9, capped
   by max_stages; 0: 1001), its RKL stage count, accept/reject and the PID
   controller update, without evaluating the model.  Starts at *t with the
   controller state ctrl and the previous proposal *dt_next (0: dt0, or
   0.9 dte when dt0 is 0); *t advances on acceptance, *dt_next receives the
   last proposal.  Stops at t_end or after n_err attempts.  The attempted
   dt, s and accept flags are written to the trace (up to cap entries);
   returns the number of attempts.  With h_given (may be NULL) the loop
   continues from the step sizes h_given[k] actually taken elsewhere (the
   controller update and the time advance use them), while the trace still
   holds the sizes this loop would have chosen: a one-attempt-ahead check
   that accumulates no difference between two loops. */
int or_drive(int integ, double dte, double t_end, double dt0, int max_stages, int n_err,
             const double *errs, const double *h_given, double *t, or_ctrl *ctrl, double *dt_next,
             int cap, double *tr_dt, int *tr_s, int *tr_acc);

#ifdef __cplusplus
}
#endif
#endif
