/*
 * pf_oracle.c -- plain FP64 reference implementation (TEST INFRASTRUCTURE ONLY;
 * never linked into the product).  Every loop is the textbook form of the
 * paper's equations: no blocking, fusion or reordering.  Built with
 * -ffp-contract=off so that no multiply-add is fused behind our back.
 *
 * Paper: Seiz & Takaki, arXiv 2601.16522.  Section numbers below refer to it.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "pf_oracle.h"

static const double PI = 3.14159265358979323846;

long or_ncells(const or_params *p) { return (long)p->nx * p->ny * p->nz; }

/* Sec. 2: A = 4 W gamma / pi, B = 4 gamma / (pi W), L = pi M / (4 W). */
void or_coeffs(const or_params *p, double *A, double *B, double *L)
{
    int N = p->N;
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            double g = p->gamma[a * N + b];
            A[a * N + b] = 4.0 * p->W * g / PI;
            B[a * N + b] = 4.0 * g / (PI * p->W);
            L[a * N + b] = p->Lover ? p->Lover[a * N + b] : PI * p->mob[a * N + b] / (4.0 * p->W);
        }
}

/* ---- neighbours and boundary ghosts (Sec. 3 cell-centred grid; Sec. 4 BCs) */

/* Neighbour of cell (x,y,z) across face f (0..5 = x-,x+,y-,y+,z-,z+).
   Returns its index, or -1 if the face is a non-periodic domain boundary. */
static long neighbour(const or_params *p, int x, int y, int z, int f)
{
    int c[3] = {x, y, z};
    int n[3] = {p->nx, p->ny, p->nz};
    int ax = f / 2;
    int v = c[ax] + ((f & 1) ? 1 : -1);
    if (v < 0 || v >= n[ax]) {
        if (p->bc_phi[f] != OR_BC_PERIODIC) return -1;
        v = (v + n[ax]) % n[ax];
    }
    c[ax] = v;
    return ((long)c[2] * p->ny + c[1]) * p->nx + c[0];
}

/* phi_a at the neighbour across face f; a zero-gradient ghost copies the cell. */
static double phi_nb(const or_params *p, const double *u, int a, long i, long j)
{
    long V = or_ncells(p);
    return j >= 0 ? u[a * V + j] : u[a * V + i];
}

/* KKS chemical potential for parabolic energies (Sec. 2):
   c = sum_a phi_a c_a, c_a = c0_a + mu/k_a  =>  mu = (c - sum phi c0)/(sum phi/k). */
static double chem_mu(const or_params *p, double c, const double *phis)
{
    double num = c, den = 0.0;
    for (int a = 0; a < p->N; ++a) {
        int t = p->ptype[a];
        num = num - phis[a] * p->c0[t];
        den = den + phis[a] * (1.0 / p->k[t]);
    }
    return num / den;
}

int or_rhs(const or_params *p, const double *u, double *r, unsigned char *nzout)
{
    int N = p->N, K = p->K, nf = 2 * p->dim;
    long V = or_ncells(p);
    double *A = malloc(sizeof(double) * N * N), *B = malloc(sizeof(double) * N * N),
           *L = malloc(sizeof(double) * N * N);
    or_coeffs(p, A, B, L);
    double dx2 = p->dx * p->dx;

    /* Every cell is computed on its own from the input, so when the oracle is
       built with OpenMP (only for the timed all-core CPU baseline) the rows
       are shared out among threads, each with its own scratch; without it
       the pragmas are ignored.  The arithmetic of a cell is the same. */
#pragma omp parallel
    {
    double *lap = malloc(sizeof(double) * N), *delta = malloc(sizeof(double) * N),
           *psi = malloc(sizeof(double) * N), *phc = malloc(sizeof(double) * N),
           *phn = malloc(sizeof(double) * N);
    int *act = malloc(sizeof(int) * N);
#pragma omp for collapse(2) schedule(static)
    for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
    for (int x = 0; x < p->nx; ++x) {
        long i = ((long)z * p->ny + y) * p->nx + x;
        long nb[6];
        for (int f = 0; f < nf; ++f) nb[f] = neighbour(p, x, y, z, f);

        /* activity n(phi_a, grad phi_a) (Eq. phieq): nontrivial over the
           cell and its face neighbours; Laplacian (Sec. 3 second-order FD). */
        int Nz = 0;
        for (int a = 0; a < N; ++a) {
            double v0 = u[a * V + i];
            double mx = v0, mn = v0, l = 0.0;
            for (int f = 0; f < nf; ++f) {
                double v = phi_nb(p, u, a, i, nb[f]);
                if (v > mx) mx = v;
                if (v < mn) mn = v;
                l = l + (v - v0);
            }
            phc[a] = v0;
            lap[a] = l / dx2;
            act[a] = (mx > 0.0 && mn < 1.0) ? 1 : 0;
            Nz += act[a];
        }
        if (nzout) nzout[i] = (unsigned char)Nz;

        /* grand potential psi_a = -mu^2/(2k_a) - mu c0_a (Sec. 2) */
        double mu = 0.0;
        for (int a = 0; a < N; ++a) psi[a] = 0.0;
        if (K) {
            mu = chem_mu(p, u[N * V + i], phc);
            for (int a = 0; a < N; ++a) {
                int t = p->ptype[a];
                psi[a] = -(mu * mu) / (2.0 * p->k[t]) - mu * p->c0[t];
            }
        }

        /* variational derivative dF/dphi_a = sum_{b != a}(A_ab lap_b + B_ab phi_b) + psi_a */
        for (int a = 0; a < N; ++a) {
            double d = 0.0;
            for (int b = 0; b < N; ++b) {
                if (b == a) continue;
                d = d + (A[a * N + b] * lap[b] + B[a * N + b] * phc[b]);
            }
            delta[a] = d + psi[a];
        }

        /* Steinbach pairwise evolution with the leading minus sign (gradient
           flow): dphi_a/dt = -(1/N_z) sum_b L_ab n_a n_b (delta_a - delta_b). */
        for (int a = 0; a < N; ++a) {
            double ra = 0.0;
            if (act[a] && Nz > 1) {
                double s = 0.0;
                for (int b = 0; b < N; ++b) {
                    if (b == a || !act[b]) continue;
                    s = s + L[a * N + b] * (delta[a] - delta[b]);
                }
                ra = -(s / (double)Nz);
            }
            r[a * V + i] = ra;
        }

        /* concentration: dc/dt = div( sum_a D_a phi_a / k_a grad mu ) (Eq. ceq),
           as face-flux differences with arithmetic face means of phi. */
        if (K) {
            double c_i = u[N * V + i], acc = 0.0;
            for (int f = 0; f < nf; ++f) {
                double cn;
                if (nb[f] >= 0) {
                    cn = u[N * V + nb[f]];
                    for (int a = 0; a < N; ++a) phn[a] = u[a * V + nb[f]];
                } else {
                    for (int a = 0; a < N; ++a) phn[a] = phc[a];
                    cn = (p->bc_c[f] == OR_BC_DIRICHLET) ? 2.0 * p->cdir[f] - c_i : c_i;
                }
                double mun = chem_mu(p, cn, phn);
                double mf = 0.0;
                for (int a = 0; a < N; ++a) {
                    int t = p->ptype[a];
                    mf = mf + (p->D[t] / p->k[t]) * (0.5 * (phc[a] + phn[a]));
                }
                acc = acc + mf * (mun - mu);
            }
            r[N * V + i] = acc / dx2;
        }
    }
    free(lap); free(delta); free(psi); free(phc); free(phn); free(act);
    }
    free(A); free(B); free(L);
    return OR_OK;
}

/* Simplex projection S (Sec. 3.1): clamp negatives to 0; if a component is
   >= 1 it becomes 1 and all others 0 (largest wins, ties to the lowest id);
   finally divide by the sum. */
/* Mobility-weighted projection of one cell (a reading of the mobility-based
   simplex that Sec. 3.1 cites for the particle cases of Sec. 5.3 without
   describing it): the point of the simplex face spanned by the phases with a
   positive value, P = {a : y_a > 0}, nearest to y in the metric
   sum_a (x_a - y_a)^2 / w_a, where w_a is the mean phase-field mobility L_ab
   of phase a towards the other phases of P.  Its optimality conditions give
   x_a = max(y_a - tau w_a, 0) with tau fixed by sum_a x_a = 1, so a phase
   that moves slowly against its neighbours (an immobile particle) takes a
   small share of the correction, and with equal mobilities this is the
   Euclidean projection.  tau by the active-set iteration (Michelot 1986, with
   weights): start from P, set tau = (sum y - 1) / sum w over the active
   phases, drop the phases with y_a - tau w_a <= 0, repeat until none is
   dropped (tau only grows, so a dropped phase stays at 0).  Sums run over
   ascending phase ids.  One phase in P becomes 1; if every weight is 0 the
   standard S is applied instead. */
int or_project_cell_mobility(int N, const double *L, double *y)
{
    int *pid = malloc(sizeof(int) * N), *on = malloc(sizeof(int) * N);
    double *w = malloc(sizeof(double) * N), *x = malloc(sizeof(double) * N);
    int np = 0, ret = 0;
    for (int a = 0; a < N; ++a)
        if (y[a] > 0.0) pid[np++] = a;
    if (np == 0) { ret = -1; goto done; }
    for (int a = 0; a < N; ++a) x[a] = 0.0;
    if (np == 1) {
        x[pid[0]] = 1.0;
    } else {
        double wsum = 0.0;
        for (int k = 0; k < np; ++k) {
            double s = 0.0;
            for (int j = 0; j < np; ++j)
                if (j != k) s = s + L[pid[k] * N + pid[j]];
            w[k] = s / (double)(np - 1);
            wsum = wsum + w[k];
            on[k] = 1;
        }
        int standard = !(wsum > 0.0);
        if (!standard) {
            double tau = 0.0;
            for (;;) {
                double sy = 0.0, sw = 0.0;
                for (int k = 0; k < np; ++k)
                    if (on[k]) { sy = sy + y[pid[k]]; sw = sw + w[k]; }
                if (!(sw > 0.0)) { standard = 1; break; }   /* only immobile phases left */
                tau = (sy - 1.0) / sw;
                int dropped = 0;
                for (int k = 0; k < np; ++k)
                    if (on[k] && y[pid[k]] - tau * w[k] <= 0.0) { on[k] = 0; dropped = 1; }
                if (!dropped) break;
            }
            if (!standard)
                for (int k = 0; k < np; ++k) x[pid[k]] = on[k] ? y[pid[k]] - tau * w[k] : 0.0;
        }
        if (standard) {
            /* no mobility to share the correction: the standard S (>= 1 rule, divide) */
            int amax = -1;
            for (int k = 0; k < np; ++k)
                if (y[pid[k]] >= 1.0 && (amax < 0 || y[pid[k]] > y[amax])) amax = pid[k];
            double s = 0.0;
            for (int k = 0; k < np; ++k) s = s + y[pid[k]];
            for (int k = 0; k < np; ++k)
                x[pid[k]] = amax >= 0 ? (pid[k] == amax ? 1.0 : 0.0) : y[pid[k]] / s;
        }
    }
    for (int a = 0; a < N; ++a) {
        if (x[a] != y[a]) ret = 1;
        y[a] = x[a];
    }
done:
    free(pid); free(on); free(w); free(x);
    return ret;
}

/* Per-cell phase slots (Sec. 3.1: each cell stores N_p phase values with
   their phase ids): a projected cell with more than n_slots nonzero values
   keeps the n_slots largest (equal values: the lower id first), the others
   become 0, and the kept ones are divided by their sum (ascending ids) so
   the cell stays on the simplex.  The paper gives no rule for a cell that
   would need more slots; this is the reading.  Returns 1 if the cell
   changed. */
int or_evict_cell(int N, int n_slots, double *y)
{
    int cnt = 0;
    for (int a = 0; a < N; ++a)
        if (y[a] != 0.0) cnt++;
    if (n_slots <= 0 || cnt <= n_slots) return 0;
    unsigned char *keep = calloc((size_t)N, 1);
    for (int a = 0; a < N; ++a) {
        if (y[a] == 0.0) continue;
        int rank = 0;   /* entries that go before a */
        for (int b = 0; b < N; ++b)
            if (b != a && y[b] != 0.0 && (y[b] > y[a] || (y[b] == y[a] && b < a))) rank++;
        keep[a] = rank < n_slots;
    }
    double s = 0.0;
    for (int a = 0; a < N; ++a)
        if (keep[a]) s = s + y[a];
    for (int a = 0; a < N; ++a) y[a] = keep[a] ? y[a] / s : 0.0;
    free(keep);
    return 1;
}

int or_keep_rhs_cell(int N, int n_slots, double *r)
{
    int cnt = 0;
    for (int a = 0; a < N; ++a)
        if (r[a] != 0.0) cnt++;
    if (n_slots <= 0 || cnt <= n_slots) return 0;
    unsigned char *keep = calloc((size_t)N, 1);
    for (int a = 0; a < N; ++a) {
        if (r[a] == 0.0) continue;
        int rank = 0;
        for (int b = 0; b < N; ++b)
            if (b != a && r[b] != 0.0 && (fabs(r[b]) > fabs(r[a]) || (fabs(r[b]) == fabs(r[a]) && b < a))) rank++;
        keep[a] = rank < n_slots;
    }
    for (int a = 0; a < N; ++a)
        if (!keep[a]) r[a] = 0.0;
    free(keep);
    return 1;
}

static int project_cells(const or_params *p, double *u, unsigned char *acted);

int or_project(const or_params *p, double *u, unsigned char *acted)
{
    int st = project_cells(p, u, acted);
    if (p->n_slots > 0) {
        int N = p->N;
        long V = or_ncells(p);
        double *y = malloc(sizeof(double) * N);
        for (long i = 0; i < V; ++i) {
            for (int a = 0; a < N; ++a) y[a] = u[a * V + i];
            if (or_evict_cell(N, p->n_slots, y)) {
                for (int a = 0; a < N; ++a) u[a * V + i] = y[a];
                if (acted) acted[i] = 1;
            }
        }
        free(y);
    }
    return st;
}

static int project_cells(const or_params *p, double *u, unsigned char *acted)
{
    int N = p->N;
    long V = or_ncells(p);
    int bad = 0;
    if (p->simplex == 1) {
        double *A = malloc(sizeof(double) * N * N), *B = malloc(sizeof(double) * N * N),
               *L = malloc(sizeof(double) * N * N), *y = malloc(sizeof(double) * N);
        or_coeffs(p, A, B, L);
        for (long i = 0; i < V; ++i) {
            for (int a = 0; a < N; ++a) y[a] = u[a * V + i];
            int r = or_project_cell_mobility(N, L, y);
            if (r < 0) { bad = 1; continue; }
            for (int a = 0; a < N; ++a) u[a * V + i] = y[a];
            if (acted) acted[i] = (unsigned char)r;
        }
        free(A); free(B); free(L); free(y);
        return bad ? OR_EUNSTABLE : OR_OK;
    }
    for (long i = 0; i < V; ++i) {
        int changed = 0;
        for (int a = 0; a < N; ++a)
            if (u[a * V + i] < 0.0) { u[a * V + i] = 0.0; changed = 1; }
        int amax = -1;
        for (int a = 0; a < N; ++a)
            if (u[a * V + i] >= 1.0 && (amax < 0 || u[a * V + i] > u[amax * V + i])) amax = a;
        if (amax >= 0)
            for (int a = 0; a < N; ++a) {
                double v = (a == amax) ? 1.0 : 0.0;
                if (u[a * V + i] != v) changed = 1;
                u[a * V + i] = v;
            }
        double s = 0.0;
        for (int a = 0; a < N; ++a) s = s + u[a * V + i];
        if (!(s > 0.0)) { bad = 1; continue; }
        for (int a = 0; a < N; ++a) u[a * V + i] = u[a * V + i] / s;
        if (acted) acted[i] = (unsigned char)changed;
    }
    return bad ? OR_EUNSTABLE : OR_OK;
}

/* Gershgorin reading of the stable Euler step (Sec. 3.2, values Sec. 5.3):
   lambda_phi = max L (A 4d/dx^2 - B) [+ max L k |dc0| max c0 if K],
   lambda_c   = 4 d D_max / dx^2 (1 + |dc0|/2);  dt_e = 2 / max. */
double or_dt_e(const or_params *p)
{
    int N = p->N;
    double *A = malloc(sizeof(double) * N * N), *B = malloc(sizeof(double) * N * N),
           *L = malloc(sizeof(double) * N * N);
    or_coeffs(p, A, B, L);
    double d4 = 4.0 * p->dim / (p->dx * p->dx);
    double lphi = 0.0, lmax = 0.0;
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            if (a == b) continue;
            double v = L[a * N + b] * (A[a * N + b] * d4 - B[a * N + b]);
            if (v > lphi) lphi = v;
            if (L[a * N + b] > lmax) lmax = L[a * N + b];
        }
    double lam = lphi;
    if (p->K) {
        double kmax = 0.0, c0max = 0.0, c0min = 1e300, Dmax = 0.0;
        int used[2] = {0, 0};
        for (int a = 0; a < N; ++a) used[p->ptype[a]] = 1;
        for (int t = 0; t < 2; ++t) {
            if (!used[t]) continue;
            if (p->k[t] > kmax) kmax = p->k[t];
            if (p->c0[t] > c0max) c0max = p->c0[t];
            if (p->c0[t] < c0min) c0min = p->c0[t];
            if (p->D[t] > Dmax) Dmax = p->D[t];
        }
        double dc0 = c0max - c0min;
        double chem = lmax * kmax * dc0 * c0max;
        double lc = d4 * Dmax * (1.0 + dc0 / 2.0);
        lam = lphi + chem;
        if (lc > lam) lam = lc;
    }
    free(A); free(B); free(L);
    return 2.0 / lam;
}

double or_energy(const or_params *p, const double *u)
{
    int N = p->N;
    long V = or_ncells(p);
    double *A = malloc(sizeof(double) * N * N), *B = malloc(sizeof(double) * N * N),
           *L = malloc(sizeof(double) * N * N), *phc = malloc(sizeof(double) * N),
           *grad = malloc(sizeof(double) * N * 3);
    or_coeffs(p, A, B, L);
    double dv = pow(p->dx, p->dim), total = 0.0;
    for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
    for (int x = 0; x < p->nx; ++x) {
        long i = ((long)z * p->ny + y) * p->nx + x;
        for (int a = 0; a < N; ++a) {
            phc[a] = u[a * V + i];
            for (int ax = 0; ax < p->dim; ++ax) {
                long j = neighbour(p, x, y, z, 2 * ax + 1);
                double vn = j >= 0 ? u[a * V + j] : phc[a];
                grad[a * 3 + ax] = (vn - phc[a]) / p->dx;
            }
        }
        double e = 0.0;
        for (int a = 0; a < N; ++a)
            for (int b = 0; b < a; ++b) {
                double gg = 0.0;
                for (int ax = 0; ax < p->dim; ++ax) gg = gg + grad[a * 3 + ax] * grad[b * 3 + ax];
                e = e - A[a * N + b] * gg;
                e = e + B[a * N + b] * phc[a] * phc[b];
            }
        if (p->K) {
            double mu = chem_mu(p, u[N * V + i], phc);
            for (int a = 0; a < N; ++a) e = e + phc[a] * (mu * mu / (2.0 * p->k[p->ptype[a]]));
        }
        total = total + e;
    }
    free(A); free(B); free(L); free(phc); free(grad);
    return total * dv;
}

void or_reduce(const or_params *p, const double *u, double *mass, double *vol, int *alive)
{
    long V = or_ncells(p);
    double dv = pow(p->dx, p->dim);
    int n_alive = 0;
    for (int a = 0; a < p->N; ++a) {
        double s = 0.0, mx = -1e300;
        for (long i = 0; i < V; ++i) {
            s = s + u[a * V + i];
            if (u[a * V + i] > mx) mx = u[a * V + i];
        }
        if (vol) vol[a] = s * dv;
        if (mx >= 0.5) n_alive++;
    }
    if (alive) *alive = n_alive;
    if (mass) {
        double s = 0.0;
        if (p->K)
            for (long i = 0; i < V; ++i) s = s + u[p->N * V + i];
        *mass = s * dv;
    }
}

/* ---- generic systems --------------------------------------------------- */

static void pde_rhs(void *ctx, const double *u, double *r) { or_rhs((const or_params *)ctx, u, r, NULL); }
static int pde_proj(void *ctx, double *u, unsigned char *acted) { return or_project((const or_params *)ctx, u, acted); }

static void pde_keep_rhs(void *ctx, double *r)
{
    const or_params *p = (const or_params *)ctx;
    int N = p->N;
    long V = or_ncells(p);
    double *y = malloc(sizeof(double) * N);
    for (long i = 0; i < V; ++i) {
        for (int a = 0; a < N; ++a) y[a] = r[a * V + i];
        if (or_keep_rhs_cell(N, p->n_slots, y))
            for (int a = 0; a < N; ++a) r[a * V + i] = y[a];
    }
    free(y);
}

void or_sys_pde(or_sys *s, const or_params *p)
{
    s->V = or_ncells(p);
    s->N = p->N;
    s->K = p->K;
    s->n = (long)(p->N + p->K) * s->V;
    s->ctx = (void *)p;
    s->rhs = pde_rhs;
    s->proj = pde_proj;
    s->keep_rhs = p->n_slots > 0 ? pde_keep_rhs : NULL;
}

static void dahl_rhs(void *ctx, const double *u, double *r)
{
    const double *l = (const double *)ctx;
    /* complex multiplication (lr + i li)(ur + i ui) */
    r[0] = l[0] * u[0] - l[1] * u[1];
    r[1] = l[1] * u[0] + l[0] * u[1];
}

void or_sys_dahlquist(or_sys *s, double *lam2)
{
    s->V = 2; s->N = 0; s->K = 1; s->n = 2;
    s->ctx = lam2;
    s->rhs = dahl_rhs;
    s->proj = NULL;
    s->keep_rhs = NULL;
}

/* ---- integrators (Sec. 3.2) ------------------------------------------- */

static void project(const or_sys *S, double *u, unsigned char *acted, int *bad)
{
    if (S->proj && S->N > 0 && S->proj(S->ctx, u, acted) != OR_OK) *bad = 1;
}

/* SSP(10,4) of Ketcheson (2008) written in Butcher form, needed only to derive
   the embedded weights: the stage values of the low-storage form are
   Y1..Y5 = Euler chain with h/6, Y6 = 3/5 u + 2/5 (Y5 + h/6 F5), Y7..Y10 the
   continued chain, and u_{n+1} = 1/25 u + 9/25 (Y5 + h/6 F5) + 3/5 Y10 + h/10 F10
   (Sec. 3.2 "SSP(10)4").  Embedded order-3 weights are not printed in the
   paper (Sec. 3.3 cites external ones).  The method's own weights are all
   1/10, which is already the minimum-norm solution of the order-3
   conditions, so that choice would give a zero estimate.  Reading: the
   embedding does not use the last stage (bh_10 = 0) and is the minimum-norm
   solution of the four order-3 conditions over bh_1..bh_9.  Parity unpinned
   for this reading: its order is pinned (Dahlquist tests and a nonlinear
   system), the minimum-norm choice is not. */
static void ssp104_tableau(double Am[10][10], double b[10])
{
    memset(Am, 0, sizeof(double) * 100);
    /* Y_i as coefficients of h*F_j (u-coefficient is 1 for every stage) */
    for (int i = 1; i < 5; ++i)
        for (int j = 0; j < i; ++j) Am[i][j] = 1.0 / 6.0;
    /* Y6 = 3/5 u + 2/5 (Y5 + h/6 F5): u-coefficient 3/5 + 2/5 = 1 */
    for (int j = 0; j < 5; ++j) Am[5][j] = 0.4 * (1.0 / 6.0);
    for (int i = 6; i < 10; ++i) {
        for (int j = 0; j < 10; ++j) Am[i][j] = Am[i - 1][j];
        Am[i][i - 1] = Am[i][i - 1] + 1.0 / 6.0;
    }
    /* u_{n+1} = 1/25 u + 9/25 (Y5 + h/6 F5) + 3/5 Y10 + h/10 F10 */
    for (int j = 0; j < 10; ++j) b[j] = 0.0;
    for (int j = 0; j < 5; ++j) b[j] = b[j] + (9.0 / 25.0) * (1.0 / 6.0);
    for (int j = 0; j < 10; ++j) b[j] = b[j] + 0.6 * Am[9][j];
    b[9] = b[9] + 0.1;
}

void or_ssp104_embedded_weights(double bh[10])
{
    double Am[10][10], b[10], c[10];
    ssp104_tableau(Am, b);
    for (int i = 0; i < 10; ++i) {
        c[i] = 0.0;
        for (int j = 0; j < 10; ++j) c[i] = c[i] + Am[i][j];
    }
    /* order-3 conditions M bh = g: sum bh = 1, sum bh c = 1/2,
       sum bh c^2 = 1/3, sum_i bh_i sum_j A_ij c_j = 1/6 */
    double M[4][10], g[4] = {1.0, 0.5, 1.0 / 3.0, 1.0 / 6.0};
    for (int i = 0; i < 10; ++i) {
        double ac = 0.0;
        for (int j = 0; j < 10; ++j) ac = ac + Am[i][j] * c[j];
        M[0][i] = 1.0; M[1][i] = c[i]; M[2][i] = c[i] * c[i]; M[3][i] = ac;
        if (i == 9) { M[0][i] = 0.0; M[1][i] = 0.0; M[2][i] = 0.0; M[3][i] = 0.0; }
    }
    /* bh = M^T (M M^T)^{-1} g  (Gaussian elimination with partial pivoting) */
    double G[4][5];
    for (int r = 0; r < 4; ++r) {
        for (int q = 0; q < 4; ++q) {
            double s = 0.0;
            for (int i = 0; i < 10; ++i) s = s + M[r][i] * M[q][i];
            G[r][q] = s;
        }
        G[r][4] = g[r];
    }
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int r = col + 1; r < 4; ++r) if (fabs(G[r][col]) > fabs(G[piv][col])) piv = r;
        for (int q = 0; q < 5; ++q) { double t = G[col][q]; G[col][q] = G[piv][q]; G[piv][q] = t; }
        for (int r = 0; r < 4; ++r) {
            if (r == col) continue;
            double f = G[r][col] / G[col][col];
            for (int q = 0; q < 5; ++q) G[r][q] = G[r][q] - f * G[col][q];
        }
    }
    double y[4];
    for (int r = 0; r < 4; ++r) y[r] = G[r][4] / G[r][r];
    for (int i = 0; i < 10; ++i) {
        double s = 0.0;
        for (int r = 0; r < 4; ++r) s = s + M[r][i] * y[r];
        bh[i] = s;
    }
}

/* RKL2 b_j (Meyer et al. 2014): b_0 = b_1 = b_2 = 1/3, b_j = (j^2+j-2)/(2j(j+1)). */
static double rkl2_b(int j)
{
    if (j < 2) return 1.0 / 3.0;
    double jj = (double)j;
    return (jj * jj + jj - 2.0) / (2.0 * jj * (jj + 1.0));
}

long or_step(const or_sys *S, int integ, double dt, int s, const double *un,
             double *unew, double *rn, double *z)
{
    long n = S->n, evals = 0;
    int bad = 0;
    double *r = malloc(sizeof(double) * n);
    double *q1 = malloc(sizeof(double) * n), *q2 = malloc(sizeof(double) * n),
           *q3 = malloc(sizeof(double) * n);
    unsigned char *acted = S->V > 0 ? calloc((size_t)S->V, 1) : NULL;

    if (integ == OR_FEULER) {
        /* u^{n+1} = S(u^n + dt rhs(u^n)) */
        S->rhs(S->ctx, un, r); evals++;
        if (rn) memcpy(rn, r, sizeof(double) * n);
        for (long i = 0; i < n; ++i) unew[i] = un[i] + dt * r[i];
        project(S, unew, NULL, &bad);
    } else if (integ == OR_SSP2) {
        /* Alg. ssp2 with the final combination on the newest stage
           (Ketcheson 2008): s-1 Euler substeps of dt/(s-1), then
           u^{n+1} = 1/s u^n + (s-1)/s q + dt/s rhs(q). */
        if (s < 2) { evals = -1; goto done; }
        memcpy(q1, un, sizeof(double) * n);
        double h = dt / (double)(s - 1);
        for (int st = 1; st <= s - 1; ++st) {
            S->rhs(S->ctx, q1, r); evals++;
            if (st == 1 && rn) memcpy(rn, r, sizeof(double) * n);
            for (long i = 0; i < n; ++i) q3[i] = q1[i] + h * r[i];
            project(S, q3, NULL, &bad);
            double *t = q1; q1 = q3; q3 = t;
        }
        S->rhs(S->ctx, q1, r); evals++;
        double a0 = 1.0 / (double)s, a1 = (double)(s - 1) / (double)s, b1 = dt / (double)s;
        for (long i = 0; i < n; ++i) unew[i] = a0 * un[i] + a1 * q1[i] + b1 * r[i];
        project(S, unew, NULL, &bad);
    } else if (integ == OR_SSP104) {
        /* Ketcheson (2008) low-storage SSP(10,4); extra buffer q3 for the
           stage output; embedded solution z = u^n + dt sum_i bh_i F_i. */
        double bh[10];
        or_ssp104_embedded_weights(bh);
        memcpy(q1, un, sizeof(double) * n);
        memcpy(q2, un, sizeof(double) * n);
        if (z) memcpy(z, un, sizeof(double) * n);
        double h6 = dt / 6.0;
        for (int st = 1; st <= 9; ++st) {
            S->rhs(S->ctx, q1, r); evals++;
            if (st == 1 && rn) memcpy(rn, r, sizeof(double) * n);
            if (z) for (long i = 0; i < n; ++i) z[i] = z[i] + (dt * bh[st - 1]) * r[i];
            for (long i = 0; i < n; ++i) q3[i] = q1[i] + h6 * r[i];
            project(S, q3, NULL, &bad);
            double *t = q1; q1 = q3; q3 = t;
            if (st == 5) {
                for (long i = 0; i < n; ++i) q2[i] = (1.0 / 25.0) * q2[i] + (9.0 / 25.0) * q1[i];
                for (long i = 0; i < n; ++i) q1[i] = 15.0 * q2[i] + (-5.0) * q1[i];
            }
        }
        S->rhs(S->ctx, q1, r); evals++;
        if (z) for (long i = 0; i < n; ++i) z[i] = z[i] + (dt * bh[9]) * r[i];
        for (long i = 0; i < n; ++i) unew[i] = 1.0 * q2[i] + 0.6 * q1[i] + (dt / 10.0) * r[i];
        project(S, unew, NULL, &bad);
    } else if (integ == OR_RKL1 || integ == OR_RKL2) {
        /* Eq. sts: u^{n,1} = u^n + mu~_1 dt F(u^n);
           u^{n,j} = (1-mu_j-nu_j) u^n + mu_j u^{n,j-1} + nu_j u^{n,j-2}
                     + dt (mu~_j F(u^{n,j-1}) + gamma~_j F(u^n)),
           coefficients of the Legendre basis (Meyer et al. 2012/2014), the
           simplex projection after every stage, and for RKL2 the first-stage
           replacement of F(u^n) where the projection acted (Sec. 3.2). */
        int o2 = (integ == OR_RKL2);
        if (s < (o2 ? 2 : 1)) { evals = -1; goto done; }
        double ds = (double)s;
        double w1 = o2 ? 4.0 / (ds * ds + ds - 2.0) : 2.0 / (ds * ds + ds);
        double mt1 = o2 ? rkl2_b(1) * w1 : w1;
        double *r0 = malloc(sizeof(double) * n);
        double *ym2 = q1, *ym1 = q2, *yj = q3;   /* Y_{j-2}, Y_{j-1}, Y_j */
        S->rhs(S->ctx, un, r0); evals++;
        for (long i = 0; i < n; ++i) ym1[i] = un[i] + (mt1 * dt) * r0[i];
        project(S, ym1, acted, &bad);
        if (o2 && acted) {
            long V = S->V;
            for (int a = 0; a < S->N; ++a)
                for (long i = 0; i < V; ++i)
                    if (acted[i]) r0[a * V + i] = (ym1[a * V + i] - un[a * V + i]) / (mt1 * dt);
        }
        if (S->keep_rhs) S->keep_rhs(S->ctx, r0);
        memcpy(ym2, un, sizeof(double) * n);
        for (int j = 2; j <= s; ++j) {
            double dj = (double)j, mu, nu, mt, gt;
            if (o2) {
                mu = ((2.0 * dj - 1.0) / dj) * (rkl2_b(j) / rkl2_b(j - 1));
                nu = -((dj - 1.0) / dj) * (rkl2_b(j) / rkl2_b(j - 2));
                mt = mu * w1;
                gt = -(1.0 - rkl2_b(j - 1)) * mt;
            } else {
                mu = (2.0 * dj - 1.0) / dj;
                nu = -(dj - 1.0) / dj;
                mt = w1 * mu;
                gt = 0.0;
            }
            S->rhs(S->ctx, ym1, r); evals++;
            double c0 = (1.0 - mu) - nu;
            for (long i = 0; i < n; ++i) {
                if (o2)
                    yj[i] = c0 * un[i] + mu * ym1[i] + nu * ym2[i] + (mt * dt) * r[i] + (gt * dt) * r0[i];
                else
                    yj[i] = mu * ym1[i] + nu * ym2[i] + (mt * dt) * r[i];
            }
            project(S, yj, NULL, &bad);
            double *t = ym2; ym2 = ym1; ym1 = yj; yj = t;
        }
        memcpy(unew, ym1, sizeof(double) * n);
        if (rn) memcpy(rn, r0, sizeof(double) * n);
        free(r0);
    } else {
        evals = -1;
    }
done:
    free(r); free(q1); free(q2); free(q3); free(acted);
    if (bad) return -2;
    return evals;
}

int or_sts_stages(int integ, double dt, double dt_e)
{
    double dte9 = 0.9 * dt_e;
    int s = (integ == OR_RKL2) ? 3 : 1;
    for (;; s += 2) {
        double ds = (double)s;
        double bound = (integ == OR_RKL2) ? (ds * ds + ds - 2.0) / 4.0 * dte9 : (ds * ds + ds) / 2.0 * dte9;
        if (bound >= dt) return s;
        if (s > 100001) return s;
    }
}

int or_order(int integ)
{
    switch (integ) {
    case OR_FEULER: return 1;
    case OR_SSP2: return 2;
    case OR_SSP104: return 4;
    case OR_RKL1: return 1;
    default: return 2;
    }
}

/* Weighted l2 norm (Eq. error_norm) with the DoF count of Sec. 3.3: phase
   entries count only where e_i != 0; a cell without such entries counts as 2;
   every concentration entry counts. */
static double weighted_norm(const or_sys *S, const or_tol *tol, const double *un,
                            const double *unew, const double *e, long *ndof)
{
    long V = S->V;
    double sum = 0.0;
    long cnt = 0;
    for (long i = 0; i < V; ++i) {
        long nc = 0;
        for (int a = 0; a < S->N; ++a) {
            long k = a * V + i;
            if (e[k] != 0.0) {
                double w = tol->r_phi * fmax(fabs(un[k]), fabs(unew[k])) + tol->a_phi;
                double q = e[k] / w;
                sum = sum + q * q;
                nc++;
            }
        }
        cnt += (nc > 0) ? nc : (S->N > 0 ? 2 : 0);
        for (int a = S->N; a < S->N + S->K; ++a) {
            long k = a * V + i;
            double w = tol->r_c * fmax(fabs(un[k]), fabs(unew[k])) + tol->a_c;
            double q = e[k] / w;
            sum = sum + q * q;
            cnt++;
        }
    }
    if (ndof) *ndof = cnt;
    return sqrt(sum / (double)cnt);
}

/* Sommeijer-type estimate (Sec. 3.3, sign read so that it is a local error):
   e = (12 (u^n - u^{n+1}) + 6 dt (F^n + F^{n+1})) / 15; phase entries whose
   trial u^n + dt/2 (F^n + F^{n+1}) leaves [0,1] carry zero error. */
double or_err_sts(const or_sys *S, const or_tol *tol, double dt, const double *un,
                  const double *unew, const double *rn, const double *rn1, long *ndof)
{
    long n = S->n, nphi = (long)S->N * S->V;
    double *e = malloc(sizeof(double) * n);
    for (long k = 0; k < n; ++k) {
        double sr = rn[k] + rn1[k];
        double ek = (12.0 * (un[k] - unew[k]) + (6.0 * dt) * sr) / 15.0;
        if (k < nphi) {
            double trial = un[k] + (dt / 2.0) * sr;
            if (trial < 0.0 || trial > 1.0) ek = 0.0;
        }
        e[k] = ek;
    }
    double r = weighted_norm(S, tol, un, unew, e, ndof);
    free(e);
    return r;
}

/* Embedded estimate e = u - z (Sec. 3.3); the phase filter uses z as trial. */
double or_err_embedded(const or_sys *S, const or_tol *tol, const double *un,
                       const double *unew, const double *z, long *ndof)
{
    long n = S->n, nphi = (long)S->N * S->V;
    double *e = malloc(sizeof(double) * n);
    for (long k = 0; k < n; ++k) {
        double ek = unew[k] - z[k];
        if (k < nphi && (z[k] < 0.0 || z[k] > 1.0)) ek = 0.0;
        e[k] = ek;
    }
    double r = weighted_norm(S, tol, un, unew, e, ndof);
    free(e);
    return r;
}

void or_ctrl_init(or_ctrl *c)
{
    c->b = 0.9; c->E1 = c->E2 = 0.0; c->dt1 = c->dt2 = 0.0; c->nhist = 0;
}

/* PID controller with bias (Sec. 3.3, Soderlind 2006 form):
   E_n = e/b, F = (E_n^-k1 E_{n-1}^-k2 E_{n-2}^-k3)^(1/(P+1)) (dt_n/dt_{n-1})^k4
   (dt_{n-1}/dt_{n-2})^k5, dt_{n+1} = dt_n (1 + 5 atan((F-1)/5)); missing
   history terms dropped; on rejection a proposed increase falls back to
   E_n^(-k1/(P+1)); bias squared on reject (>= 0.1), square-rooted on accept
   (<= 0.98).  E is floored at 1e-10 so that a vanishing error stays finite. */
double or_ctrl_update(or_ctrl *c, double err, double dt, int P, int *accept)
{
    const double k1 = 1.25, k2 = 0.5, k3 = -0.6, k4 = 0.25, k5 = 0.0;
    double ex = 1.0 / (double)(P + 1);
    double E = err / c->b;
    if (E < 1e-10) E = 1e-10;
    double F = pow(E, -k1 * ex);
    if (c->nhist >= 1) F = F * pow(c->E1, -k2 * ex) * pow(dt / c->dt1, k4);
    if (c->nhist >= 2) F = F * pow(c->E2, -k3 * ex) * pow(c->dt1 / c->dt2, k5);
    int acc = err < 1.0;
    if (acc) {
        c->E2 = c->E1; c->E1 = E;
        c->dt2 = c->dt1; c->dt1 = dt;
        if (c->nhist < 2) c->nhist++;
        double nb = sqrt(c->b);
        c->b = nb > 0.98 ? 0.98 : nb;
    } else {
        double nb = c->b * c->b;
        c->b = nb < 0.1 ? 0.1 : nb;
        if (F > 1.0) F = pow(E, -k1 * ex);
    }
    *accept = acc;
    return dt * (1.0 + 5.0 * atan((F - 1.0) / 5.0));
}

/* ---- driver ------------------------------------------------------------ */
/* Size h, stage count s and "lands on t_end" flag of the next attempt, given
   the proposed step dt and the remaining time rem (Sec. 3.2 stage rule;
   Sec. 5 output at target times).  Adaptive: a proposal within 1e-9 of the
   remaining time is stretched onto it.  Fixed: step kfix + 1 of nfix; the
   last one is shortened to land on t_end.  An RKL step that needs more than
   max_stages stages is refused for fixed steps (OR_EINVAL) and cut to the
   largest step that max_stages (rounded up to odd) allows for adaptive ones. */
static int plan_attempt(int integ, int adaptive, double dt, double rem, long kfix, long nfix,
                        double dte, int ssp_stages, int max_stages, double *h, int *s, int *last)
{
    int sts = (integ == OR_RKL1 || integ == OR_RKL2);
    *last = 0;
    if (adaptive) {
        *h = dt;
        if (*h >= rem * (1.0 - 1e-9)) { *h = rem; *last = 1; }
    } else {
        *last = (kfix + 1 >= nfix);
        *h = *last ? rem : dt;
    }
    *s = sts ? or_sts_stages(integ, *h, dte) : (integ == OR_SSP2 ? ssp_stages : (integ == OR_SSP104 ? 10 : 1));
    if (sts && *s > max_stages && !adaptive) return OR_EINVAL;
    if (sts && *s > max_stages) {
        *s = max_stages | 1;
        double ds = (double)*s;
        *h = (integ == OR_RKL2 ? (ds * ds + ds - 2.0) / 4.0 : (ds * ds + ds) / 2.0) * 0.9 * dte;
        *last = 0;
    }
    return OR_OK;
}

int or_drive(int integ, double dte, double t_end, double dt0, int max_stages, int n_err,
             const double *errs, const double *h_given, double *t, or_ctrl *ctrl, double *dt_next,
             int cap, double *tr_dt, int *tr_s, int *tr_acc)
{
    if (max_stages <= 0) max_stages = 1001;
    double dt = *dt_next > 0.0 ? *dt_next : (dt0 > 0.0 ? dt0 : 0.9 * dte);
    int k = 0;
    while (*t < t_end && k < n_err) {
        double h;
        int s, last, acc;
        plan_attempt(integ, 1, dt, t_end - *t, 0, 0, dte, 0, max_stages, &h, &s, &last);
        if (k < cap) tr_dt[k] = h;
        if (h_given) h = h_given[k];       /* continue from the step actually taken */
        dt = or_ctrl_update(ctrl, errs[k], h, or_order(integ), &acc);
        if (k < cap) { tr_s[k] = s; tr_acc[k] = acc; }
        k++;
        if (acc) *t = last ? t_end : *t + h;
    }
    *dt_next = dt;
    return k;
}

int or_run(const or_params *p, int integ, double t_end, const or_tol *tol,
           double dt_mult, double dt0, int ssp_stages, int max_stages,
           double *u, double *t, or_ctrl *ctrl, or_stats *st,
           int cap, double *tr_dt, int *tr_s, double *tr_err, int *tr_acc, int *tr_len,
           int replay_n, const double *replay_dt, const int *replay_s, const int *replay_acc)
{
    or_sys S;
    or_sys_pde(&S, p);
    long n = S.n;
    double dte = or_dt_e(p);
    int adaptive = !(dt_mult > 0.0);
    int sts = (integ == OR_RKL1 || integ == OR_RKL2);
    if (adaptive && (integ == OR_FEULER || integ == OR_SSP2) && replay_n == 0) return OR_EINVAL;
    if (max_stages <= 0) max_stages = 1001;
    double *unew = malloc(sizeof(double) * n), *rn = malloc(sizeof(double) * n),
           *rn1 = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
    int status = OR_OK, ntr = 0, attempt = 0;
    double dt = adaptive ? (st->dt_next > 0.0 ? st->dt_next : (dt0 > 0.0 ? dt0 : 0.9 * dte)) : dt_mult * dte;
    /* fixed steps: the k-th step ends at t0 + k dt (no accumulated drift) and
       the last one is shortened to land on t_end (Sec. 5) */
    double t0 = *t;
    long nfix = 0, kfix = 0;
    if (!adaptive) {
        nfix = (long)ceil((t_end - t0) / dt - 1e-9);
        if (nfix < 1) nfix = 1;
    }
    while (*t < t_end) {
        double rem = t_end - *t, h;
        int s, last = 0;
        if (replay_n > 0) {
            if (attempt >= replay_n) break;
            h = replay_dt[attempt];
            s = replay_s[attempt];
            last = (h >= rem * (1.0 - 1e-9));
        } else if (plan_attempt(integ, adaptive, dt, rem, kfix, nfix, dte, ssp_stages, max_stages,
                                &h, &s, &last) != OR_OK) {
            status = OR_EINVAL;
            break;
        }
        long ev = or_step(&S, integ, h, s, u, unew, rn, integ == OR_SSP104 ? z : NULL);
        if (ev < 0) { status = ev == -2 ? OR_EUNSTABLE : OR_EINVAL; break; }
        st->rhs_evals += ev;
        double err = 0.0;
        int acc = 1;
        if (adaptive || replay_n > 0) {
            if (sts) {
                or_rhs(p, unew, rn1, NULL);
                st->rhs_evals++;
                err = or_err_sts(&S, tol, h, u, unew, rn, rn1, NULL);
            } else if (integ == OR_SSP104) {
                err = or_err_embedded(&S, tol, u, unew, z, NULL);
            }
            if (!isfinite(err)) { status = OR_EUNSTABLE; break; }
            if (replay_n > 0) {
                acc = replay_acc[attempt];
                int dummy;
                if (adaptive) dt = or_ctrl_update(ctrl, err, h, or_order(integ), &dummy);
            } else {
                dt = or_ctrl_update(ctrl, err, h, or_order(integ), &acc);
            }
        }
        if (ntr < cap) {
            if (tr_dt) tr_dt[ntr] = h;
            if (tr_s) tr_s[ntr] = s;
            if (tr_err) tr_err[ntr] = err;
            if (tr_acc) tr_acc[ntr] = acc;
            ntr++;
        }
        attempt++;
        if (acc) {
            memcpy(u, unew, sizeof(double) * n);
            if (!adaptive && replay_n == 0) { kfix++; *t = last ? t_end : t0 + (double)kfix * dt; }
            else *t = last ? t_end : *t + h;
            st->accepted++;
        } else {
            st->rejected++;
        }
        st->dt_last = h;
        st->err_last = err;
        if (st->rejected > 100000) { status = OR_EUNSTABLE; break; }
    }
    st->dt_next = adaptive ? dt : 0.0;
    if (tr_len) *tr_len = ntr;
    free(unew); free(rn); free(rn1); free(z);
    return status;
}
