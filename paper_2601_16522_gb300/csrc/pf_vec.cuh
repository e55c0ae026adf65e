// pf_vec.cuh -- the FP32 dense stage passes with two cells per thread.
//
// Hot passes of FP32 dense storage (N <= 128 phases, nx even; Sec. 3 finite
// differences, Sec. 3.1 projection, Sec. 3.2 stage combinations, Sec. 3.3
// error sweep).  Every thread owns two x-adjacent cells (x, x + 1), so each
// load and store of a phase plane moves a float2 (a warp covers 64
// consecutive cells, 256 B), the x neighbours inside the pair come from the
// pair itself and across lanes from warp shuffles, and the address
// arithmetic of a phase is shared by both cells.
//
// The stage value of a phase that is not nontrivial at a cell (the n(phi)
// filter of Eq. phieq) has a zero RHS, so after the first sweep it is final
// up to the projection's normalisation and is written at once; only the
// nontrivial phases (at most VACT per cell, in a shared-memory list) wait for
// the pairwise sums.  The normalisation rewrites an already written entry
// only where it is nonzero and the cell's simplex sum is not exactly one (or
// the >= 1 rule changed the cell): bulk cells, whose sum is exactly one, and
// zero entries are never touched again.  No per-phase register array is
// needed, so the phase loop is rolled and the next phase's loads are issued
// before the current phase is processed.  A cell with more than VACT
// nontrivial phases is recomputed on the wide path.  The arithmetic is that
// of fast_cell (the same combination, projection, fix and error terms); the
// concentration sums are formed per chemical type, so rounding differs from
// the other FP32 kernels (FP32 is not compared bit for bit).
#pragma once
#include "pf_kernels.cuh"

namespace pfk {

constexpr int VTX = 32;              // threads along x: 64 cells
// Rows per block (4; measured at 256^3 x 32: 2 rows at 10/14 blocks per SM
// and 8 rows at 2/3 give RKL2 passes of 2.13 and 2.43 ms against 2.11 ms).
#ifndef PF_VEC_TY
#define PF_VEC_TY 4
#endif
constexpr int VTY = PF_VEC_TY;       // rows per block
constexpr int VBLOCK = VTX * VTY;    // 128 threads
constexpr int VCELLS = 2 * VBLOCK;   // 256 cells per block
// List capacity per cell: passes with two extra pointwise streams (RKL2 body)
// run fewer blocks per SM and keep 8 entries; the lighter passes keep 6 so
// that more blocks fit in shared memory (a cell with more goes to the wide
// pass; in grain growth fewer than 0.05 % of cells have more than 6).
#ifndef PF_VEC_ACT
#define PF_VEC_ACT 8
#endif
#ifndef PF_VEC_ACT_LIGHT
#define PF_VEC_ACT_LIGHT 6
#endif
// Resident blocks per SM the register budget targets.
#ifndef PF_VEC_MINB
#define PF_VEC_MINB 5
#endif
#ifndef PF_VEC_MINB_LIGHT
#define PF_VEC_MINB_LIGHT 7
#endif
// Phases ahead whose planes are prefetched into L2 (0: none).
#ifndef PF_VEC_PREFETCH
#define PF_VEC_PREFETCH 4
#endif
// ... for the passes with fewer pointwise streams
#ifndef PF_VEC_PREFETCH_LIGHT
#define PF_VEC_PREFETCH_LIGHT 0
#endif
// Register double buffering of the phase loads (1) or one phase at a time (0).
#ifndef PF_VEC_DB
#define PF_VEC_DB 1
#endif

// Blocks of the x-y plane of the two-cell kernels (one z plane per block).
__host__ __device__ inline long long vec_tiles(const Geom &g)
{
    return (long long)((g.nx + 2 * VTX - 1) / (2 * VTX)) * ((g.ny + VTY - 1) / VTY);
}

// Whether the two-cell kernels can run a problem (dense FP32 storage).
__host__ __device__ inline bool vec_eligible(const Geom &g)
{
    return (g.nx % 2) == 0 && g.N <= 128 && g.V < 0x7fffffffLL;
}

// Whether a pass is one of the heavy ones (two extra pointwise streams).
template <unsigned SIG>
__host__ __device__ constexpr bool vec_heavy() { return (SIG & (SIG_P0 | SIG_P2)) == (SIG_P0 | SIG_P2); }

template <unsigned SIG>
__host__ __device__ constexpr int vec_act() { return vec_heavy<SIG>() ? PF_VEC_ACT : PF_VEC_ACT_LIGHT; }

template <int ACT>
struct VecSmem {
    unsigned char id[ACT][VCELLS];
    float lap[ACT][VCELLS];    // Laplacian, later the RHS of the listed phase
    float cen[ACT][VCELLS];    // phi at the cell
    float dl[ACT][VCELLS];     // variational derivative
    float val[ACT][VCELLS];    // stage value before the RHS term
};

// Dynamic shared memory of a two-cell pass.
template <unsigned SIG>
__host__ __device__ constexpr size_t vec_smem() { return sizeof(VecSmem<vec_act<SIG>()>); }

__device__ __forceinline__ float2 ldg2(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }

__device__ __forceinline__ float2 ld_stream2(const float *p)
{
    float2 v;
    asm("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}

__device__ __forceinline__ void st2(float *p, float a, float b) { *reinterpret_cast<float2 *>(p) = make_float2(a, b); }

// three-input minimum and maximum (sm_100+ PTX)
__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Loads of one phase for the thread's two cells.
struct VPhase {
    float2 c, ym, yp, zm, zp;  // stencil input at the pair and its y/z neighbours
    float el, er;              // x neighbours across the tile edge (edge lanes only)
    float2 p0, p2, r0;         // pointwise inputs
};

// Per-cell state of the sweep over the phases.
struct VCell {
    int nz, bestid, nc;
    float best, ssum;
    bool changed;
    int nzcnt;                 // phases not listed written with a nonzero value
    double es;                 // error partial (MODE_ERR)
    long long ec;
};

// One block of a two-cell pass: tile (bx, by) of plane bz, one of nblk
// blocks of the pass (a packed launch maps its blocks to several problems).
template <int DIM, int KC, unsigned SIG>
__device__ __forceinline__ void vec_body(const Geom &g, const Pass<float> &P, const float *__restrict__ tabA,
                                         const float *__restrict__ tabB, const float *__restrict__ tabL,
                                         const signed char *__restrict__ ptype, int bx, int by, int bz, int nblk)
{
    typedef float T;
    constexpr bool ERR = (SIG & SIG_ERR) != 0;
    constexpr bool HP0 = (SIG & SIG_P0) != 0 || ERR;
    constexpr bool HP2 = (SIG & SIG_P2) != 0;
    constexpr bool HR0 = (SIG & SIG_R0IN) != 0 || ERR;
    constexpr bool R0OUT = (SIG & SIG_R0OUT) != 0;
    constexpr bool PROJ = (SIG & SIG_PROJECT) != 0;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    if (pass_skipped(P.flag)) return;
    constexpr int VACT = vec_act<SIG>();   // nontrivial phases per cell in the shared-memory list
    VecSmem<VACT> &S = *reinterpret_cast<VecSmem<VACT> *>(smem_raw);
    const int tid = threadIdx.x;
    const int lane = tid & 31, ty = tid >> 5;
    const int tiles_x = (g.nx + 2 * VTX - 1) / (2 * VTX), tiles_y = (g.ny + VTY - 1) / VTY;
    const int bid = bx + tiles_x * (by + tiles_y * bz);
    const int x = bx * (2 * VTX) + 2 * lane;
    const int y = by * VTY + ty;
    const int z = bz;
    const int N = g.N;
    const int Vs = (int)g.Vs;
    VCell C[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        C[c].nz = 0; C[c].bestid = -1; C[c].nc = 0; C[c].best = (T)-1; C[c].ssum = (T)0;
        C[c].changed = false; C[c].nzcnt = 0; C[c].es = 0.0; C[c].ec = 0;
    }
    bool crowd[2] = {false, false};
    if (y < g.ny) {   // warp-uniform (a warp is one row)
        const bool here = x < g.nx;
        const int i = (z * g.ny + y) * g.nx + x;
        // lanes past nx load the last pair of their row (in bounds, unused)
        const int il = here ? i : (z * g.ny + y) * g.nx + (g.nx - 2);
        // y / z neighbour offsets (a zero-gradient ghost is the cell itself)
        long long off64[6];
        int ghost[6];
        face_offsets(g, x, y, z, off64, ghost);
        const int oym = ghost[2] ? 0 : (int)off64[2], oyp = ghost[3] ? 0 : (int)off64[3];
        const int ozm = DIM == 3 ? (ghost[4] ? 0 : (int)off64[4]) : 0;
        const int ozp = DIM == 3 ? (ghost[5] ? 0 : (int)off64[5]) : 0;
        // x neighbours of the pair: left of cell x, right of cell x + 1
        const bool lsh = lane > 0;                          // from lane - 1 (cell x - 1)
        const bool rsh = lane < 31 && x + 2 < g.nx;         // from lane + 1 (cell x + 2)
        const bool lself = !lsh && x == 0 && g.bc_phi[0] != BC_PERIODIC;
        const bool rself = !rsh && x + 2 >= g.nx && g.bc_phi[1] != BC_PERIODIC;
        const bool lneed = here && !lsh && !lself, rneed = here && !rsh && !rself;
        const int lofs = x > 0 ? -1 : g.nx - 1;
        const int rofs = x + 2 < g.nx ? 2 : 2 - g.nx;
        const T idx2 = (T)(1.0 / g.dx2);
        const T a0c = (T)P.a0, a2c = (T)P.a2, b1c = (T)P.b1, b0c = (T)P.b0;
        const T ib1 = (T)(1.0 / P.b1);
        const T dt = (T)P.dt, rph = (T)P.r_phi, aph = (T)P.a_phi;

        // concentration: per chemical type, phase sums of the two cells, of
        // their y/z neighbours and of the x edge cells
        T Ph[2][2], Pn[2][4][2], Pe[2][2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            Ph[0][t] = Ph[1][t] = Pe[0][t] = Pe[1][t] = (T)0;
#pragma unroll
            for (int f = 0; f < 4; ++f) Pn[0][f][t] = Pn[1][f][t] = (T)0;
        }

        // per-thread 32-bit element offsets inside a phase plane; the phase
        // bases below are the same for every thread (uniform)
        const int oc = il, oym_ = il + oym, oyp_ = il + oyp, ozm_ = il + ozm, ozp_ = il + ozp;
        const int oel = il + lofs, oer = il + rofs;
        auto fetch = [&](int a, VPhase &q) {
            const long long pb = (long long)a * Vs;
            const float *b = P.in + pb;
            constexpr int PD = (HP0 && HP2) ? PF_VEC_PREFETCH : PF_VEC_PREFETCH_LIGHT;
            if (PD > 0 && a + PD < N) {
                const long long pa = pb + (long long)PD * Vs;
                prefetch_l2(P.in + pa + oc);
                if (HP0) prefetch_l2(P.p0 + pa + oc);
                if (HP2) prefetch_l2(P.p2 + pa + oc);
                if (HR0) prefetch_l2(P.r0in + pa + oc);
            }
            q.c = ldg2(b + oc);
            q.ym = ldg2(b + oym_);
            q.yp = ldg2(b + oyp_);
            if (DIM == 3) {
                q.zm = ldg2(b + ozm_);
                q.zp = ldg2(b + ozp_);
            }
            if (HP0) q.p0 = ld_stream2(P.p0 + pb + oc);
            if (HP2) q.p2 = ld_stream2(P.p2 + pb + oc);
            if (HR0) q.r0 = ld_stream2(P.r0in + pb + oc);
            if (lneed) q.el = __ldg(b + oel);
            if (rneed) q.er = __ldg(b + oer);
        };

        // one phase at one cell: activity, list entry, stage value (returned)
        auto cell_phase = [&](VCell &Cc, int slot, int a, T v, T xl, T xr, T ym, T yp, T zm, T zp, T p0v, T p2v,
                              T r0v) -> T {
            // every input +0 (most phases of most cells): the phase is not
            // nontrivial, its stage value is exactly +0, it adds nothing to the
            // sum, the count or the error -- the result of the steps below
            unsigned bits = __float_as_uint(v) | __float_as_uint(xl) | __float_as_uint(xr) | __float_as_uint(ym) |
                            __float_as_uint(yp);
            if (DIM == 3) bits |= __float_as_uint(zm) | __float_as_uint(zp);
            if (HP0) bits |= __float_as_uint(p0v);
            if (HP2) bits |= __float_as_uint(p2v);
            if (HR0) bits |= __float_as_uint(r0v);
            if (bits == 0u) return (T)0;
            T mx, mn;
            if (DIM == 3) {
                mx = fmax3(fmax3(v, xl, xr), fmax3(ym, yp, zm), zp);
                mn = fmin3(fmin3(v, xl, xr), fmin3(ym, yp, zm), zp);
            } else {
                mx = fmax3(fmax3(v, xl, xr), ym, yp);
                mn = fmin3(fmin3(v, xl, xr), ym, yp);
            }
            const bool act = mx > (T)0 && mn < (T)1;
            T acc = (T)0;
            if (!ERR) {
                acc = affine<HP0, HP2>(v, p0v, p2v, a0c, a2c);
                if (HR0) acc = acc + b0c * r0v;
            }
            if (act) {
                if (Cc.nz < VACT) {
                    const T l = DIM == 3 ? (((xl + xr) + (ym + yp)) + (zm + zp)) - (T)6 * v
                                         : ((xl + xr) + (ym + yp)) - (T)4 * v;
                    S.id[Cc.nz][slot] = (unsigned char)a;
                    S.lap[Cc.nz][slot] = l * idx2;
                    S.cen[Cc.nz][slot] = v;
                    if (!ERR) S.val[Cc.nz][slot] = acc;
                }
                Cc.nz++;
            } else if (ERR) {
                // in = u^{n+1}, p0 = u^n, r0in = F^n; a trivial phase has F^{n+1} = 0
                T e = ((T)12 * (p0v - v) + ((T)6 * dt) * r0v) * ((T)1 / (T)15);
                const T trial = p0v + (dt * (T)0.5) * r0v;
                if (trial < (T)0 || trial > (T)1) e = (T)0;
                if (e != (T)0) {
                    const T w = rph * fmaxf(fabsf(p0v), fabsf(v)) + aph;
                    const T q = e / w;
                    Cc.es += (double)(q * q);
                    Cc.nc++;
                }
            } else if (PROJ) {
                if (acc < (T)0) { acc = (T)0; Cc.changed = true; }
                if (acc >= (T)1 && acc > Cc.best) { Cc.best = acc; Cc.bestid = a; }
                Cc.ssum = Cc.ssum + acc;
                if (acc != (T)0) Cc.nzcnt++;
            }
            return acc;
        };

        // ---- the sweep over the phases ---------------------------------------
        auto process = [&](int a, const VPhase &q) {
            const float sl = __shfl_up_sync(0xffffffffu, q.c.y, 1);
            const float sr = __shfl_down_sync(0xffffffffu, q.c.x, 1);
            const T left = lsh ? sl : (lself ? q.c.x : q.el);
            const T right = rsh ? sr : (rself ? q.c.y : q.er);
            const T zm0 = DIM == 3 ? q.zm.x : (T)0, zm1 = DIM == 3 ? q.zm.y : (T)0;
            const T zp0 = DIM == 3 ? q.zp.x : (T)0, zp1 = DIM == 3 ? q.zp.y : (T)0;
            const T p00 = HP0 ? q.p0.x : (T)0, p01 = HP0 ? q.p0.y : (T)0;
            const T p20 = HP2 ? q.p2.x : (T)0, p21 = HP2 ? q.p2.y : (T)0;
            const T r00 = HR0 ? q.r0.x : (T)0, r01 = HR0 ? q.r0.y : (T)0;
            if (here) {
                const T w0 = cell_phase(C[0], tid, a, q.c.x, left, q.c.y, q.ym.x, q.yp.x, zm0, zp0, p00, p20, r00);
                const T w1 = cell_phase(C[1], VBLOCK + tid, a, q.c.y, q.c.x, right, q.ym.y, q.yp.y, zm1, zp1, p01,
                                        p21, r01);
                const long long pb = (long long)a * Vs;
                if (!ERR) st2(P.out + pb + i, w0, w1);
                if (R0OUT) st2(P.r0out + pb + i, (T)0, (T)0);   // listed phases get theirs below
                if (KC) {
                    const int t = ptype[a];
                    // per-type sums: own cells, y/z neighbours, edge cells
                    Ph[0][t] += q.c.x;
                    Ph[1][t] += q.c.y;
                    Pn[0][0][t] += q.ym.x; Pn[1][0][t] += q.ym.y;
                    Pn[0][1][t] += q.yp.x; Pn[1][1][t] += q.yp.y;
                    if (DIM == 3) {
                        Pn[0][2][t] += zm0; Pn[1][2][t] += zm1;
                        Pn[0][3][t] += zp0; Pn[1][3][t] += zp1;
                    }
                    if (lneed) Pe[0][t] += q.el;
                    if (rneed) Pe[1][t] += q.er;
                }
            }
        };
        // two phases per iteration: the loads of the next phase are in flight
        // while the current one is processed, without register copies
        if (PF_VEC_DB) {
            VPhase qa, qb;
            fetch(0, qa);
            int a = 0;
#pragma unroll 1
            for (; a + 1 < N; a += 2) {
                fetch(a + 1, qb);
                process(a, qa);
                if (a + 2 < N) fetch(a + 2, qa);
                process(a + 1, qb);
            }
            if (a < N) process(a, qa);
        } else {
#pragma unroll 1
            for (int a = 0; a < N; ++a) {
                VPhase q;
                fetch(a, q);
                process(a, q);
            }
        }

        // ---- concentration: mu of the cells and their neighbours, c RHS ------
        T mu[2] = {(T)0, (T)0}, rc[2] = {(T)0, (T)0}, cc[2] = {(T)0, (T)0};
        if (KC) {
            const T c00 = (T)g.c0[0], c01 = (T)g.c0[1], ik0 = (T)g.invk[0], ik1 = (T)g.invk[1];
            const T dk0 = (T)g.Dk[0], dk1 = (T)g.Dk[1];
            const float *cf = P.in + (long long)N * Vs + i;
            float2 c2 = make_float2(0.f, 0.f), cym = c2, cyp = c2, czm = c2, czp = c2;
            float cel = 0.f, cer = 0.f;
            if (here) {
                c2 = ldg2(cf);
                cym = ldg2(cf + oym);
                cyp = ldg2(cf + oyp);
                if (DIM == 3) {
                    czm = ldg2(cf + ozm);
                    czp = ldg2(cf + ozp);
                }
            }
            if (lneed) cel = __ldg(cf + lofs);
            if (rneed) cer = __ldg(cf + rofs);
            cc[0] = c2.x;
            cc[1] = c2.y;
            auto muof = [&](T cv, const T *ph) { return (cv - (c00 * ph[0] + c01 * ph[1])) / (ph[0] * ik0 + ph[1] * ik1); };
            auto mof = [&](const T *ph) { return ph[0] * dk0 + ph[1] * dk1; };
            T M[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                mu[c] = muof(cc[c], Ph[c]);
                M[c] = mof(Ph[c]);
            }
            // x neighbours: inside the pair, across lanes, or the edge cells
            const T mul_s = __shfl_up_sync(0xffffffffu, mu[1], 1), Ml_s = __shfl_up_sync(0xffffffffu, M[1], 1);
            const T mur_s = __shfl_down_sync(0xffffffffu, mu[0], 1), Mr_s = __shfl_down_sync(0xffffffffu, M[0], 1);
            T mul, Ml, mur, Mr;
            if (lsh) { mul = mul_s; Ml = Ml_s; }
            else if (lself) {
                // zero-gradient phi; c Dirichlet (ghost 2 c_b - c) or zero-gradient
                mul = g.bc_c[0] == BC_DIRICHLET ? muof((T)2 * (T)g.cdir[0] - cc[0], Ph[0]) : mu[0];
                Ml = M[0];
            } else { mul = muof(cel, Pe[0]); Ml = mof(Pe[0]); }
            if (rsh) { mur = mur_s; Mr = Mr_s; }
            else if (rself) {
                mur = g.bc_c[1] == BC_DIRICHLET ? muof((T)2 * (T)g.cdir[1] - cc[1], Ph[1]) : mu[1];
                Mr = M[1];
            } else { mur = muof(cer, Pe[1]); Mr = mof(Pe[1]); }
            const float2 cnb[4] = {cym, cyp, czm, czp};
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                T acc = (T)0;
                // x faces
                const T mxl = c == 0 ? mul : mu[0], Mxl = c == 0 ? Ml : M[0];
                const T mxr = c == 0 ? mu[1] : mur, Mxr = c == 0 ? M[1] : Mr;
                acc = acc + ((T)0.5 * (M[c] + Mxl)) * (mxl - mu[c]);
                acc = acc + ((T)0.5 * (M[c] + Mxr)) * (mxr - mu[c]);
                // y and z faces (face 2 + f of the cell)
#pragma unroll
                for (int f = 0; f < 2 * (DIM - 1); ++f) {
                    T cv = c == 0 ? cnb[f].x : cnb[f].y;
                    if (ghost[2 + f] && g.bc_c[2 + f] == BC_DIRICHLET) cv = (T)2 * (T)g.cdir[2 + f] - cc[c];
                    const T mun = muof(cv, Pn[c][f]);
                    acc = acc + ((T)0.5 * (M[c] + mof(Pn[c][f]))) * (mun - mu[c]);
                }
                rc[c] = acc * idx2;
            }
        }

        // ---- pairwise sums over each cell's list ----------------------------
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            VCell &Cc = C[c];
            const int slot = c * VBLOCK + tid;
            if (!here) continue;
            if (Cc.nz > VACT) { crowd[c] = true; continue; }
            const int nz = Cc.nz;
            for (int k = 0; k < nz; ++k) {
                const int a = S.id[k][slot];
                const T *Aa = tabA + a * N, *Ba = tabB + a * N;
                T d = (T)0;
                for (int k2 = 0; k2 < nz; ++k2) {
                    if (k2 == k) continue;
                    const int b = S.id[k2][slot];
                    d = d + (__ldg(Aa + b) * S.lap[k2][slot] + __ldg(Ba + b) * S.cen[k2][slot]);
                }
                if (KC) {
                    const int t = ptype[a];
                    d = d + (-(mu[c] * mu[c]) / ((T)2 * (T)g.k[t]) - mu[c] * (T)g.c0[t]);
                }
                S.dl[k][slot] = d;
            }
            const T inz = nz > 1 ? (T)1 / (T)nz : (T)0;
            for (int k = 0; k < nz; ++k) {
                T rk = (T)0;
                const int a = S.id[k][slot];
                if (nz > 1) {
                    const T *La = tabL + a * N;
                    const T dk = S.dl[k][slot];
                    T s = (T)0;
                    for (int k2 = 0; k2 < nz; ++k2) {
                        if (k2 == k) continue;
                        s = s + __ldg(La + S.id[k2][slot]) * (dk - S.dl[k2][slot]);
                    }
                    rk = -(s * inz);
                }
                S.lap[k][slot] = rk;              // the list now holds the RHS
                const long long fo = (long long)a * Vs + i + c;
                if (ERR) {
                    const T p0v = __ldg(P.p0 + fo), v0 = S.cen[k][slot], r0v = __ldg(P.r0in + fo);
                    const T sr = r0v + rk;
                    T e = ((T)12 * (p0v - v0) + ((T)6 * dt) * sr) * ((T)1 / (T)15);
                    const T trial = p0v + (dt * (T)0.5) * sr;
                    if (trial < (T)0 || trial > (T)1) e = (T)0;
                    if (e != (T)0) {
                        const T w = rph * fmaxf(fabsf(p0v), fabsf(v0)) + aph;
                        const T q = e / w;
                        Cc.es += (double)(q * q);
                        Cc.nc++;
                    }
                    if (R0OUT) P.r0out[fo] = rk;   // F(u^{n+1}) kept for reuse
                } else {
                    T acc = S.val[k][slot] + b1c * rk;
                    if (PROJ) {
                        if (acc < (T)0) { acc = (T)0; Cc.changed = true; }
                        if (acc >= (T)1 && (acc > Cc.best || (acc == Cc.best && a < Cc.bestid))) {
                            Cc.best = acc;
                            Cc.bestid = a;
                        }
                        Cc.ssum = Cc.ssum + acc;
                    }
                    S.val[k][slot] = acc;
                }
            }
        }

        // ---- projection, final values, concentration ------------------------
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            VCell &Cc = C[c];
            const int slot = c * VBLOCK + tid;
            if (!here || crowd[c]) continue;
            const int nz = Cc.nz;
            if (ERR) {
                Cc.ec += (Cc.nc > 0 ? Cc.nc : 2);
                if (KC) {
                    const long long o = (long long)N * Vs + i + c;
                    const T un = __ldg(P.p0 + o), un1 = cc[c], rn = __ldg(P.r0in + o);
                    const T e = ((T)12 * (un - un1) + ((T)6 * dt) * (rn + rc[c])) * ((T)1 / (T)15);
                    const T w = (T)P.r_c * fmaxf(fabsf(un + (T)g.cref), fabsf(un1 + (T)g.cref)) + (T)P.a_c;
                    const T q = e / w;
                    Cc.es += (double)(q * q);
                    Cc.ec += 1;
                    if (R0OUT) P.r0out[o] = rc[c];
                }
                continue;
            }
            bool rewrite = false;     // inactive nonzero entries need their final value
            if (PROJ) {
                if (Cc.bestid >= 0) {
                    // the winner becomes 1, the others 0: a change unless the
                    // winner is exactly 1 and every other phase already zero.
                    // Unlisted entries need rewriting only where nonzero
                    // (nzcnt of them, the winner among them if unlisted).
                    bool listed = false, others = false;
                    for (int k = 0; k < nz; ++k) {
                        if (S.id[k][slot] == Cc.bestid) listed = true;
                        else if (S.val[k][slot] != (T)0) others = true;
                    }
                    const int unl_others = Cc.nzcnt - (listed ? 0 : 1);
                    if (others || unl_others > 0 || Cc.best != (T)1) Cc.changed = true;
                    rewrite = unl_others > 0 || (!listed && Cc.best != (T)1);
                    Cc.ssum = (T)1;
                }
                if (!(Cc.ssum > (T)0)) raise_flag(P.flag, FLAG_SIMPLEX);
            }
            const T inv = (Cc.ssum > (T)0) ? (T)1 / Cc.ssum : (T)1;
            if (PROJ && Cc.bestid < 0 && inv != (T)1 && Cc.nzcnt > 0) rewrite = true;
            const bool fix = R0OUT && P.fix_first && Cc.changed;
            // listed phases
            for (int k = 0; k < nz; ++k) {
                const int a = S.id[k][slot];
                const long long fo = (long long)a * Vs + i + c;
                T w = S.val[k][slot];
                if (PROJ) w = (Cc.bestid >= 0) ? ((a == Cc.bestid) ? (T)1 : (T)0) : w * inv;
                P.out[fo] = w;
                if (R0OUT) {
                    T r = S.lap[k][slot];
                    if (fix) r = (w - S.cen[k][slot]) * ib1;
                    P.r0out[fo] = r;
                }
            }
            // phases not listed whose written value is nonzero (rare outside
            // bulk cells): the >= 1 rule or the normalisation
            if (rewrite) {
                int kk = 0;
                for (int a = 0; a < N; ++a) {
                    if (kk < nz && S.id[kk][slot] == a) { kk++; continue; }
                    const long long fo = (long long)a * Vs + i + c;
                    const T o = P.out[fo];
                    if (o == (T)0) continue;
                    const T w = (Cc.bestid >= 0) ? ((a == Cc.bestid) ? (T)1 : (T)0) : o * inv;
                    P.out[fo] = w;
                    if (fix) P.r0out[fo] = (w - __ldg(P.in + fo)) * ib1;
                }
            }
            if (KC) {
                const long long o = (long long)N * Vs + i + c;
                // the small increments are summed first: c is rounded once per stage
                T d = b1c * rc[c];
                if (HR0) d = d + b0c * __ldg(P.r0in + o);
                if (HP0) d = d + a0c * (__ldg(P.p0 + o) - cc[c]);
                if (HP2) d = d + a2c * (__ldg(P.p2 + o) - cc[c]);
                const T acc = cc[c] + d;
                if (!isfinite(acc)) raise_flag(P.flag, FLAG_NONFINITE);
                if (R0OUT) P.r0out[o] = rc[c];
                P.out[o] = acc;
            }
        }
    }
    // crowded cells (more than VACT nontrivial phases): recorded for the wide
    // pass that follows (wide_fix_kernel); their outputs and error terms come
    // from there.  The block appends one entry: its index and a 256-bit mask.
    __shared__ unsigned cmask[VCELLS / 32];
    if (tid < VCELLS / 32) cmask[tid] = 0u;
    if (__syncthreads_or(crowd[0] || crowd[1])) {
#pragma unroll
        for (int c = 0; c < 2; ++c)
            if (crowd[c]) {
                const int bit = ty * (2 * VTX) + 2 * lane + c;
                atomicOr(&cmask[bit >> 5], 1u << (bit & 31));
            }
        __syncthreads();
        if (tid == 0) {
            const int e = atomicAdd(P.crowd, 1);
            int *ent = P.crowd + 2 + e * (1 + VCELLS / 32);
            ent[0] = bid;
#pragma unroll
            for (int w = 0; w < VCELLS / 32; ++w) ent[1 + w] = (int)cmask[w];
        }
    }
    if (ERR) block_partials(C[0].es + C[1].es, C[0].ec + C[1].ec, P.part_sum, P.part_cnt, bid, P.part_n, nblk);
    // the step is counted by the wide pass, after the crowded cells
}

// The wide pass after a two-cell pass: every crowded cell recorded by the
// two-cell blocks is recomputed by the generic body with the WIDEACT-entry
// list (wide_cell), which rewrites all of that cell's outputs; the block's
// error terms are added to its partial in a fixed order (cells ascending),
// so the norm stays deterministic.  Blocks take the recorded entries in a
// grid-stride loop; the last block to finish clears the record and, for a
// pass that completes a fixed step, counts the step.  It runs after every
// two-cell pass (with no entries it only does the bookkeeping).
constexpr int WIDE_FIX_BLOCKS = 152;

// The recorded entries e = w, w + nw, ... of one two-cell pass.
template <int DIM, int KC>
__device__ __forceinline__ void wide_fix_entries(const Geom &g, const Pass<float> &P, const float *tabA,
                                                 const float *tabB, const float *tabL, const signed char *ptype,
                                                 int w, int nw)
{
    __shared__ double rs[VCELLS];
    __shared__ long long rc[VCELLS];
    const int n = *(volatile int *)P.crowd;
    const int tid = threadIdx.x;
    const int tiles_x = (g.nx + 2 * VTX - 1) / (2 * VTX), tiles_y = (g.ny + VTY - 1) / VTY;
    for (int e = w; e < n; e += nw) {
        const int *ent = P.crowd + 2 + e * (1 + VCELLS / 32);
        const int b = ent[0];
        const unsigned m = (unsigned)ent[1 + (tid >> 5)];
        double es = 0.0;
        long long ec = 0;
        if ((m >> (tid & 31)) & 1u) {
            const int bx = b % tiles_x, by = (b / tiles_x) % tiles_y, bz = b / (tiles_x * tiles_y);
            const int x = bx * (2 * VTX) + (tid % (2 * VTX)), y = by * VTY + tid / (2 * VTX);
            wide_cell<float, DIM, KC>(&g, &P, tabA, tabB, tabL, ptype, x, y, bz, &es, &ec);
        }
        if (P.mode == MODE_ERR) {
            rs[tid] = es;
            rc[tid] = ec;
            __syncthreads();
            if (tid == 0) {
                double s = 0.0;
                long long c = 0;
                for (int k = 0; k < VCELLS; ++k) { s += rs[k]; c += rc[k]; }
                P.part_sum[b] += s;
                P.part_cnt[b] += c;
            }
            __syncthreads();
        }
    }
}

// After every block of the wide pass: clear the record and, for a pass
// that completes a fixed step without a flag, count the step.
__device__ __forceinline__ void wide_fix_close(const Pass<float> &P)
{
    atomicExch(P.crowd, 0);
    atomicExch(P.crowd + 1, 0);
    if (P.count_step && !pass_skipped(P.flag)) atomicAdd(P.flag + 1, 1);
}

template <int DIM, int KC>
__device__ __forceinline__ void wide_fix_body(const Geom &g, const Pass<float> &P, const float *tabA,
                                              const float *tabB, const float *tabL, const signed char *ptype)
{
    wide_fix_entries<DIM, KC>(g, P, tabA, tabB, tabL, ptype, blockIdx.x, gridDim.x);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(P.crowd + 1, 1) == (int)gridDim.x - 1) wide_fix_close(P);
    }
}

template <int DIM, int KC>
__global__ void __launch_bounds__(VCELLS)
wide_fix_kernel(const __grid_constant__ Geom g, const __grid_constant__ Pass<float> P, const float *__restrict__ tabA,
                const float *__restrict__ tabB, const float *__restrict__ tabL, const signed char *__restrict__ ptype)
{
    wide_fix_body<DIM, KC>(g, P, tabA, tabB, tabL, ptype);
}

template <int DIM, int KC>
__global__ void __launch_bounds__(VCELLS)
wide_fix_kernel_d(const __grid_constant__ Geom g, const Pass<float> *__restrict__ Pd, const float *__restrict__ tabA,
                  const float *__restrict__ tabB, const float *__restrict__ tabL,
                  const signed char *__restrict__ ptype)
{
    __shared__ Pass<float> Ps;
    if (threadIdx.x == 0) Ps = *Pd;
    __syncthreads();
    wide_fix_body<DIM, KC>(g, Ps, tabA, tabB, tabL, ptype);
}

// Resident blocks per SM by pass: the passes with fewer pointwise streams
// fit a smaller register budget.
template <int KC, unsigned SIG>
__host__ __device__ constexpr int vec_minb()
{
    return KC ? 4 : (vec_heavy<SIG>() ? PF_VEC_MINB : PF_VEC_MINB_LIGHT);
}

template <int DIM, int KC, unsigned SIG>
__global__ void __launch_bounds__(VBLOCK, (vec_minb<KC, SIG>()))
vec_kernel(const __grid_constant__ Geom g, const __grid_constant__ Pass<float> P, const float *__restrict__ tabA,
           const float *__restrict__ tabB, const float *__restrict__ tabL, const signed char *__restrict__ ptype)
{
    vec_body<DIM, KC, SIG>(g, P, tabA, tabB, tabL, ptype, blockIdx.x, blockIdx.y, blockIdx.z,
                           (int)(gridDim.x * gridDim.y * gridDim.z));
}

// The same pass with its description read from device memory (device-driven
// adaptive steps; see cell_kernel_d).
template <int DIM, int KC, unsigned SIG>
__global__ void __launch_bounds__(VBLOCK, (vec_minb<KC, SIG>()))
vec_kernel_d(const __grid_constant__ Geom g, const Pass<float> *__restrict__ Pd, const float *__restrict__ tabA,
             const float *__restrict__ tabB, const float *__restrict__ tabL, const signed char *__restrict__ ptype)
{
    __shared__ Pass<float> Ps;
    if (threadIdx.x == 0) Ps = *Pd;
    __syncthreads();
    vec_body<DIM, KC, SIG>(g, Ps, tabA, tabB, tabL, ptype, blockIdx.x, blockIdx.y, blockIdx.z,
                           (int)(gridDim.x * gridDim.y * gridDim.z));
}


// ---------------------------------------------------------------------------
// Packed launches (batched serving): one launch runs the same pass kind
// (dimension, K, signature) of several problems.  The blocks of problem k
// are blocks bstart[k] .. bstart[k + 1] - 1 of the launch; each block finds
// its problem by binary search, copies that problem's constants and pass
// description into shared memory and runs the two-cell body on its tile, so
// every problem computes exactly what its own launch would.
// ---------------------------------------------------------------------------
struct VecInst {
    Geom g;
    Pass<float> P;
    const float *A, *B, *L;
    const signed char *ptype;
    int nblk;                        // two-cell blocks of this problem
};

__device__ __forceinline__ int packed_find(const int *__restrict__ bstart, int n, int b)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(bstart + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int DIM, int KC, unsigned SIG>
__global__ void __launch_bounds__(VBLOCK, (vec_minb<KC, SIG>()))
packed_kernel(const VecInst *__restrict__ tab, const int *__restrict__ bstart, int n)
{
    __shared__ Geom gs;
    __shared__ Pass<float> Ps;
    __shared__ int ks;
    if (threadIdx.x == 0) {
        const int k = packed_find(bstart, n, blockIdx.x);
        ks = k;
        gs = tab[k].g;
        Ps = tab[k].P;
    }
    __syncthreads();
    const int k = ks;
    const VecInst &I = tab[k];
    const int b = blockIdx.x - __ldg(bstart + k);
    const int tiles_x = (gs.nx + 2 * VTX - 1) / (2 * VTX), tiles_y = (gs.ny + VTY - 1) / VTY;
    vec_body<DIM, KC, SIG>(gs, Ps, I.A, I.B, I.L, I.ptype, b % tiles_x, (b / tiles_x) % tiles_y,
                           b / (tiles_x * tiles_y), I.nblk);
}

// The wide pass of a packed launch: the blocks share out every problem's
// recorded entries; the last block to finish closes every problem's pass
// (done: a counter of the batch, zero between launches).
template <int DIM, int KC>
__global__ void __launch_bounds__(VCELLS)
packed_wide_fix_kernel(const VecInst *__restrict__ tab, int n, int *done)
{
    for (int k = 0; k < n; ++k) {
        const VecInst &I = tab[k];
        wide_fix_entries<DIM, KC>(I.g, I.P, I.A, I.B, I.L, I.ptype, blockIdx.x, gridDim.x);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(done, 1) == (int)gridDim.x - 1) {
            for (int k = 0; k < n; ++k) wide_fix_close(tab[k].P);
            atomicExch(done, 0);
        }
    }
}

}  // namespace pfk
