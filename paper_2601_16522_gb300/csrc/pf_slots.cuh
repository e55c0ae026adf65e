// pf_slots.cuh -- FP32 stage passes on per-cell phase slots (Sec. 3.1).
//
// Slot storage keeps, per cell, at most NSLOT phase values with their phase
// ids (Sec. 3.1: N_p values and N_p integers per cell, N_p = 12 in the
// paper's final benchmark), so a state of N phases costs NSLOT * 6 bytes
// per cell whatever N is: 256^3 cells with 2000 grains take 1.3 GB per state
// vector where dense planes would take 134 GB.  Layout of one state vector
// (Vs = V rounded up to 64): NSLOT value planes (float), then NSLOT id planes
// (uint16, SLOT_EMPTY where unused; a cell's used slots come first, in
// ascending id order), then the concentration plane (float) when K = 1, at
// float offset SLOT_C_PLANES * Vs.
//
// A pass merges the sorted slot lists of the stencil input at the cell and
// its 2d face neighbours and of the pointwise inputs (ascending ids, one
// cursor per list), which visits the phases nonzero anywhere in them in
// ascending order -- the order in which the masked and dense one-cell passes
// visit them -- and applies the same arithmetic as those passes (a phase that
// is zero in every list contributes exactly nothing there), so results equal
// the dense ones bit for bit as long as no cell needs more than NSLOT slots.
// A projected cell with more nonzero values keeps the NSLOT largest (equal
// values: the lower id), the rest become zero and the kept ones are divided
// by their sum (ascending ids): the paper gives no rule for it; this is the
// reading the oracle restates.  "S acted" (the RKL2 first-stage fix) then
// includes that step.  The stored RHS F(u^n) of the STS schemes keeps, in a
// cell with more than NSLOT nonzero entries, the NSLOT largest in magnitude
// (equal magnitudes: the lower id): the same kind of reading.
#pragma once
#include "pf_kernels.cuh"

namespace pfk {

constexpr int NSLOT = 12;                              // slots per cell (N_p)
constexpr int SLOT_C_PLANES = NSLOT + NSLOT / 2;       // float planes before c
constexpr unsigned SLOT_EMPTY = 0xffffu;
constexpr int SLOT_MAXN = 32768;                       // largest phase count (N^2 tables)

// Floats per cell-plane of one slot state vector.
__host__ __device__ constexpr int slot_planes(int K) { return SLOT_C_PLANES + K; }

__device__ __forceinline__ const unsigned short *slot_ids(const float *base, int Vs)
{
    return reinterpret_cast<const unsigned short *>(base + (long long)NSLOT * Vs);
}

// The active list of a slot pass: phase ids need 16 bits.
struct SlotSmem {
    unsigned short id[MAXACT][BLOCK];
    float lap[MAXACT][BLOCK];    // Laplacian, later the RHS of the listed phase
    float cen[MAXACT][BLOCK];    // phi at the cell
    float dl[MAXACT][BLOCK];     // variational derivative
};

struct SlotListS {
    static constexpr int CAP = MAXACT;
    SlotSmem *S;
    int tid;
    __device__ __forceinline__ unsigned short &id(int k) { return S->id[k][tid]; }
    __device__ __forceinline__ float &lap(int k) { return S->lap[k][tid]; }
    __device__ __forceinline__ float &cen(int k) { return S->cen[k][tid]; }
    __device__ __forceinline__ float &dl(int k) { return S->dl[k][tid]; }
};

struct SlotListW {
    static constexpr int CAP = WIDEACT;
    unsigned short id_[WIDEACT];
    float lap_[WIDEACT], cen_[WIDEACT], dl_[WIDEACT];
    __device__ __forceinline__ unsigned short &id(int k) { return id_[k]; }
    __device__ __forceinline__ float &lap(int k) { return lap_[k]; }
    __device__ __forceinline__ float &cen(int k) { return cen_[k]; }
    __device__ __forceinline__ float &dl(int k) { return dl_[k]; }
};

// Cursor over one sorted slot list: the value of phase a if the list's next
// entry is a (advancing past it), else 0.
struct SlotCursor {
    const float *v;              // value planes of the vector
    const unsigned short *ids;   // id planes
    int ix;                      // cell index
    int cur;                     // next slot
    unsigned head;               // id of the next slot (SLOT_EMPTY: none)
    __device__ __forceinline__ void start(const float *base, int Vs, int cell)
    {
        v = base;
        ids = slot_ids(base, Vs);
        ix = cell;
        cur = 0;
        head = __ldg(ids + cell);
    }
    __device__ __forceinline__ float take(unsigned a, int Vs)
    {
        if (head != a) return 0.0f;
        const float x = __ldg(v + cur * Vs + ix);
        cur++;
        head = cur < NSLOT ? (unsigned)__ldg(ids + cur * Vs + ix) : SLOT_EMPTY;
        return x;
    }
};

// Union capacity: every slot of every list a pass merges.
template <int DIM>
__host__ __device__ constexpr int slot_ucap() { return (1 + 2 * DIM + 3) * NSLOT; }

// Per-cell body of a slot pass (one cell per thread).  LST is the active
// list (SlotListS in shared memory, SlotListW for the crowded-cell rerun);
// returns false, having written nothing, when more than LST::CAP phases are
// nontrivial at the cell.  The arithmetic and its order are those of
// masked_cell (see the file comment).
template <int DIM, int KC, unsigned SIG, class LST>
__device__ __forceinline__ bool slot_cell(const Geom &g, const Pass<float> &P, LST &S, int i, const int *off,
                                          const int *ghost, const float *__restrict__ tabA,
                                          const float *__restrict__ tabB, const float *__restrict__ tabL,
                                          const signed char *__restrict__ ptype, double &esum, long long &ecnt)
{
    typedef float T;
    constexpr int NFACE = 2 * DIM;
    constexpr int UCAP = slot_ucap<DIM>();
    constexpr bool RHS = (SIG & SIG_RHS) != 0;
    constexpr bool ERR = (SIG & SIG_ERR) != 0;
    constexpr bool HP0 = (SIG & SIG_P0) != 0 || ERR;
    constexpr bool HP2 = (SIG & SIG_P2) != 0;
    constexpr bool HR0 = (SIG & SIG_R0IN) != 0 || ERR;
    constexpr bool R0OUT = (SIG & SIG_R0OUT) != 0;
    constexpr bool PROJ = (SIG & SIG_PROJECT) != 0;
    const int N = g.N;
    const int Vs = (int)g.Vs;
    const long long co = (long long)SLOT_C_PLANES * Vs;   // concentration plane
    const T idx2 = (T)(1.0 / g.dx2);
    const T a0c = (T)P.a0, a2c = (T)P.a2, b1c = (T)P.b1, b0c = (T)P.b0;
    const T ib1 = (T)(1.0 / P.b1);   // first-stage fix: F <- (S(u1) - u^n) / (mu~_1 dt)
    const T dt = (T)P.dt, rph = (T)P.r_phi, aph = (T)P.a_phi;

    // concentration
    T cc = (T)0, num_c = (T)0, den_c = (T)0, num_n[NFACE], den_n[NFACE], mf[NFACE];
#pragma unroll
    for (int f = 0; f < NFACE; ++f) { num_n[f] = (T)0; den_n[f] = (T)0; mf[f] = (T)0; }
    if (KC) {
        const T *cf = P.in + co + i;
        cc = ldg(cf);
        num_c = cc;
#pragma unroll
        for (int f = 0; f < NFACE; ++f) {
            T v = ldg(cf + off[f]);
            if (ghost[f] && g.bc_c[f] == BC_DIRICHLET) v = (T)2 * (T)g.cdir[f] - cc;
            num_n[f] = v;
        }
    }

    // cursors: the stencil input at the cell and its face neighbours, then
    // the pointwise inputs
    SlotCursor cin, cnb[NFACE], cp0, cp2, cr0;
    cin.start(P.in, Vs, i);
#pragma unroll
    for (int f = 0; f < NFACE; ++f) cnb[f].start(P.in, Vs, i + off[f]);
    if (HP0) cp0.start(P.p0, Vs, i);
    if (HP2) cp2.start(P.p2, Vs, i);
    if (HR0) cr0.start(P.r0in, Vs, i);

    // the visited phases (ascending ids) with their stage values, input
    // values (first-stage fix) and list positions
    unsigned short uid[UCAP];
    T uv[UCAP], uin[R0OUT ? UCAP : 1];
    signed char ulist[UCAP];
    T lp0[ERR ? LST::CAP : 1], lr0[ERR ? LST::CAP : 1];
    int nu = 0, nz = 0, nc = 0;
    bool changed = false;
    T best = (T)-1, ssum = (T)0;
    int bestid = -1;
    for (;;) {
        unsigned a = cin.head;
#pragma unroll
        for (int f = 0; f < NFACE; ++f) a = min(a, cnb[f].head);
        if (HP0) a = min(a, cp0.head);
        if (HP2) a = min(a, cp2.head);
        if (HR0) a = min(a, cr0.head);
        if (a >= (unsigned)N) {
            // the end of every list; an id beyond the phases is a broken state
            if (a != SLOT_EMPTY) raise_flag(P.flag, FLAG_NZ_OVERFLOW);
            break;
        }
        const T v0 = cin.take(a, Vs);
        T nb[NFACE];
#pragma unroll
        for (int f = 0; f < NFACE; ++f) nb[f] = cnb[f].take(a, Vs);
        const T p0v = HP0 ? cp0.take(a, Vs) : (T)0;
        const T p2v = HP2 ? cp2.take(a, Vs) : (T)0;
        const T r0v = HR0 ? cr0.take(a, Vs) : (T)0;
        T mx = v0, mn = v0;
#pragma unroll
        for (int f = 0; f < NFACE; ++f) {
            mx = fmaxf(mx, nb[f]);
            mn = fminf(mn, nb[f]);
        }
        if (KC) {
            const int t = ptype[a];
            const T c0t = (T)g.c0[t], ikt = (T)g.invk[t], dkt = (T)g.Dk[t];
            num_c = num_c - v0 * c0t;
            den_c = den_c + v0 * ikt;
#pragma unroll
            for (int f = 0; f < NFACE; ++f) {
                num_n[f] = num_n[f] - nb[f] * c0t;
                den_n[f] = den_n[f] + nb[f] * ikt;
                mf[f] = mf[f] + dkt * ((T)0.5 * (v0 + nb[f]));
            }
        }
        const bool act = mx > (T)0 && mn < (T)1;
        signed char li = -1;
        if (act) {
            if (nz >= LST::CAP) return false;
            T l = (T)0;
#pragma unroll
            for (int f = 0; f < NFACE; ++f) l = l + (nb[f] - v0);
            S.id(nz) = (unsigned short)a;
            S.lap(nz) = l * idx2;
            S.cen(nz) = v0;
            if (ERR) { lp0[nz] = p0v; lr0[nz] = r0v; }
            li = (signed char)nz;
            nz++;
        }
        if (ERR) {
            if (!act) {
                T e = ((T)12 * (p0v - v0) + ((T)6 * dt) * r0v) * ((T)1 / (T)15);
                const T trial = p0v + (dt * (T)0.5) * r0v;
                if (trial < (T)0 || trial > (T)1) e = (T)0;
                if (e != (T)0) {
                    const T wt = rph * fmaxf(fabsf(p0v), fabsf(v0)) + aph;
                    const T q = e / wt;
                    esum += (double)(q * q);
                    nc++;
                }
            }
        } else if (!RHS) {
            T acc = affine<HP0, HP2>(v0, p0v, p2v, a0c, a2c);
            if (HR0) acc = acc + b0c * r0v;
            if (!act && PROJ) {
                if (acc < (T)0) { acc = (T)0; changed = true; }
                if (acc >= (T)1 && acc > best) { best = acc; bestid = (int)a; }
                ssum = ssum + acc;
            }
            uid[nu] = (unsigned short)a;
            uv[nu] = acc;
            ulist[nu] = li;
            if (R0OUT) uin[nu] = v0;
            nu++;
        }
    }

    T mu = (T)0, rc = (T)0;
    if (KC) {
        mu = num_c / den_c;
        T acc = (T)0;
#pragma unroll
        for (int f = 0; f < NFACE; ++f) acc = acc + mf[f] * (num_n[f] / den_n[f] - mu);
        rc = acc * idx2;
    }
    // variational derivative and pairwise sum over the listed phases (with
    // uniform tables the coefficients come from the constants: same values)
    const bool uni = g.uni != 0;
    for (int k = 0; k < nz; ++k) {
        const long long a = S.id(k);
        const T *Aa = tabA + a * N, *Ba = tabB + a * N;
        T d = (T)0;
        for (int k2 = 0; k2 < nz; ++k2) {
            if (k2 == k) continue;
            const int b = S.id(k2);
            const T Aab = uni ? g.uA : ldg(Aa + b), Bab = uni ? g.uB : ldg(Ba + b);
            d = d + (Aab * S.lap(k2) + Bab * S.cen(k2));
        }
        if (KC) {
            const int t = ptype[a];
            d = d + (-(mu * mu) / ((T)2 * (T)g.k[t]) - mu * (T)g.c0[t]);
        }
        S.dl(k) = d;
    }
    const T inz = nz > 1 ? (T)1 / (T)nz : (T)0;
    for (int k = 0; k < nz; ++k) {
        T rk = (T)0;
        if (nz > 1) {
            const T *La = tabL + (long long)S.id(k) * N;
            const T dk = S.dl(k);
            T s = (T)0;
            for (int k2 = 0; k2 < nz; ++k2) {
                if (k2 == k) continue;
                const T Lab = uni ? g.uL : ldg(La + S.id(k2));
                s = s + Lab * (dk - S.dl(k2));
            }
            rk = -(s * inz);
        }
        S.lap(k) = rk;                 // the list now holds the RHS
        if (ERR) {
            const T p0v = lp0[k], v0 = S.cen(k), r0v = lr0[k];
            const T sr = r0v + rk;
            T e = ((T)12 * (p0v - v0) + ((T)6 * dt) * sr) * ((T)1 / (T)15);
            const T trial = p0v + (dt * (T)0.5) * sr;
            if (trial < (T)0 || trial > (T)1) e = (T)0;
            if (e != (T)0) {
                const T wt = rph * fmaxf(fabsf(p0v), fabsf(v0)) + aph;
                const T q = e / wt;
                esum += (double)(q * q);
                nc++;
            }
        }
    }
    if constexpr (RHS) {
        // pf_rhs: the listed phases' RHS into the zeroed FP64 output
        if (P.rhs_pm) {
            for (int k = 0; k < nz; ++k) P.rhs_pm[(long long)S.id(k) * g.V + i] = (double)S.lap(k);
            if (KC) P.rhs_pm[(long long)N * g.V + i] = (double)rc;
        }
        if (P.nz_out) P.nz_out[i] = (unsigned char)(nz < 255 ? nz : 255);
        return true;
    } else if constexpr (ERR) {
        ecnt += (nc > 0 ? nc : 2);
        if (KC) {
            const T un = ldg(P.p0 + co + i), un1 = cc, rn = ldg(P.r0in + co + i);
            const T e = ((T)12 * (un - un1) + ((T)6 * dt) * (rn + rc)) * ((T)1 / (T)15);
            const T wt = (T)P.r_c * fmaxf(fabsf(un + (T)g.cref), fabsf(un1 + (T)g.cref)) + (T)P.a_c;
            const T q = e / wt;
            esum += (double)(q * q);
            ecnt += 1;
        }
        return true;
    } else {
    // listed phases (ascending ids): add the RHS term, clamp, >= 1 candidates, sum
    for (int j = 0; j < nu; ++j) {
        if (ulist[j] < 0) continue;
        const int a = uid[j];
        T acc = uv[j] + b1c * S.lap(ulist[j]);
        if (PROJ) {
            if (acc < (T)0) { acc = (T)0; changed = true; }
            if (acc >= (T)1 && (acc > best || (acc == best && a < bestid))) { best = acc; bestid = a; }
            ssum = ssum + acc;
        }
        uv[j] = acc;
    }
    if (PROJ) {
        if (bestid >= 0) {
            for (int j = 0; j < nu; ++j)
                if (uv[j] != (((int)uid[j] == bestid) ? (T)1 : (T)0)) changed = true;
            ssum = (T)1;
        }
        if (!(ssum > (T)0)) raise_flag(P.flag, FLAG_SIMPLEX);
    }
    const T inv = (ssum > (T)0) ? (T)1 / ssum : (T)1;
    // projected values; then the slot rule where more than NSLOT are nonzero
    int cnt = 0;
    for (int j = 0; j < nu; ++j) {
        T wv = uv[j];
        if (PROJ) wv = (bestid >= 0) ? (((int)uid[j] == bestid) ? (T)1 : (T)0) : wv * inv;
        uv[j] = wv;
        if (wv != (T)0) cnt++;
    }
    if (cnt > NSLOT) {
        // keep the NSLOT largest (equal values: the lower id), renormalise
        bool keep[UCAP];
        for (int j = 0; j < nu; ++j) {
            keep[j] = false;
            if (uv[j] == (T)0) continue;
            int rank = 0;
            for (int m = 0; m < nu; ++m)
                if (m != j && uv[m] != (T)0 && (uv[m] > uv[j] || (uv[m] == uv[j] && uid[m] < uid[j]))) rank++;
            keep[j] = rank < NSLOT;
        }
        T sk = (T)0;
        for (int j = 0; j < nu; ++j)
            if (keep[j]) sk = sk + uv[j];
        for (int j = 0; j < nu; ++j) uv[j] = keep[j] ? uv[j] / sk : (T)0;
        changed = true;
    }
    const bool fix = R0OUT && P.fix_first && changed;
    // the stored RHS F(u^n) (stage 1): its nonzero entries; more than NSLOT
    // keep the NSLOT largest in magnitude (equal magnitudes: the lower id)
    unsigned short *rid = R0OUT ? const_cast<unsigned short *>(slot_ids(P.r0out, Vs)) : nullptr;
    int kr = 0;
    if constexpr (R0OUT) {
        T ur[UCAP];
        int nr = 0;
        for (int j = 0; j < nu; ++j) {
            T r = ulist[j] >= 0 ? S.lap(ulist[j]) : (T)0;
            if (fix) r = (uv[j] - uin[j]) * ib1;
            ur[j] = r;
            if (r != (T)0) nr++;
        }
        for (int j = 0; j < nu; ++j) {
            if (ur[j] == (T)0) continue;
            if (nr > NSLOT) {
                int rank = 0;
                for (int m = 0; m < nu; ++m)
                    if (m != j && ur[m] != (T)0 &&
                        (fabsf(ur[m]) > fabsf(ur[j]) || (fabsf(ur[m]) == fabsf(ur[j]) && uid[m] < uid[j])))
                        rank++;
                if (rank >= NSLOT) continue;
            }
            if (kr < NSLOT) {       // (more only with non-finite values)
                P.r0out[kr * Vs + i] = ur[j];
                rid[kr * Vs + i] = uid[j];
                kr++;
            }
        }
    }
    // outputs: the nonzero entries in ascending id order, then empty slots
    unsigned short *oid = const_cast<unsigned short *>(slot_ids(P.out, Vs));
    int ko = 0;
    for (int j = 0; j < nu; ++j) {
        if (uv[j] != (T)0 && ko < NSLOT) {     // (more only with non-finite values, flagged)
            P.out[ko * Vs + i] = uv[j];
            oid[ko * Vs + i] = uid[j];
            ko++;
        }
    }
    for (int k = ko; k < NSLOT; ++k) {
        P.out[k * Vs + i] = (T)0;
        oid[k * Vs + i] = (unsigned short)SLOT_EMPTY;
    }
    if (R0OUT) {
        for (int k = kr; k < NSLOT; ++k) {
            P.r0out[k * Vs + i] = (T)0;
            rid[k * Vs + i] = (unsigned short)SLOT_EMPTY;
        }
    }
    if (KC) {
        // the small increments are summed first: c is rounded once per stage
        T d = b1c * rc;
        if (HR0) d = d + b0c * ldg(P.r0in + co + i);
        if (HP0) d = d + a0c * (ldg(P.p0 + co + i) - cc);
        if (HP2) d = d + a2c * (ldg(P.p2 + co + i) - cc);
        const T acc = cc + d;
        if (!isfinite(acc)) raise_flag(P.flag, FLAG_NONFINITE);
        if (R0OUT) P.r0out[co + i] = rc;
        P.out[co + i] = acc;
    }
    return true;
    }
}

// A cell with more than MAXACT nontrivial phases: the same body with a
// WIDEACT-entry list in local memory (out of line: only the rare threads
// that need it touch its local arrays); beyond WIDEACT the pass raises
// FLAG_NZ_OVERFLOW.
template <int DIM, int KC, unsigned SIG>
__device__ __noinline__ void slot_wide(const Geom *g, const Pass<float> *P, int i, const int *off, const int *ghost,
                                       const float *tabA, const float *tabB, const float *tabL,
                                       const signed char *ptype, double *esum, long long *ecnt)
{
    SlotListW L;
    double es = 0.0;
    long long ec = 0;
    if (!slot_cell<DIM, KC, SIG, SlotListW>(*g, *P, L, i, off, ghost, tabA, tabB, tabL, ptype, es, ec)) {
        raise_flag(P->flag, FLAG_NZ_OVERFLOW);
        return;
    }
    *esum += es;
    *ecnt += ec;
}

// Resident blocks per SM (register budget): 4 for the RKL2 body, 3 for the
// other passes (measured on 256^3 x 2000 grains with table gathers: the RKL2
// pass takes 6.6 ms at 2 resident blocks, 3.2 ms at 3, 2.9 ms at 4; with the
// uniform coefficients 2.46 ms at 4 and 4.2 ms at 5, where 48 registers
// spill).
template <unsigned SIG>
constexpr int slot_minb() { return (SIG & (SIG_P0 | SIG_P2)) == (SIG_P0 | SIG_P2) ? 4 : 3; }

// One slot pass: one cell per thread, 32 x 8 tiles, one z plane per block.
template <int DIM, int KC, unsigned SIG>
__global__ void __launch_bounds__(BLOCK, slot_minb<SIG>())
slot_kernel(const __grid_constant__ Geom g, const __grid_constant__ Pass<float> P, const float *__restrict__ tabA,
            const float *__restrict__ tabB, const float *__restrict__ tabL, const signed char *__restrict__ ptype)
{
    __shared__ SlotSmem Sm;
    if (pass_skipped(P.flag)) return;
    const int tid = threadIdx.x;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int x = blockIdx.x * TX + (tid % TX);
    const int y = blockIdx.y * TY + (tid / TX);
    const int z = blockIdx.z;
    double esum = 0.0;
    long long ecnt = 0;
    if (x < g.nx && y < g.ny) {
        const int i = (int)(((long long)z * g.ny + y) * g.nx + x);
        long long off64[6];
        int ghost[6], off[6];
        face_offsets(g, x, y, z, off64, ghost);
#pragma unroll
        for (int f = 0; f < 6; ++f) off[f] = ghost[f] ? 0 : (int)off64[f];
        SlotListS S{&Sm, tid};
        if (!slot_cell<DIM, KC, SIG, SlotListS>(g, P, S, i, off, ghost, tabA, tabB, tabL, ptype, esum, ecnt)) {
            esum = 0.0;
            ecnt = 0;
            slot_wide<DIM, KC, SIG>(&g, &P, i, off, ghost, tabA, tabB, tabL, ptype, &esum, &ecnt);
        }
    }
    if (SIG & SIG_ERR) block_partials(esum, ecnt, P.part_sum, P.part_cnt, bid, P.part_n);
    if (P.count_step) count_step_done(P.flag);
}

}  // namespace pfk
