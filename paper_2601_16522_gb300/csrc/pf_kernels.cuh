// pf_kernels.cuh -- sm_103a device code for one explicit stage of the
// obstacle-potential multi-phase-field + KKS model (Seiz & Takaki,
// arXiv 2601.16522, Sec. 2-3).
//
// Layout in HBM: a state vector holds NF = N + K fields, field f at
// u + f * Vs (Vs = V rounded up to 64 cells, so every field starts 256-byte
// aligned); inside a field cells are x-fastest.  One thread owns one cell:
// every load of a warp is 32 consecutive cells of one field (coalesced), and
// the per-cell loops over phases run over phase planes with stage values of a
// chunk of phases held in shared memory.  The nontrivial phases of a cell (the n(phi) filter of Eq. phieq,
// at most MAXACT of them) are gathered into a small static-index list in
// ascending phase order (per-thread slots in shared memory), so the pairwise
// sums run over the N_z entries only, in the same order as a plain loop over
// all phases.
//
// One pass computes the RHS of its stencil input and, fused, the stage
// combination, the simplex projection (Sec. 3.1), the RKL2 first-stage fix
// (Sec. 3.2), the SSP(10)4 embedded accumulator and the per-thread partials
// of the error norm (Sec. 3.3).  With more phases than one chunk holds the
// unnormalised stage values are written and re-read (L2-resident) for the
// projection's normalisation.  The hot passes are compiled per signature
// (which inputs and outputs they use); everything else takes the generic
// instantiation that reads the options at run time.
#pragma once
#include <cuda.h>            // CUtensorMap (type only)
#include <cuda_runtime.h>
#include <stdint.h>

namespace pfk {

enum { BC_PERIODIC = 0, BC_NEUMANN = 1, BC_DIRICHLET = 2 };
constexpr int MAXACT = 12;      // nontrivial phases per cell in the fast (shared-memory) list
constexpr int WIDEACT = 64;     // ... in the per-thread fallback list of crowded cells
constexpr int TX = 32, TY = 8;  // cells per block: 32 (x) by 8 (y), one z plane
constexpr int BLOCK = TX * TY;

// Stage combination a0 p0 + a1 v + a2 p2 of every pass, whose coefficients
// sum to one (affine combinations of states, Eq. sts, Alg. ssp2, SSP(10)4),
// evaluated as v + a0 (p0 - v) + a2 (p2 - v).  A constant field then stays
// exactly constant whatever the rounding of the coefficients, so in FP32 the
// solute total is not scaled by (a0 + a1 + a2 rounded) at every stage; the
// coefficient rounding only reaches the small stage differences.
template <bool HP0, bool HP2, typename T>
__device__ __forceinline__ T affine(T v, T p0, T p2, T a0, T a2)
{
    T acc = v;
    if (HP0) acc = acc + a0 * (p0 - v);
    if (HP2) acc = acc + a2 * (p2 - v);
    return acc;
}

// Problem constants shared by every pass (passed by value).
struct Geom {
    int nx, ny, nz, dim;
    long long V, Vs;                    // cells, field stride
    int N, K, NF;
    int bc_phi[6], bc_c[6];
    double cdir[6];                     // Dirichlet value of c per face, minus cref
    double dx2;                         // dx * dx
    double k[2], c0[2], invk[2], Dk[2]; // per chemical type: k, c0 - cref, 1/k, D/k
    double cref;                        // FP32 storage holds c - cref (0 in FP64); c0 and cdir
                                        // are shifted by it, so mu and the face fluxes are those
                                        // of c, and only the error weights |c| add it back
    int tiles_x, tiles_y;               // block tiling of the x-y plane (one-cell kernels)
    int kvar;                           // FP32 dense passes: KVAR_TWO_CELL or KVAR_ONE_CELL
    int simplex;                        // projection S: SIMPLEX_STANDARD or SIMPLEX_MOBILITY
    int slots;                          // 1: per-cell phase slots (FP32; see pf_slots.cuh)
    int uni;                            // slot passes: 1 if every off-diagonal entry of each
    float uA, uB, uL;                   // FP32 table A, B, L is the same value (these), which
                                        // the pairwise sums then use instead of gathers
};
// Kernel variants of the FP32 dense passes (chosen per handle, pf_autotune).
enum { KVAR_TWO_CELL = 0, KVAR_ONE_CELL = 1 };
// The projection onto the simplex after every stage (Sec. 3.1): the standard
// one (clamp, >= 1 rule, divide by the sum) or the mobility-weighted one
// (mob_project; the generic body only).
enum { SIMPLEX_STANDARD = 0, SIMPLEX_MOBILITY = 1 };

// What one pass does (passed by value).
template <typename T>
struct Pass {
    int mode;            // MODE_RHS, MODE_STAGE or MODE_ERR
    const T *in;         // stencil input (the RHS is evaluated on it)
    const T *p0;         // pointwise input with coefficient a0 (may be null)
    const T *p2;         // pointwise input with coefficient a2 (may be null)
    const T *r0in;       // pointwise RHS with coefficient b0 (may be null)
    T *out;              // stage output
    T *r0out;            // store the RHS of `in` (RKL stage 1); may be null
    int fix_first;       // RKL2 first-stage replacement where S acted (Sec. 3.2)
    const T *zin;        // SSP(10)4 embedded accumulator input (may be null)
    T *zout;             // SSP(10)4 embedded accumulator output (may be null)
    T *out2;             // SSP(10)4 after stage 5: q2 output (with q2in)
    const T *q2in;
    const T *uw;         // u^n for the error weights (SSP(10)4 final stage)
    int project;         // apply the simplex projection to the phases
    int embedded_err;    // final SSP(10)4 stage: e = u - z into the error partials
    double a0, a1, a2, b1, b0, bz;   // combination coefficients (dt folded into b*);
                                     // a0 + a1 + a2 = 1, see affine()
    double m25, m15;                 // SSP(10)4 after stage 5: q2 <- q1 + m25 (q2in - q1),
                                     // q1 <- q1 + m15 (q2 - q1)
    double dt;                       // step size (error sweep)
    double r_phi, a_phi, r_c, a_c;   // tolerances (error partials)
    double *part_sum;    // per-block partial sums of (e/w)^2
    long long *part_cnt; // per-block partial DoF counts
    int *part_n;         // number of partials the pass wrote (its block count)
    double *rhs_pm;      // MODE_RHS: FP64 output, field f at rhs_pm + f * V
    unsigned char *nz_out; // MODE_RHS: N_z per cell (may be null)
    int *flag;           // device status words (see raise_flag)
    int *crowd;          // two-cell passes: record of crowded cells for the wide pass
    int count_step;      // this pass completes a fixed step: count it (see count_step_done)
    // Occupancy masks (masked storage, FP32 fast path, N <= 32): bit a of a
    // cell's word is set where phase a may be nonzero; every entry whose bit
    // is clear holds zero.  Null: dense pass.
    const unsigned *m_in, *m_p0, *m_p2, *m_r0;
    unsigned *m_out, *m_r0out;
    // the same for the SSP(10)4 vectors: z accumulator in/out, q2 in/out, u^n
    const unsigned *m_zin, *m_q2in, *m_uw;
    unsigned *m_zout, *m_out2;
};

enum { MODE_RHS = 0, MODE_STAGE = 1, MODE_ERR = 2 };

// Device status words behind Pass::flag (four ints, cleared by the engine at
// the start of every pf_step / pf_rhs call):
//   [0]  FLAG_* bits raised by any pass of the call;
//   [1]  fixed steps completed so far in the call (counted by the last pass
//        of every fixed step, see count_step_done);
//   [2]  blocks of the current counting pass that have finished;
//   [3]  1 + [1] at the moment the first flag was raised (0: none), i.e. the
//        number of the step in which the failure happened.
// A pass that starts while [0] is non-zero does nothing, so once a step has
// failed no state buffer is written any more: u^n of the failed step, which
// no pass of a step overwrites, stays intact for the engine to return.
enum { FLAG_SIMPLEX = 1, FLAG_NZ_OVERFLOW = 2, FLAG_TIMEOUT = 4, FLAG_NONFINITE = 8 };

__device__ __forceinline__ bool pass_skipped(const int *flag) { return *(const volatile int *)flag != 0; }

__device__ __forceinline__ void raise_flag(int *flag, int bits)
{
    atomicOr(flag, bits);
    atomicCAS(flag + 3, 0, 1 + *(volatile int *)(flag + 1));
}

// End of a pass that completes a fixed step (every thread of the block calls
// it): the last block of the grid to finish counts the step.  A flag raised
// during the pass is recorded (raise_flag) before the raising block finishes,
// hence before the count moves on.
__device__ __forceinline__ void count_step_done(int *flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
        if (atomicAdd((unsigned *)(flag + 2), 1u) == nb - 1u) {
            atomicExch(flag + 2, 0);
            atomicAdd(flag + 1, 1);
        }
    }
}

template <typename T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

template <typename T>
__device__ __forceinline__ T tabs(T v) { return v < (T)0 ? -v : v; }

// Phases ahead for which the FP32 fast path asks L2 to fetch the lines of the
// pointwise inputs and of the stencil input's cell (0: off).
#ifndef PF_PREFETCH_DIST
#define PF_PREFETCH_DIST 4
#endif
// Resident 256-thread blocks per SM the fast kernel's register budget targets.
#ifndef PF_FAST_MINB
#define PF_FAST_MINB 4
#endif
// Dense FP32 stage passes through the rolled phase loop (every phase
// occupied) instead of the register-unrolled one (the error sweep, which
// holds no stage values, always takes the rolled loop: it measured faster).
#ifndef PF_DENSE_ROLLED
#define PF_DENSE_ROLLED 0
#endif
// ... and of its masked-storage instantiations.
#ifndef PF_MASK_MINB
#define PF_MASK_MINB 4
#endif

// Streaming load that does not allocate in L1 (pointwise stage inputs are
// used once; L1 is left to the stencil rows shared between warps).
#ifndef PF_STREAM_NOALLOC
#define PF_STREAM_NOALLOC 1
#endif
__device__ __forceinline__ float ld_stream(const float *p)
{
#if PF_STREAM_NOALLOC
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
#else
    return __ldg(p);
#endif
}

__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Offsets (in cells) of the 2d face neighbours of (x,y,z); ghost[f] = 1 for a
// non-periodic domain face (the caller builds the ghost value), else 0.
__device__ __forceinline__ void face_offsets(const Geom &g, int x, int y, int z, long long off[6], int ghost[6])
{
    const long long sx = 1, sy = g.nx, sz = (long long)g.nx * g.ny;
    const int c[3] = {x, y, z};
    const int n[3] = {g.nx, g.ny, g.nz};
    const long long s[3] = {sx, sy, sz};
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        const int ax = f >> 1;
        const bool plus = f & 1;
        ghost[f] = 0;
        if (!plus) {
            if (c[ax] > 0) off[f] = -s[ax];
            else if (g.bc_phi[f] == BC_PERIODIC) off[f] = (long long)(n[ax] - 1) * s[ax];
            else { off[f] = 0; ghost[f] = 1; }
        } else {
            if (c[ax] < n[ax] - 1) off[f] = s[ax];
            else if (g.bc_phi[f] == BC_PERIODIC) off[f] = -(long long)(n[ax] - 1) * s[ax];
            else { off[f] = 0; ghost[f] = 1; }
        }
    }
}

// Fixed-order block reduction of (sum, count) into the per-block partials;
// block 0 records how many partials the launch writes (pn, may be null).
__device__ __forceinline__ void block_partials(double esum, long long ecnt, double *ps, long long *pc, int bid,
                                               int *pn = nullptr, int nblk = -1)
{
    if (pn && bid == 0 && threadIdx.x == 0) *pn = nblk >= 0 ? nblk : (int)(gridDim.x * gridDim.y * gridDim.z);
    constexpr int MAXW = 16;                 // blocks of up to 512 threads
    __shared__ double rs_sum[MAXW];
    __shared__ long long rs_cnt[MAXW];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        esum += __shfl_xor_sync(0xffffffffu, esum, o);
        ecnt += __shfl_xor_sync(0xffffffffu, ecnt, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { rs_sum[wid] = esum; rs_cnt[wid] = ecnt; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        long long c = 0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) { s += rs_sum[w]; c += rs_cnt[w]; }
        ps[bid] = s;
        pc[bid] = c;
    }
}

// Compile-time pass signature: which optional inputs/outputs a pass uses.
// SIG_GENERIC reads every option from the Pass at run time.
enum : unsigned {
    SIG_P0 = 1u, SIG_P2 = 2u, SIG_R0IN = 4u, SIG_R0OUT = 8u, SIG_PROJECT = 16u,
    SIG_ERR = 32u, SIG_RHS = 64u,
    // SSP(10)4 (Sec. 3.3): embedded accumulator z <- z + bz F, the q2 combination
    // after stage 5, and the embedded error of the final stage (implies SIG_Z)
    SIG_Z = 128u, SIG_O2 = 256u, SIG_EMB = 512u,
    SIG_GENERIC = 1u << 30
};

template <typename T>
struct Smem {
    static constexpr int NV = sizeof(T) == 4 ? 32 : 16;   // stage values held per chunk
    unsigned char id[MAXACT][BLOCK];
    T lap[MAXACT][BLOCK];    // Laplacian, later the RHS of the listed phase
    T cen[MAXACT][BLOCK];    // phi at the cell
    T dl[MAXACT][BLOCK];     // variational derivative
    T nv[NV][BLOCK];         // stage values of the current chunk
};

// Where the generic body keeps a cell's list of nontrivial phases.
// SlotList: the thread's slots of the block's shared memory (MAXACT entries,
// plus a chunk of NV stage values).  WideList: a per-thread array in local
// memory (WIDEACT entries, no stage-value chunk: the stage values go through
// the output buffer), the fallback for cells where more than MAXACT phases
// are nontrivial.
template <typename T>
struct SlotList {
    static constexpr int CAP = MAXACT;
    static constexpr int NV = Smem<T>::NV;
    Smem<T> *S;
    int tid;
    __device__ __forceinline__ unsigned char &id(int k) { return S->id[k][tid]; }
    __device__ __forceinline__ T &lap(int k) { return S->lap[k][tid]; }
    __device__ __forceinline__ T &cen(int k) { return S->cen[k][tid]; }
    __device__ __forceinline__ T &dl(int k) { return S->dl[k][tid]; }
    __device__ __forceinline__ T &nv(int a) { return S->nv[a][tid]; }
};

template <typename T>
struct WideList {
    static constexpr int CAP = WIDEACT;
    static constexpr int NV = 0;
    unsigned char id_[WIDEACT];
    T lap_[WIDEACT], cen_[WIDEACT], dl_[WIDEACT];
    __device__ __forceinline__ unsigned char &id(int k) { return id_[k]; }
    __device__ __forceinline__ T &lap(int k) { return lap_[k]; }
    __device__ __forceinline__ T &cen(int k) { return cen_[k]; }
    __device__ __forceinline__ T &dl(int k) { return dl_[k]; }
    __device__ __forceinline__ T &nv(int) { return lap_[0]; }   // never used (NV = 0)
};

// Mobility-weighted projection of one cell (a reading of the mobility-based
// simplex Sec. 3.1 cites for the particle cases of Sec. 5.3): on the phases
// with a positive value, P = {a : y_a > 0}, the point of the simplex face
// they span nearest to y in the metric sum (x_a - y_a)^2 / w_a, w_a the mean
// phase-field mobility L_ab of a towards the other phases of P:
// x_a = max(y_a - tau w_a, 0), sum x_a = 1.  tau by the weighted active-set
// iteration (drop the phases that reach zero, recompute, until none does);
// sums in ascending phase order.  No mobility to share the correction: the
// standard S on P.  The N values sit at v[a * Vs] (raw on entry, projected
// on return).  Returns 1 if a value changed, 0 if none did, -1 if no value is
// positive, -2 if more than MOBCAP are.  Out of line: only the generic
// passes of a handle created with this projection call it.
constexpr int MOBCAP = 64;
template <typename T>
__device__ __noinline__ int mob_project(int N, long long Vs, T *v, const T *__restrict__ tabL)
{
    unsigned char pid[MOBCAP];
    T yv[MOBCAP], w[MOBCAP];
    int np = 0;
    bool nonpos = false;     // a nonzero value <= 0 (becomes 0)
    for (int a = 0; a < N; ++a) {
        const T y = v[(long long)a * Vs];
        if (y > (T)0) {
            if (np >= MOBCAP) return -2;
            pid[np] = (unsigned char)a;
            yv[np] = y;
            np++;
        } else if (y != (T)0) {
            nonpos = true;
        }
    }
    if (np == 0) return -1;
    unsigned long long on = 0ull;
    T tau = (T)0;
    bool standard = false;
    if (np > 1) {
        T wsum = (T)0;
        for (int k = 0; k < np; ++k) {
            const T *La = tabL + pid[k] * N;
            T s = (T)0;
            for (int j = 0; j < np; ++j)
                if (j != k) s = s + La[pid[j]];
            w[k] = s / (T)(np - 1);
            wsum = wsum + w[k];
            on |= 1ull << k;
        }
        standard = !(wsum > (T)0);
        while (!standard) {
            T sy = (T)0, sw = (T)0;
            for (int k = 0; k < np; ++k)
                if ((on >> k) & 1ull) { sy = sy + yv[k]; sw = sw + w[k]; }
            if (!(sw > (T)0)) { standard = true; break; }
            tau = (sy - (T)1) / sw;
            bool dropped = false;
            for (int k = 0; k < np; ++k)
                if (((on >> k) & 1ull) && yv[k] - tau * w[k] <= (T)0) { on &= ~(1ull << k); dropped = true; }
            if (!dropped) break;
        }
    }
    int amax = -1;
    T s = (T)0;
    if (standard) {
        for (int k = 0; k < np; ++k)
            if (yv[k] >= (T)1 && (amax < 0 || yv[k] > yv[amax])) amax = k;
        for (int k = 0; k < np; ++k) s = s + yv[k];
    }
    bool changed = nonpos;
    int k = 0;
    for (int a = 0; a < N; ++a) {
        T x = (T)0;
        if (k < np && pid[k] == a) {
            if (np == 1) x = (T)1;
            else if (standard) x = amax >= 0 ? (k == amax ? (T)1 : (T)0) : yv[k] / s;
            else x = ((on >> k) & 1ull) ? yv[k] - tau * w[k] : (T)0;
            if (x != yv[k]) changed = true;
            k++;
        }
        v[(long long)a * Vs] = x;
    }
    return changed ? 1 : 0;
}

// Whether a value is +0 (its encoding is all zero bits): integer tests that
// let the generic body skip arithmetic whose result is exactly known.
__device__ __forceinline__ bool zbits(double x) { return __double_as_longlong(x) == 0; }
__device__ __forceinline__ bool zbits(float x) { return __float_as_int(x) == 0; }
__device__ __forceinline__ bool same_bits(double a, double b) { return __double_as_longlong(a) == __double_as_longlong(b); }
__device__ __forceinline__ bool same_bits(float a, float b) { return __float_as_int(a) == __float_as_int(b); }

// The activity filter of Eq. phieq on a phase's stencil values: max > 0 and
// min < 1.  In FP64 it runs on the encodings (for finite values x > 0 and
// x < 1 are signed integer comparisons of the bits), off the FP64 pipe.
template <int NFACE>
__device__ __forceinline__ bool nontrivial(double v0, const double *nb)
{
    long long bx = __double_as_longlong(v0), bn = bx;
#pragma unroll
    for (int f = 0; f < NFACE; ++f) {
        const long long b = __double_as_longlong(nb[f]);
        bx = b > bx ? b : bx;
        bn = b < bn ? b : bn;
    }
    return bx > 0 && bn < 0x3ff0000000000000LL;
}
template <int NFACE>
__device__ __forceinline__ bool nontrivial(float v0, const float *nb)
{
    float mx = v0, mn = v0;
#pragma unroll
    for (int f = 0; f < NFACE; ++f) {
        mx = nb[f] > mx ? nb[f] : mx;
        mn = nb[f] < mn ? nb[f] : mn;
    }
    return mx > 0.0f && mn < 1.0f;
}

// The generic per-cell body: RHS, stage combination, projection, first-stage
// fix, SSP(10)4 accumulators and error partials of one cell (x, y, z), with
// every option read from P at run time (SIG_GENERIC) or fixed by SIG.
// Returns false, having written nothing and accumulated nothing, when more
// than LST::CAP phases are nontrivial at the cell (the caller then takes the
// wide path).
template <typename T, int DIM, int KC, unsigned SIG, class LST>
__device__ __forceinline__ bool cell_core(const Geom &g, const Pass<T> &P, LST &S, const T *__restrict__ tabA,
                                          const T *__restrict__ tabB, const T *__restrict__ tabL,
                                          const signed char *__restrict__ ptype, int x, int y, int z,
                                          double &esum, long long &ecnt)
{
    constexpr int NFACE = 2 * DIM;
    constexpr bool GEN = (SIG & SIG_GENERIC) != 0;
    constexpr int NV = LST::NV;

    // pass options: compile-time for the specialised signatures, run time for GENERIC
    const int mode = GEN ? P.mode : ((SIG & SIG_ERR) ? MODE_ERR : (SIG & SIG_RHS) ? MODE_RHS : MODE_STAGE);
    const bool has_p0 = GEN ? P.p0 != nullptr : (SIG & SIG_P0) != 0;
    const bool has_p2 = GEN ? P.p2 != nullptr : (SIG & SIG_P2) != 0;
    const bool has_r0in = GEN ? P.r0in != nullptr : (SIG & SIG_R0IN) != 0;
    const bool has_r0out = GEN ? P.r0out != nullptr : (SIG & SIG_R0OUT) != 0;
    const bool project = GEN ? P.project != 0 : (SIG & SIG_PROJECT) != 0;
    const bool has_z = GEN && P.zout != nullptr;
    const bool emb = GEN && P.embedded_err != 0;
    const bool has_out2 = GEN && P.out2 != nullptr;

    const int N = g.N;
    const int K = KC;
    const long long Vs = g.Vs;
    const long long i = ((long long)z * g.ny + y) * g.nx + x;
    const T dx2 = (T)g.dx2;

    long long off[6];
    int ghost[6];
    face_offsets(g, x, y, z, off, ghost);
    // a zero-gradient ghost of phi is the cell itself: offset 0
#pragma unroll
    for (int f = 0; f < 6; ++f) if (ghost[f]) off[f] = 0;

    // ---- concentration at the cell and its face neighbours -----------------
    T cc = (T)0, num_c = (T)0, den_c = (T)0, num_n[NFACE], den_n[NFACE], mf[NFACE];
#pragma unroll
    for (int f = 0; f < NFACE; ++f) { num_n[f] = (T)0; den_n[f] = (T)0; mf[f] = (T)0; }
    if (K) {
        const T *cf = P.in + (long long)N * Vs + i;
        cc = ldg(cf);
        num_c = cc;
#pragma unroll
        for (int f = 0; f < NFACE; ++f) {
            T v = ldg(cf + off[f]);
            if (ghost[f] && g.bc_c[f] == BC_DIRICHLET) v = (T)2 * (T)g.cdir[f] - cc;
            num_n[f] = v;
        }
    }

    // ---- pass 1: activity, Laplacian, chemistry sums (Sec. 2-3) ------------
    int nz = 0;
    {
        const T *fp = P.in + i;
#pragma unroll 4
        for (int a = 0; a < N; ++a, fp += Vs) {
            const T v0 = ldg(fp);
            T nb[NFACE];
#pragma unroll
            for (int f = 0; f < NFACE; ++f) nb[f] = ldg(fp + off[f]);
            const bool act = nontrivial<NFACE>(v0, nb);
            if (K) {
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
            if (act) {
                T l = (T)0;
#pragma unroll
                for (int f = 0; f < NFACE; ++f) l = l + (nb[f] - v0);
                if (nz < LST::CAP) {
                    S.id(nz) = (unsigned char)a;
                    S.lap(nz) = l / dx2;
                    S.cen(nz) = v0;
                }
                nz++;
            }
        }
    }
    if (nz > LST::CAP) return false;

    // ---- grand potential and concentration RHS -----------------------------
    T mu = (T)0, rc = (T)0;
    if (K) {
        mu = num_c / den_c;
        T acc = (T)0;
#pragma unroll
        for (int f = 0; f < NFACE; ++f) {
            const T mun = num_n[f] / den_n[f];
            acc = acc + mf[f] * (mun - mu);
        }
        rc = acc / dx2;
    }

    // ---- variational derivative and pairwise sum over the list -------------
    for (int k = 0; k < nz; ++k) {
        const int a = S.id(k);
        const T *Aa = tabA + a * N, *Ba = tabB + a * N;
        T d = (T)0;
        for (int k2 = 0; k2 < nz; ++k2) {
            if (k2 == k) continue;
            const int b = S.id(k2);
            d = d + (ldg(Aa + b) * S.lap(k2) + ldg(Ba + b) * S.cen(k2));
        }
        T psi = (T)0;
        if (K) {
            const int t = ptype[a];
            psi = -(mu * mu) / ((T)2 * (T)g.k[t]) - mu * (T)g.c0[t];
        }
        S.dl(k) = d + psi;
    }
    for (int k = 0; k < nz; ++k) {
        T rk = (T)0;
        if (nz > 1) {
            const int a = S.id(k);
            const T *La = tabL + a * N;
            const T dk = S.dl(k);
            T s = (T)0;
            for (int k2 = 0; k2 < nz; ++k2) {
                if (k2 == k) continue;
                s = s + ldg(La + S.id(k2)) * (dk - S.dl(k2));
            }
            rk = -(s / (T)nz);
        }
        S.lap(k) = rk;                  // the list now holds the RHS
    }

    // list cursor: phases are visited in ascending order
    int kk = 0;
    int curid = nz > 0 ? S.id(0) : -1;
#define PF_NEXT_RHS(a_, r_)                                          \
    if ((a_) == curid) {                                             \
        r_ = S.lap(kk);                                              \
        kk++;                                                        \
        curid = kk < nz ? S.id(kk) : -1;                             \
    }

    if (mode == MODE_RHS) {
        // ---- RHS only (pf_rhs); without rhs_pm only N_z (pf_get_state) -----
        if (P.rhs_pm) {
            for (int a = 0; a < N; ++a) {
                T r = (T)0;
                PF_NEXT_RHS(a, r)
                P.rhs_pm[(long long)a * g.V + i] = (double)r;
            }
            if (K) P.rhs_pm[(long long)N * g.V + i] = (double)rc;
        }
        if (P.nz_out) P.nz_out[i] = (unsigned char)nz;
    } else if (mode == MODE_ERR) {
        // ---- STS error sweep (Sec. 3.3): in = u^{n+1}, p0 = u^n, r0in = F^n
        const T dt = (T)P.dt;
        const T rph = (T)P.r_phi, aph = (T)P.a_phi;
        int nc = 0;
        long long o = i;
#pragma unroll 4
        for (int a = 0; a < N; ++a, o += Vs) {
            T r1 = (T)0;
            PF_NEXT_RHS(a, r1)
            if (P.r0out) P.r0out[o] = r1;      // F(u^{n+1}) kept for reuse
            const T un = ldg(P.p0 + o), un1 = ldg(P.in + o), rn = ldg(P.r0in + o);
            // no change and no RHS: e is exactly zero (skipped like any zero e)
            if (same_bits(un, un1) && zbits(rn) && zbits(r1)) continue;
            const T sr = rn + r1;
            T e = ((T)12 * (un - un1) + ((T)6 * dt) * sr) / (T)15;
            const T trial = un + (dt / (T)2) * sr;
            if (trial < (T)0 || trial > (T)1) e = (T)0;
            if (e != (T)0) {
                const T au = tabs(un), av = tabs(un1);
                const T w = rph * (au > av ? au : av) + aph;
                const T q = e / w;
                esum += (double)(q * q);
                nc++;
            }
        }
        ecnt += (nc > 0 ? nc : 2);
        if (K) {
            const long long oc = (long long)N * Vs + i;
            if (P.r0out) P.r0out[oc] = rc;
            const T un = ldg(P.p0 + oc), un1 = ldg(P.in + oc), rn = ldg(P.r0in + oc);
            const T sr = rn + rc;
            const T e = ((T)12 * (un - un1) + ((T)6 * dt) * sr) / (T)15;
            const T au = tabs(un + (T)g.cref), av = tabs(un1 + (T)g.cref);
            const T w = (T)P.r_c * (au > av ? au : av) + (T)P.a_c;
            const T q = e / w;
            esum += (double)(q * q);
            ecnt += 1;
        }
    } else {
        // ---- stage combination (Eq. sts / Alg. ssp2 / SSP(10)4) -------------
        const T a0c = (T)P.a0, a2c = (T)P.a2, b1c = (T)P.b1, b0c = (T)P.b0, bzc = (T)P.bz;
        // the mobility-weighted projection works on the stage values in the output
        const bool mob = GEN && project && g.simplex == SIMPLEX_MOBILITY;
        const bool chunked = N > NV || mob;
        bool changed = false;
        T best = (T)-1;
        int bestid = -1;
        T ssum = (T)0;
        for (int a0 = 0; a0 < N; a0 += (NV > 0 ? NV : N)) {
            const int an = NV > 0 ? ((N - a0) < NV ? (N - a0) : NV) : N;
            long long o = (long long)a0 * Vs + i;
#pragma unroll 4
            for (int aa = 0; aa < an; ++aa, o += Vs) {
                const int a = a0 + aa;
                T r = (T)0;
                PF_NEXT_RHS(a, r)
                const T v = ldg(P.in + o);
                const T p0v = has_p0 ? ldg(P.p0 + o) : (T)0, p2v = has_p2 ? ldg(P.p2 + o) : (T)0;
                const T r0v = has_r0in ? ldg(P.r0in + o) : (T)0;
                T acc = v;
                // every input +0: the combination is exactly 0 (no arithmetic)
                if (!(zbits(v) && zbits(p0v) && zbits(p2v) && zbits(r0v) && zbits(r))) {
                    if (has_p0) acc = acc + a0c * (p0v - v);
                    if (has_p2) acc = acc + a2c * (p2v - v);
                    acc = acc + b1c * r;
                    if (has_r0in) acc = acc + b0c * r0v;
                }
                if (has_r0out) P.r0out[o] = r;      // replaced below where S acts (RKL2)
                if (has_z) P.zout[o] = P.zin[o] + bzc * r;   // zin may alias zout
                if (project && !mob && !zbits(acc)) {
                    // S step 1: clamp negatives; step 2 candidate: largest >= 1;
                    // the sum for step 3 in ascending order (+0 entries add nothing)
                    if (acc < (T)0) { acc = (T)0; changed = true; }
                    if (acc >= (T)1 && acc > best) { best = acc; bestid = a; }
                    ssum = ssum + acc;
                }
                if (chunked) P.out[o] = acc;
                else S.nv(aa) = acc;
            }
        }
        // S step 2 (the >= 1 rule); the sum for step 3 is formed above
        if (mob) {
            const int r = mob_project<T>(N, Vs, P.out + i, tabL);
            if (r == -1) raise_flag(P.flag, FLAG_SIMPLEX);
            if (r == -2) raise_flag(P.flag, FLAG_NZ_OVERFLOW);
            changed = r == 1;
        } else if (project) {
            if (bestid >= 0) {
                // the winner becomes 1, the others 0; the sum is then exactly 1
                if (!chunked) {
                    for (int aa = 0; aa < N; ++aa) {
                        const T w = (aa == bestid) ? (T)1 : (T)0;
                        if (S.nv(aa) != w) changed = true;
                    }
                } else {
                    changed = true;
                }
                ssum = (T)1;
            }
            if (!(ssum > (T)0)) raise_flag(P.flag, FLAG_SIMPLEX);
        }
        const bool fix = has_r0out && P.fix_first && changed;
        // a cell whose values are final as written (sum exactly 1, no >= 1 rule,
        // nothing else to store) is not swept again: the bulk of every grain
        const bool final_vals = chunked && !mob && bestid < 0 && (!project || ssum == (T)1) && !fix && !emb &&
                                !has_out2;
        // store pass: S step 3, first-stage fix, embedded error, SSP(10)4 mid combination
        int nc = 0;
        if (!final_vals) {
            long long o = i;
#pragma unroll 4
            for (int a = 0; a < N; ++a, o += Vs) {
                T w = chunked ? P.out[o] : S.nv(a);
                if (project && !mob) {
                    if (bestid >= 0) w = (a == bestid) ? (T)1 : (T)0;
                    else if (ssum > (T)0 && ssum != (T)1 && !zbits(w)) w = w / ssum;
                }
                if (fix) P.r0out[o] = (w - ldg(P.in + o)) / b1c;
                if (emb) {
                    const T zv = P.zout[o];
                    T e = w - zv;
                    if (zv < (T)0 || zv > (T)1) e = (T)0;
                    if (e != (T)0) {
                        const T au = tabs(ldg(P.uw + o)), av = tabs(w);
                        const T wt = (T)P.r_phi * (au > av ? au : av) + (T)P.a_phi;
                        const T q = e / wt;
                        esum += (double)(q * q);
                        nc++;
                    }
                }
                if (has_out2) {
                    const T q2 = w + (T)P.m25 * (ldg(P.q2in + o) - w);
                    P.out2[o] = q2;
                    P.out[o] = w + (T)P.m15 * (q2 - w);
                } else {
                    P.out[o] = w;
                }
            }
        }
        if (emb) ecnt += (nc > 0 ? nc : 2);
        // concentration field (no projection)
        if (K) {
            const long long o = (long long)N * Vs + i;
            // the small increments are summed first: c is rounded once per stage
            T d = b1c * rc;
            if (has_r0in) d = d + b0c * ldg(P.r0in + o);
            if (has_p0) d = d + a0c * (ldg(P.p0 + o) - cc);
            if (has_p2) d = d + a2c * (ldg(P.p2 + o) - cc);
            const T acc = cc + d;
            if (!isfinite(acc)) raise_flag(P.flag, FLAG_NONFINITE);
            if (has_r0out) P.r0out[o] = rc;
            if (has_z) {
                const T zv = P.zin[o] + bzc * rc;
                P.zout[o] = zv;
                if (emb) {
                    const T e = acc - zv;
                    const T au = tabs(ldg(P.uw + o) + (T)g.cref), av = tabs(acc + (T)g.cref);
                    const T wt = (T)P.r_c * (au > av ? au : av) + (T)P.a_c;
                    const T q = e / wt;
                    esum += (double)(q * q);
                    ecnt += 1;
                }
            }
            if (has_out2) {
                const T q2 = acc + (T)P.m25 * (ldg(P.q2in + o) - acc);
                P.out2[o] = q2;
                P.out[o] = acc + (T)P.m15 * (q2 - acc);
            } else {
                P.out[o] = acc;
            }
        }
    }
#undef PF_NEXT_RHS
    return true;
}

// Occupancy words (masked storage) of the cell's outputs after the wide path
// rewrote every phase of it: bit set where the value is nonzero.
__device__ __forceinline__ void wide_masks(const Geom &g, const Pass<float> &P, long long i)
{
    const int nwr = (g.N + 31) / 32;
    for (int w = 0; w < nwr; ++w) {
        unsigned mo = 0u, mr = 0u, mz = 0u, m2 = 0u;
        for (int b = 0; b < 32 && 32 * w + b < g.N; ++b) {
            const long long o = (long long)(32 * w + b) * g.Vs + i;
            if (P.out[o] != 0.0f) mo |= 1u << b;
            if (P.r0out && P.r0out[o] != 0.0f) mr |= 1u << b;
            if (P.zout && P.zout[o] != 0.0f) mz |= 1u << b;
            if (P.out2 && P.out2[o] != 0.0f) m2 |= 1u << b;
        }
        const long long ow = (long long)w * g.Vs + i;
        if (P.m_out) P.m_out[ow] = mo;
        if (P.m_r0out) P.m_r0out[ow] = mr;
        if (P.m_zout) P.m_zout[ow] = mz;
        if (P.m_out2) P.m_out2[ow] = m2;
    }
}
__device__ __forceinline__ void wide_masks(const Geom &, const Pass<double> &, long long) {}

// A cell where more than MAXACT phases are nontrivial (phases crowding at
// junctions and particle fringes; Sec. 3.1 sets no limit): the whole cell is
// recomputed by the generic body with a WIDEACT-entry list in local memory,
// rewriting every output of the pass for this cell (and, in masked storage,
// its occupancy words); its error-norm contribution is added to esum/ecnt,
// which the caller has reset.  Beyond WIDEACT phases the pass raises
// FLAG_NZ_OVERFLOW.  Kept out of line: its local array is touched only by
// the rare threads that take it.
template <typename T, int DIM, int KC>
__device__ __noinline__ void wide_cell(const Geom *g, const Pass<T> *P, const T *tabA, const T *tabB, const T *tabL,
                                       const signed char *ptype, int x, int y, int z, double *esum, long long *ecnt)
{
    WideList<T> L;
    double es = 0.0;
    long long ec = 0;
    if (!cell_core<T, DIM, KC, SIG_GENERIC, WideList<T>>(*g, *P, L, tabA, tabB, tabL, ptype, x, y, z, es, ec)) {
        raise_flag(P->flag, FLAG_NZ_OVERFLOW);
        return;
    }
    if (P->mode == MODE_STAGE) wide_masks(*g, *P, ((long long)z * g->ny + y) * g->nx + x);
    *esum += es;
    *ecnt += ec;
}

template <typename T, int DIM, int KC, unsigned SIG>
__device__ __forceinline__ void cell_body(const Geom &g, const Pass<T> &P, const T *__restrict__ tabA,
                                          const T *__restrict__ tabB, const T *__restrict__ tabL,
                                          const signed char *__restrict__ ptype)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    if (pass_skipped(P.flag)) return;
    SlotList<T> S{reinterpret_cast<Smem<T> *>(smem_raw), (int)threadIdx.x};
    const int tid = threadIdx.x;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int x = blockIdx.x * TX + (tid % TX);
    const int y = blockIdx.y * TY + (tid / TX);
    const int z = blockIdx.z;
    double esum = 0.0;
    long long ecnt = 0;
    if (x < g.nx && y < g.ny) {
        if (!cell_core<T, DIM, KC, SIG, SlotList<T>>(g, P, S, tabA, tabB, tabL, ptype, x, y, z, esum, ecnt))
            wide_cell<T, DIM, KC>(&g, &P, tabA, tabB, tabL, ptype, x, y, z, &esum, &ecnt);
    }
    const bool errp = (SIG & SIG_GENERIC) ? (P.mode == MODE_ERR || P.embedded_err != 0) : (SIG & SIG_ERR) != 0;
    if (errp) block_partials(esum, ecnt, P.part_sum, P.part_cnt, bid, P.part_n);
    if (P.count_step) count_step_done(P.flag);
}

template <typename T, int DIM, int KC, unsigned SIG>
__global__ void __launch_bounds__(BLOCK)
cell_kernel(const __grid_constant__ Geom g, const __grid_constant__ Pass<T> P, const T *__restrict__ tabA,
            const T *__restrict__ tabB, const T *__restrict__ tabL, const signed char *__restrict__ ptype)
{
    cell_body<T, DIM, KC, SIG>(g, P, tabA, tabB, tabL, ptype);
}

// The same pass with its description read from device memory: the passes
// of device-driven adaptive steps, whose buffers and coefficients a planning
// kernel writes before each launch runs.
template <typename T, int DIM, int KC, unsigned SIG>
__global__ void __launch_bounds__(BLOCK)
cell_kernel_d(const __grid_constant__ Geom g, const Pass<T> *__restrict__ Pd, const T *__restrict__ tabA,
              const T *__restrict__ tabB, const T *__restrict__ tabL, const signed char *__restrict__ ptype)
{
    __shared__ Pass<T> Ps;
    if (threadIdx.x == 0) Ps = *Pd;
    __syncthreads();
    cell_body<T, DIM, KC, SIG>(g, Ps, tabA, tabB, tabL, ptype);
}

// ---------------------------------------------------------------------------
// TMA staging (sm_90+ bulk tensor copies, used on sm_103a): a block streams
// the phase planes of its 32x8 tile through a ring of TMA_R shared-memory
// slots.  Slot r holds, for one phase, the stencil input's planes z-1, z, z+1
// (one 4D box of 32x8x3 cells) and the pointwise inputs' plane z, and is
// signalled by an mbarrier with a transaction count.  Every wait is bounded.
// ---------------------------------------------------------------------------
constexpr int TMA_R = 4;
constexpr unsigned TMA_SPIN = 1u << 22;   // bounded mbarrier polls before giving up

struct TmaMaps {
    CUtensorMap in3;   // stencil input, box 32 x 8 x 3 planes x 1 field
    CUtensorMap in1;   // stencil input, box 32 x 8 x 1 (domain z faces)
    CUtensorMap p0, p2, r0;   // pointwise inputs, box 32 x 8 x 1 x 1
};

template <typename T>
struct ListSmem;

struct alignas(1024) TmaSmem {
    float in[TMA_R][3][TY][TX];
    float p0[TMA_R][TY][TX];
    float p2[TMA_R][TY][TX];
    float r0[TMA_R][TY][TX];
    unsigned long long full[TMA_R];    // copies of the slot landed (tx count)
    unsigned long long empty[TMA_R];   // every consumer warp has read the slot
};

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *b, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(b)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bounded wait: false after `polls` polls (the caller raises FLAG_TIMEOUT).
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, unsigned parity, unsigned polls = TMA_SPIN)
{
    for (unsigned k = 0; k < polls; ++k)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load4(void *dst, const CUtensorMap *m, int x, int y, int z, int f,
                                          unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(smem_u32(dst)), "l"((unsigned long long)m), "r"(x), "r"(y), "r"(z), "r"(f), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory slots of the per-cell active list (no stage values).
template <typename T>
struct ListSmem {
    unsigned char id[MAXACT][BLOCK];
    T lap[MAXACT][BLOCK];    // Laplacian, later the RHS of the listed phase
    T cen[MAXACT][BLOCK];    // phi at the cell
    T dl[MAXACT][BLOCK];     // variational derivative
    T val[MAXACT][BLOCK];    // stage value of the listed phase (N > 32 path)
};

// Loader policies of the FP32 fast path: where the values of phase a come
// from.  PlainLoader reads global memory; TmaLoader reads the shared-memory
// ring filled by the producer warp (and releases the slot afterwards).
template <int DIM>
struct PlainLoader {
    // per-phase base pointers (64-bit phase offsets a * Vs) are the same for
    // every thread (uniform); the per-thread part is a 32-bit cell index
    // (Vs < 2^31, checked at dispatch)
    const float *in, *p0, *p2, *r0;
    int Vs, nph;
    int ic, inb[6];
    __device__ __forceinline__ void load(int a, long long, float &v0, float *nb, float &p0v, float &p2v, float &r0v,
                                         bool hp0, bool hp2, bool hr0)
    {
        if (PF_PREFETCH_DIST > 0 && a + PF_PREFETCH_DIST < nph) {   // stays inside the phase fields
            const long long pa = (long long)(a + PF_PREFETCH_DIST) * Vs + ic;
            prefetch_l2(in + pa);
            if (hp0) prefetch_l2(p0 + pa);
            if (hp2) prefetch_l2(p2 + pa);
            if (hr0) prefetch_l2(r0 + pa);
        }
        const float *b = in + (long long)a * Vs;
        v0 = ldg(b + ic);
#pragma unroll
        for (int f = 0; f < 2 * DIM; ++f) nb[f] = ldg(b + inb[f]);
        if (hp0) p0v = ld_stream(p0 + (long long)a * Vs + ic);
        if (hp2) p2v = ld_stream(p2 + (long long)a * Vs + ic);
        if (hr0) r0v = ld_stream(r0 + (long long)a * Vs + ic);
    }
    __device__ __forceinline__ void release(int) {}
};

struct TmaLoader {
    TmaSmem *Q;
    const float *pin;
    int off[6];
    int tx, ty;
    bool zin;
    bool ok;
    __device__ __forceinline__ void load(int a, long long fo, float &v0, float *nb, float &p0v, float &p2v, float &r0v,
                                         bool hp0, bool hp2, bool hr0)
    {
        const int r = a % TMA_R;
        if (ok && !mbar_wait(&Q->full[r], (unsigned)((a / TMA_R) & 1))) ok = false;
        if (!ok) {
            // a wait gave up (the pass reports PF_ETIMEOUT): touch no slot
            // any more; the stencil values come from global memory, the
            // pointwise ones are zero (the results of this pass are void)
            v0 = ldg(pin + fo);
#pragma unroll
            for (int f = 0; f < 6; ++f) nb[f] = ldg(pin + fo + off[f]);
            p0v = p2v = r0v = 0.0f;
            return;
        }
        v0 = Q->in[r][1][ty][tx];
        nb[0] = tx > 0 ? Q->in[r][1][ty][tx - 1] : ldg(pin + fo + off[0]);
        nb[1] = tx < TX - 1 ? Q->in[r][1][ty][tx + 1] : ldg(pin + fo + off[1]);
        nb[2] = ty > 0 ? Q->in[r][1][ty - 1][tx] : ldg(pin + fo + off[2]);
        nb[3] = ty < TY - 1 ? Q->in[r][1][ty + 1][tx] : ldg(pin + fo + off[3]);
        nb[4] = zin ? Q->in[r][0][ty][tx] : ldg(pin + fo + off[4]);
        nb[5] = zin ? Q->in[r][2][ty][tx] : ldg(pin + fo + off[5]);
        if (hp0) p0v = Q->p0[r][ty][tx];
        if (hp2) p2v = Q->p2[r][ty][tx];
        if (hr0) r0v = Q->r0[r][ty][tx];
    }
    // one arrival per consumer warp once all its lanes have read slot a
    // (none once a wait gave up: the producer then stops issuing copies)
    __device__ __forceinline__ void release(int a)
    {
        const bool all_ok = __all_sync(0xffffffffu, ok);
        if ((threadIdx.x & 31) == 0 && all_ok) mbar_arrive(&Q->empty[a % TMA_R]);
    }
};

// Per-cell body of the FP32 fast path (N <= NMAX).  The loop over phases is
// unrolled NMAX times (guarded by a < N) so the stage values stay in
// registers and the loads of a phase (stencil and pointwise) issue together.
// A phase that is not nontrivial has a zero RHS, so its stage value (or error
// term) is final in that first loop; only the N_z listed phases receive their
// RHS term after the pairwise sums.  Rounding order differs from the generic
// kernel; FP32 is not compared bit for bit.
template <int DIM, int KC, unsigned SIG, int NMAX, class LD>
__device__ __forceinline__ bool fast_cell(const Geom &g, const Pass<float> &P, LD &ld, ListSmem<float> &S, int tid,
                                          long long i, const int *off, const int *ghost, const float *tabA,
                                          const float *tabB, const float *tabL, const signed char *ptype,
                                          double &esum, long long &ecnt)
{
    typedef float T;
    constexpr int NFACE = 2 * DIM;
    constexpr bool ERR = (SIG & SIG_ERR) != 0;
    constexpr bool HP0 = (SIG & SIG_P0) != 0 || ERR;
    constexpr bool HP2 = (SIG & SIG_P2) != 0;
    constexpr bool HR0 = (SIG & SIG_R0IN) != 0 || ERR;
    constexpr bool R0OUT = (SIG & SIG_R0OUT) != 0;
    constexpr bool PROJ = (SIG & SIG_PROJECT) != 0;
    const int N = g.N;
    const int Vs = (int)g.Vs;
    const int i32 = (int)i;
    const T idx2 = (T)(1.0 / g.dx2);
    const T a0c = (T)P.a0, a2c = (T)P.a2, b1c = (T)P.b1, b0c = (T)P.b0;
    const T ib1 = (T)(1.0 / P.b1);   // first-stage fix: F <- (S(u1) - u^n) / (mu~_1 dt)
    const T dt = (T)P.dt, rph = (T)P.r_phi, aph = (T)P.a_phi;

    // concentration
    T cc = (T)0, num_c = (T)0, den_c = (T)0, num_n[NFACE], den_n[NFACE], mf[NFACE];
#pragma unroll
    for (int f = 0; f < NFACE; ++f) { num_n[f] = (T)0; den_n[f] = (T)0; mf[f] = (T)0; }
    if (KC) {
        const T *cf = P.in + (long long)N * Vs + i;
        cc = ldg(cf);
        num_c = cc;
#pragma unroll
        for (int f = 0; f < NFACE; ++f) {
            T v = ldg(cf + off[f]);
            if (ghost[f] && g.bc_c[f] == BC_DIRICHLET) v = (T)2 * (T)g.cdir[f] - cc;
            num_n[f] = v;
        }
    }

    int nz = 0, nc = 0;
    bool changed = false;
    T best = (T)-1, ssum = (T)0;
    int bestid = -1;
    T nv[NMAX];
    unsigned actmask = 0u;
#pragma unroll
    for (int a = 0; a < NMAX; ++a) {
        nv[a] = (T)0;
        if (a < N) {
            const long long fo = (long long)a * Vs;
            T v0, nb[NFACE], p0v = (T)0, p2v = (T)0, r0v = (T)0;
            ld.load(a, fo, v0, nb, p0v, p2v, r0v, HP0, HP2, HR0);
            ld.release(a);
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
            if (act) {
                T l = (T)0;
#pragma unroll
                for (int f = 0; f < NFACE; ++f) l = l + (nb[f] - v0);
                if (nz < MAXACT) {
                    S.id[nz][tid] = (unsigned char)a;
                    S.lap[nz][tid] = l * idx2;
                    S.cen[nz][tid] = v0;
                    actmask |= 1u << a;
                }
                nz++;
            }
            if (ERR) {
                // in = u^{n+1}, p0 = u^n, r0in = F^n; a trivial phase has F^{n+1} = 0
                if (!act) {
                    T e = ((T)12 * (p0v - v0) + ((T)6 * dt) * r0v) * ((T)1 / (T)15);
                    const T trial = p0v + (dt * (T)0.5) * r0v;
                    if (trial < (T)0 || trial > (T)1) e = (T)0;
                    if (e != (T)0) {
                        const T w = rph * fmaxf(fabsf(p0v), fabsf(v0)) + aph;
                        const T q = e / w;
                        esum += (double)(q * q);
                        nc++;
                    }
                }
            } else {
                T acc = affine<HP0, HP2>(v0, p0v, p2v, a0c, a2c);
                if (HR0) acc = acc + b0c * r0v;
                if (!act && PROJ) {
                    if (acc < (T)0) { acc = (T)0; changed = true; }
                    if (acc >= (T)1 && acc > best) { best = acc; bestid = a; }
                    ssum = ssum + acc;
                }
                nv[a] = acc;
            }
        }
    }
    if (nz > MAXACT) return false;      // crowded cell: the caller takes the wide path

    T mu = (T)0, rc = (T)0;
    if (KC) {
        mu = num_c / den_c;
        T acc = (T)0;
#pragma unroll
        for (int f = 0; f < NFACE; ++f) acc = acc + mf[f] * (num_n[f] / den_n[f] - mu);
        rc = acc * idx2;
    }
    // variational derivative and pairwise sum over the listed phases
    for (int k = 0; k < nz; ++k) {
        const int a = S.id[k][tid];
        const T *Aa = tabA + a * N, *Ba = tabB + a * N;
        T d = (T)0;
        for (int k2 = 0; k2 < nz; ++k2) {
            if (k2 == k) continue;
            const int b = S.id[k2][tid];
            d = d + (ldg(Aa + b) * S.lap[k2][tid] + ldg(Ba + b) * S.cen[k2][tid]);
        }
        if (KC) {
            const int t = ptype[a];
            d = d + (-(mu * mu) / ((T)2 * (T)g.k[t]) - mu * (T)g.c0[t]);
        }
        S.dl[k][tid] = d;
    }
    const T inz = nz > 1 ? (T)1 / (T)nz : (T)0;
    for (int k = 0; k < nz; ++k) {
        T rk = (T)0;
        if (nz > 1) {
            const int a = S.id[k][tid];
            const T *La = tabL + a * N;
            const T dk = S.dl[k][tid];
            T s = (T)0;
            for (int k2 = 0; k2 < nz; ++k2) {
                if (k2 == k) continue;
                s = s + ldg(La + S.id[k2][tid]) * (dk - S.dl[k2][tid]);
            }
            rk = -(s * inz);
        }
        S.lap[k][tid] = rk;                 // the list now holds the RHS
        if (ERR) {
            const int a = S.id[k][tid];
            const long long fo = (long long)a * Vs;
            const T p0v = ldg(P.p0 + fo + i), v0 = S.cen[k][tid], r0v = ldg(P.r0in + fo + i);
            const T sr = r0v + rk;
            T e = ((T)12 * (p0v - v0) + ((T)6 * dt) * sr) * ((T)1 / (T)15);
            const T trial = p0v + (dt * (T)0.5) * sr;
            if (trial < (T)0 || trial > (T)1) e = (T)0;
            if (e != (T)0) {
                const T w = rph * fmaxf(fabsf(p0v), fabsf(v0)) + aph;
                const T q = e / w;
                esum += (double)(q * q);
                nc++;
            }
        }
    }
    if (ERR) {
        ecnt += (nc > 0 ? nc : 2);
        if (KC) {
            const long long o = (long long)N * Vs + i;
            const T un = ldg(P.p0 + o), un1 = cc, rn = ldg(P.r0in + o);
            const T e = ((T)12 * (un - un1) + ((T)6 * dt) * (rn + rc)) * ((T)1 / (T)15);
            const T w = (T)P.r_c * fmaxf(fabsf(un + (T)g.cref), fabsf(un1 + (T)g.cref)) + (T)P.a_c;
            const T q = e / w;
            esum += (double)(q * q);
            ecnt += 1;
        }
        return true;
    }
    // listed phases: add the RHS term, clamp, >= 1 candidates, sum
    {
        int kk = 0;
#pragma unroll
        for (int a = 0; a < NMAX; ++a) {
            if ((actmask >> a) & 1u) {
                const T rk = S.lap[kk][tid];
                kk++;
                T acc = nv[a] + b1c * rk;
                if (PROJ) {
                    if (acc < (T)0) { acc = (T)0; changed = true; }
                    if (acc >= (T)1 && (acc > best || (acc == best && a < bestid))) { best = acc; bestid = a; }
                    ssum = ssum + acc;
                }
                nv[a] = acc;
            }
        }
    }
    if (PROJ) {
        if (bestid >= 0) {
#pragma unroll
            for (int a = 0; a < NMAX; ++a)
                if (a < N && nv[a] != ((a == bestid) ? (T)1 : (T)0)) changed = true;
            ssum = (T)1;
        }
        if (!(ssum > (T)0)) raise_flag(P.flag, FLAG_SIMPLEX);
    }
    const T inv = (ssum > (T)0) ? (T)1 / ssum : (T)1;
    const bool fix = R0OUT && P.fix_first && changed;
    int kr = 0;      // list cursor for the RHS of listed phases (R0OUT)
#pragma unroll
    for (int a = 0; a < NMAX; ++a) {
        if (a < N) {
            const long long fo = (long long)a * Vs;
            T w = nv[a];
            if (PROJ) w = (bestid >= 0) ? ((a == bestid) ? (T)1 : (T)0) : w * inv;
            if (R0OUT) {
                T r = (T)0;
                if ((actmask >> a) & 1u) { r = S.lap[kr][tid]; kr++; }
                if (fix) r = (w - ldg(P.in + fo + i)) * ib1;
                (P.r0out + fo)[i32] = r;
            }
            (P.out + fo)[i32] = w;
        }
    }
    if (KC) {
        const long long o = (long long)N * Vs + i;
        // the small increments are summed first: c is rounded once per stage
        T d = b1c * rc;
        if (HR0) d = d + b0c * ldg(P.r0in + o);
        if (HP0) d = d + a0c * (ldg(P.p0 + o) - cc);
        if (HP2) d = d + a2c * (ldg(P.p2 + o) - cc);
        const T acc = cc + d;
        if (!isfinite(acc)) raise_flag(P.flag, FLAG_NONFINITE);
        if (R0OUT) P.r0out[o] = rc;
        P.out[o] = acc;
    }
    return true;
}

// Bits of occupancy word w that belong to phases below N.
__device__ __forceinline__ unsigned word_bits(int N, int w)
{
    const int r = N - 32 * w;
    return r >= 32 ? 0xffffffffu : (r <= 0 ? 0u : ((1u << r) - 1u));
}

// Per-cell body of the FP32 fast path in masked storage (N <= 32 NW).  The
// arithmetic and its order are those of fast_cell; what changes is which
// phases are visited: the warp walks the union of its lanes' occupied phases
// (the occupancy words of the stencil input at the cell and its face
// neighbours and of the pointwise inputs), word by word, in a rolled loop,
// so the code stays small, and a lane loads only the entries whose bits are
// set (the others are zero).  A phase outside the union has a zero RHS and a
// zero stage value; it is written only where the output still holds an
// older nonzero value.  Stage values live in a per-thread array indexed by
// phase (local memory, of which only the visited entries are touched).
// Word w of a cell's occupancy covers phases 32w .. 32w + 31 and lives in
// the plane at w * Vs.
template <int DIM, int KC, unsigned SIG, bool OCC = true, int NW = 1>
__device__ __forceinline__ void masked_cell(const Geom &g, const Pass<float> &P, ListSmem<float> &S, int tid,
                                            long long i, const int *off, const int *ghost, const float *tabA,
                                            const float *tabB, const float *tabL, const signed char *ptype,
                                            double &esum, long long &ecnt, unsigned am, bool &over)
{
    typedef float T;
    constexpr int NFACE = 2 * DIM;
    constexpr bool ERR = (SIG & SIG_ERR) != 0;
    constexpr bool HP0 = (SIG & SIG_P0) != 0 || ERR;
    constexpr bool HP2 = (SIG & SIG_P2) != 0;
    constexpr bool HR0 = (SIG & SIG_R0IN) != 0 || ERR;
    constexpr bool R0OUT = (SIG & SIG_R0OUT) != 0;
    constexpr bool PROJ = (SIG & SIG_PROJECT) != 0;
    constexpr bool EMB = (SIG & SIG_EMB) != 0;
    constexpr bool HZ = (SIG & SIG_Z) != 0 || EMB;
    constexpr bool HO2 = (SIG & SIG_O2) != 0;
    const int N = g.N;
    const int Vs = (int)g.Vs;
    const int i32 = (int)i;
    const T idx2 = (T)(1.0 / g.dx2);
    const T a0c = (T)P.a0, a2c = (T)P.a2, b1c = (T)P.b1, b0c = (T)P.b0;
    const T ib1 = (T)(1.0 / P.b1);   // first-stage fix: F <- (S(u1) - u^n) / (mu~_1 dt)
    const T dt = (T)P.dt, rph = (T)P.r_phi, aph = (T)P.a_phi;
    const T bzc = (T)P.bz, m25 = (T)P.m25, m15 = (T)P.m15;

    // concentration
    T cc = (T)0, num_c = (T)0, den_c = (T)0, num_n[NFACE], den_n[NFACE], mf[NFACE];
#pragma unroll
    for (int f = 0; f < NFACE; ++f) { num_n[f] = (T)0; den_n[f] = (T)0; mf[f] = (T)0; }
    if (KC) {
        const T *cf = P.in + (long long)N * Vs + i;
        cc = ldg(cf);
        num_c = cc;
#pragma unroll
        for (int f = 0; f < NFACE; ++f) {
            T v = ldg(cf + off[f]);
            if (ghost[f] && g.bc_c[f] == BC_DIRICHLET) v = (T)2 * (T)g.cdir[f] - cc;
            num_n[f] = v;
        }
    }

    // occupancy: U[w] is the warp's union of word w (a uniform loop bound).
    // Without words (OCC false: dense storage) every phase is occupied.
    // only the words of existing phases exist in memory: w < nwr
    const int nwr = (N + 31) / 32;
    unsigned U[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const unsigned full = word_bits(N, w);
        unsigned u = full;
        if (OCC && w < nwr) {
            const long long o = (long long)w * Vs + i;
            u = __ldg(P.m_in + o);
#pragma unroll
            for (int f = 0; f < NFACE; ++f) u |= __ldg(P.m_in + o + off[f]);
            if (HP0) u |= __ldg(P.m_p0 + o);
            if (HP2) u |= __ldg(P.m_p2 + o);
            if (HR0) u |= __ldg(P.m_r0 + o);
            u = __reduce_or_sync(am, u) & full;
        }
        U[w] = u;
    }

    int nz = 0, nc = 0;
    bool changed = false;
    T best = (T)-1, ssum = (T)0;
    int bestid = -1;
    T nv[32 * NW];
    unsigned actmask[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) actmask[w] = 0u;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      if (w >= nwr || !U[w]) continue;
      const unsigned full = word_bits(N, w);
      const long long ow = (long long)w * Vs + i;
      const unsigned mc = OCC ? __ldg(P.m_in + ow) : full;
      unsigned mnb[NFACE];
#pragma unroll
      for (int f = 0; f < NFACE; ++f) mnb[f] = OCC ? __ldg(P.m_in + ow + off[f]) : full;
      const unsigned mp0 = HP0 ? (OCC ? __ldg(P.m_p0 + ow) : full) : 0u;
      const unsigned mp2 = HP2 ? (OCC ? __ldg(P.m_p2 + ow) : full) : 0u;
      const unsigned mr0 = HR0 ? (OCC ? __ldg(P.m_r0 + ow) : full) : 0u;
      for (unsigned m = U[w]; m; m &= m - 1u) {
        const int bit = __ffs(m) - 1;
        const int a = 32 * w + bit;
        const long long fo = (long long)a * Vs;
        const T *b = P.in + fo + i;
        if (!OCC && PF_PREFETCH_DIST > 0 && a + PF_PREFETCH_DIST < N) {
            const long long pa = (long long)PF_PREFETCH_DIST * Vs;
            prefetch_l2(b + pa);
            if (HP0) prefetch_l2(P.p0 + fo + pa + i);
            if (HP2) prefetch_l2(P.p2 + fo + pa + i);
            if (HR0) prefetch_l2(P.r0in + fo + pa + i);
        }
        const T v0 = ((mc >> bit) & 1u) ? ldg(b) : (T)0;
        T nb[NFACE];
#pragma unroll
        for (int f = 0; f < NFACE; ++f) nb[f] = ((mnb[f] >> bit) & 1u) ? ldg(b + off[f]) : (T)0;
        T p0v = (T)0, p2v = (T)0, r0v = (T)0;
        if (HP0 && ((mp0 >> bit) & 1u)) p0v = ld_stream(P.p0 + fo + i);
        if (HP2 && ((mp2 >> bit) & 1u)) p2v = ld_stream(P.p2 + fo + i);
        if (HR0 && ((mr0 >> bit) & 1u)) r0v = ld_stream(P.r0in + fo + i);
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
        if (act) {
            T l = (T)0;
#pragma unroll
            for (int f = 0; f < NFACE; ++f) l = l + (nb[f] - v0);
            if (nz < MAXACT) {
                S.id[nz][tid] = (unsigned char)a;
                S.lap[nz][tid] = l * idx2;
                S.cen[nz][tid] = v0;
                actmask[w] |= 1u << bit;
            }
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
        } else {
            T acc = affine<HP0, HP2>(v0, p0v, p2v, a0c, a2c);
            if (HR0) acc = acc + b0c * r0v;
            if (!act && PROJ) {
                if (acc < (T)0) { acc = (T)0; changed = true; }
                if (acc >= (T)1 && acc > best) { best = acc; bestid = a; }
                ssum = ssum + acc;
            }
            nv[a] = acc;
        }
      }
    }
    // a crowded cell finishes with the truncated list (the warp's collective
    // operations below need every lane) and is then redone on the wide path
    if (nz > MAXACT) {
        over = true;
        nz = MAXACT;
    }

    T mu = (T)0, rc = (T)0;
    if (KC) {
        mu = num_c / den_c;
        T acc = (T)0;
#pragma unroll
        for (int f = 0; f < NFACE; ++f) acc = acc + mf[f] * (num_n[f] / den_n[f] - mu);
        rc = acc * idx2;
    }
    // variational derivative and pairwise sum over the listed phases
    for (int k = 0; k < nz; ++k) {
        const int a = S.id[k][tid];
        const T *Aa = tabA + a * N, *Ba = tabB + a * N;
        T d = (T)0;
        for (int k2 = 0; k2 < nz; ++k2) {
            if (k2 == k) continue;
            const int b = S.id[k2][tid];
            d = d + (ldg(Aa + b) * S.lap[k2][tid] + ldg(Ba + b) * S.cen[k2][tid]);
        }
        if (KC) {
            const int t = ptype[a];
            d = d + (-(mu * mu) / ((T)2 * (T)g.k[t]) - mu * (T)g.c0[t]);
        }
        S.dl[k][tid] = d;
    }
    const T inz = nz > 1 ? (T)1 / (T)nz : (T)0;
    for (int k = 0; k < nz; ++k) {
        T rk = (T)0;
        if (nz > 1) {
            const int a = S.id[k][tid];
            const T *La = tabL + a * N;
            const T dk = S.dl[k][tid];
            T s = (T)0;
            for (int k2 = 0; k2 < nz; ++k2) {
                if (k2 == k) continue;
                s = s + ldg(La + S.id[k2][tid]) * (dk - S.dl[k2][tid]);
            }
            rk = -(s * inz);
        }
        S.lap[k][tid] = rk;                 // the list now holds the RHS
        if (ERR) {
            const int a = S.id[k][tid];
            const long long fo = (long long)a * Vs;
            const T p0v = ldg(P.p0 + fo + i), v0 = S.cen[k][tid], r0v = ldg(P.r0in + fo + i);
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
    if (ERR) {
        if constexpr (R0OUT && !OCC) {
            // keep F(u^{n+1}), the RHS just evaluated, for reuse as the next
            // step's F(u^n) (listed phases in ascending order, others zero)
            int kr = 0;
            for (int a = 0; a < N; ++a) {
                T r = (T)0;
                if (kr < nz && S.id[kr][tid] == a) { r = S.lap[kr][tid]; kr++; }
                (P.r0out + (long long)a * Vs)[i32] = r;
            }
            if (KC) P.r0out[(long long)N * Vs + i] = rc;
        }
        ecnt += (nc > 0 ? nc : 2);
        if (KC) {
            const long long o = (long long)N * Vs + i;
            const T un = ldg(P.p0 + o), un1 = cc, rn = ldg(P.r0in + o);
            const T e = ((T)12 * (un - un1) + ((T)6 * dt) * (rn + rc)) * ((T)1 / (T)15);
            const T wt = (T)P.r_c * fmaxf(fabsf(un + (T)g.cref), fabsf(un1 + (T)g.cref)) + (T)P.a_c;
            const T q = e / wt;
            esum += (double)(q * q);
            ecnt += 1;
        }
        return;
    }
    // listed phases (ascending ids): add the RHS term, clamp, >= 1 candidates, sum
    {
        int kk = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w)
        for (unsigned m = actmask[w]; m; m &= m - 1u) {
            const int a = 32 * w + __ffs(m) - 1;
            const T rk = S.lap[kk][tid];
            kk++;
            T acc = nv[a] + b1c * rk;
            if (PROJ) {
                if (acc < (T)0) { acc = (T)0; changed = true; }
                if (acc >= (T)1 && (acc > best || (acc == best && a < bestid))) { best = acc; bestid = a; }
                ssum = ssum + acc;
            }
            nv[a] = acc;
        }
    }
    if (PROJ) {
        if (bestid >= 0) {
#pragma unroll
            for (int w = 0; w < NW; ++w)
                for (unsigned m = U[w]; m; m &= m - 1u) {
                    const int a = 32 * w + __ffs(m) - 1;
                    if (nv[a] != ((a == bestid) ? (T)1 : (T)0)) changed = true;
                }
            ssum = (T)1;
        }
        // (a crowded cell's truncated sum says nothing: the wide path decides)
        if (!(ssum > (T)0) && !over) raise_flag(P.flag, FLAG_SIMPLEX);
    }
    const T inv = (ssum > (T)0) ? (T)1 / ssum : (T)1;
    const bool fix = R0OUT && P.fix_first && changed;
    int kr = 0;      // list cursor for the RHS of listed phases (R0OUT, z)
    int nce = 0;     // entries of the SSP(10)4 embedded error
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        if (w >= nwr) break;
        const unsigned full = word_bits(N, w);
        const long long ow = (long long)w * Vs + i;
        const unsigned mo_old = OCC ? P.m_out[ow] : 0u;
        const unsigned mr_old = (R0OUT && OCC) ? P.m_r0out[ow] : 0u;
        // SSP(10)4: a phase held by z or by q2in gets a z or q2 entry (and,
        // through the q2 combination, an output entry) where its stage value
        // is zero
        const unsigned mzi = (HZ && OCC) ? P.m_zin[ow] : full;
        const unsigned mz_old = (HZ && OCC) ? P.m_zout[ow] : 0u;
        const unsigned mq2 = (HO2 && OCC) ? __ldg(P.m_q2in + ow) : full;
        const unsigned m2_old = (HO2 && OCC) ? P.m_out2[ow] : 0u;
        const unsigned muw = (EMB && OCC) ? __ldg(P.m_uw + ow) : full;
        unsigned tu = U[w] | mo_old | mr_old;
        if (HZ) tu |= mzi | mz_old;
        if (HO2) tu |= mq2 | m2_old;
        const unsigned touch = OCC ? (__reduce_or_sync(am, tu) & full) : full;
        unsigned nmask = 0u, nrmask = 0u, nzmask = 0u, n2mask = 0u;
        for (unsigned m = touch; m; m &= m - 1u) {
            const int bit = __ffs(m) - 1;
            const int a = 32 * w + bit;
            const long long fo = (long long)a * Vs;
            T wv = ((U[w] >> bit) & 1u) ? nv[a] : (T)0;
            if (PROJ) wv = (bestid >= 0) ? ((a == bestid) ? (T)1 : (T)0) : wv * inv;
            T rl = (T)0;     // RHS of the phase (zero unless listed)
            if (R0OUT || HZ)
                if ((actmask[w] >> bit) & 1u) { rl = S.lap[kr][tid]; kr++; }
            if (R0OUT) {
                T r = rl;
                if (fix) r = (wv - ldg(P.in + fo + i)) * ib1;
                if (r != (T)0) nrmask |= 1u << bit;
                if (!OCC || r != (T)0 || ((mr_old >> bit) & 1u)) (P.r0out + fo)[i32] = r;
            }
            if (HZ) {
                // z <- z + bz F (zin may alias zout; a crowded cell leaves z
                // to the wide path, which reads it again)
                const T zi = ((mzi >> bit) & 1u) ? P.zin[fo + i] : (T)0;
                const T zv = zi + bzc * rl;
                if (zv != (T)0) nzmask |= 1u << bit;
                if (!over && (!OCC || zv != (T)0 || ((mz_old >> bit) & 1u))) (P.zout + fo)[i32] = zv;
                if (EMB) {
                    T e = wv - zv;
                    if (zv < (T)0 || zv > (T)1) e = (T)0;
                    if (e != (T)0) {
                        const T uv = ((muw >> bit) & 1u) ? ldg(P.uw + fo + i) : (T)0;
                        const T wt = rph * fmaxf(fabsf(uv), fabsf(wv)) + aph;
                        const T q = e / wt;
                        esum += (double)(q * q);
                        nce++;
                    }
                }
            }
            if (HO2) {
                // after stage 5: q2 <- q1 + m25 (u^n - q1), q1 <- q1 + m15 (q2 - q1)
                const T qi = ((mq2 >> bit) & 1u) ? ldg(P.q2in + fo + i) : (T)0;
                const T q2 = wv + m25 * (qi - wv);
                if (q2 != (T)0) n2mask |= 1u << bit;
                if (!OCC || q2 != (T)0 || ((m2_old >> bit) & 1u)) (P.out2 + fo)[i32] = q2;
                wv = wv + m15 * (q2 - wv);
            }
            if (wv != (T)0) nmask |= 1u << bit;
            if (!OCC || wv != (T)0 || ((mo_old >> bit) & 1u)) (P.out + fo)[i32] = wv;
        }
        if (OCC) {
            P.m_out[ow] = nmask;
            if (R0OUT) P.m_r0out[ow] = nrmask;
            if (HZ && !over) P.m_zout[ow] = nzmask;
            if (HO2) P.m_out2[ow] = n2mask;
        }
    }
    if (EMB) ecnt += (nce > 0 ? nce : 2);
    if (KC) {
        const long long o = (long long)N * Vs + i;
        // the small increments are summed first: c is rounded once per stage
        T d = b1c * rc;
        if (HR0) d = d + b0c * ldg(P.r0in + o);
        if (HP0) d = d + a0c * (ldg(P.p0 + o) - cc);
        if (HP2) d = d + a2c * (ldg(P.p2 + o) - cc);
        const T acc = cc + d;
        if (!isfinite(acc) && !over) raise_flag(P.flag, FLAG_NONFINITE);
        if (R0OUT) P.r0out[o] = rc;
        T cv = acc;
        if (HZ) {
            const T zv = P.zin[o] + bzc * rc;
            if (!over) P.zout[o] = zv;
            if (EMB) {
                const T e = acc - zv;
                const T au = fabsf(ldg(P.uw + o) + (T)g.cref), av = fabsf(acc + (T)g.cref);
                const T wt = (T)P.r_c * fmaxf(au, av) + (T)P.a_c;
                const T q = e / wt;
                esum += (double)(q * q);
                ecnt += 1;
            }
        }
        if (HO2) {
            const T q2 = acc + m25 * (ldg(P.q2in + o) - acc);
            P.out2[o] = q2;
            cv = acc + m15 * (q2 - acc);
        }
        P.out[o] = cv;
    }
}

// FP32 path for N > 32 phases: phases are taken in register-unrolled chunks
// of 32.  A trivial phase's stage value is final in the first sweep and is
// written, unnormalised, to the output; listed phases get their RHS term
// after the pairwise sums; a second sweep re-reads the output (written by the
// same thread moments before, so it is still in L2) and applies the
// projection's normalisation.  No per-phase register array is needed.
template <int DIM, int KC, unsigned SIG>
__device__ __forceinline__ bool big_cell(const Geom &g, const Pass<float> &P, PlainLoader<DIM> &ld,
                                         ListSmem<float> &S, int tid, long long i, const int *off, const int *ghost,
                                         const float *tabA, const float *tabB, const float *tabL,
                                         const signed char *ptype, double &esum, long long &ecnt)
{
    typedef float T;
    constexpr int NFACE = 2 * DIM;
    constexpr int CHK = 32;
    constexpr bool ERR = (SIG & SIG_ERR) != 0;
    constexpr bool HP0 = (SIG & SIG_P0) != 0 || ERR;
    constexpr bool HP2 = (SIG & SIG_P2) != 0;
    constexpr bool HR0 = (SIG & SIG_R0IN) != 0 || ERR;
    constexpr bool R0OUT = (SIG & SIG_R0OUT) != 0;
    constexpr bool PROJ = (SIG & SIG_PROJECT) != 0;
    const int N = g.N;
    const long long Vs = g.Vs;
    const int i32 = (int)i;
    const T idx2 = (T)(1.0 / g.dx2);
    const T a0c = (T)P.a0, a2c = (T)P.a2, b1c = (T)P.b1, b0c = (T)P.b0;
    const T ib1 = (T)(1.0 / P.b1);   // first-stage fix: F <- (S(u1) - u^n) / (mu~_1 dt)
    const T dt = (T)P.dt, rph = (T)P.r_phi, aph = (T)P.a_phi;
    auto combo = [&](T p0v, T v0, T p2v, T r0v) {
        T acc = affine<HP0, HP2>(v0, p0v, p2v, a0c, a2c);
        if (HR0) acc = acc + b0c * r0v;
        return acc;
    };

    T cc = (T)0, num_c = (T)0, den_c = (T)0, num_n[NFACE], den_n[NFACE], mf[NFACE];
#pragma unroll
    for (int f = 0; f < NFACE; ++f) { num_n[f] = (T)0; den_n[f] = (T)0; mf[f] = (T)0; }
    if (KC) {
        const T *cf = P.in + (long long)N * Vs + i;
        cc = ldg(cf);
        num_c = cc;
#pragma unroll
        for (int f = 0; f < NFACE; ++f) {
            T v = ldg(cf + off[f]);
            if (ghost[f] && g.bc_c[f] == BC_DIRICHLET) v = (T)2 * (T)g.cdir[f] - cc;
            num_n[f] = v;
        }
    }

    int nz = 0, nc = 0;
    bool changed = false;
    T best = (T)-1, ssum = (T)0;
    int bestid = -1;
    for (int a0 = 0; a0 < N; a0 += CHK) {
#pragma unroll
        for (int aa = 0; aa < CHK; ++aa) {
            const int a = a0 + aa;
            if (a < N) {
                const long long fo = (long long)a * Vs;
                T v0, nb[NFACE], p0v = (T)0, p2v = (T)0, r0v = (T)0;
                ld.load(a, fo, v0, nb, p0v, p2v, r0v, HP0, HP2, HR0);
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
                if (act) {
                    T l = (T)0;
#pragma unroll
                    for (int f = 0; f < NFACE; ++f) l = l + (nb[f] - v0);
                    if (nz < MAXACT) {
                        S.id[nz][tid] = (unsigned char)a;
                        S.lap[nz][tid] = l * idx2;
                        S.cen[nz][tid] = v0;
                        if (!ERR) S.val[nz][tid] = combo(p0v, v0, p2v, r0v);
                    }
                    nz++;
                } else if (ERR) {
                    T e = ((T)12 * (p0v - v0) + ((T)6 * dt) * r0v) * ((T)1 / (T)15);
                    const T trial = p0v + (dt * (T)0.5) * r0v;
                    if (trial < (T)0 || trial > (T)1) e = (T)0;
                    if (e != (T)0) {
                        const T w = rph * fmaxf(fabsf(p0v), fabsf(v0)) + aph;
                        const T q = e / w;
                        esum += (double)(q * q);
                        nc++;
                    }
                } else {
                    T c = combo(p0v, v0, p2v, r0v);
                    if (PROJ) {
                        if (c < (T)0) { c = (T)0; changed = true; }
                        if (c >= (T)1 && c > best) { best = c; bestid = a; }
                        ssum = ssum + c;
                    }
                    (P.out + fo)[i32] = c;
                }
            }
        }
    }
    if (nz > MAXACT) return false;      // crowded cell: the caller takes the wide path
    T mu = (T)0, rc = (T)0;
    if (KC) {
        mu = num_c / den_c;
        T acc = (T)0;
#pragma unroll
        for (int f = 0; f < NFACE; ++f) acc = acc + mf[f] * (num_n[f] / den_n[f] - mu);
        rc = acc * idx2;
    }
    for (int k = 0; k < nz; ++k) {
        const int a = S.id[k][tid];
        const T *Aa = tabA + a * N, *Ba = tabB + a * N;
        T d = (T)0;
        for (int k2 = 0; k2 < nz; ++k2) {
            if (k2 == k) continue;
            const int b = S.id[k2][tid];
            d = d + (ldg(Aa + b) * S.lap[k2][tid] + ldg(Ba + b) * S.cen[k2][tid]);
        }
        if (KC) {
            const int t = ptype[a];
            d = d + (-(mu * mu) / ((T)2 * (T)g.k[t]) - mu * (T)g.c0[t]);
        }
        S.dl[k][tid] = d;
    }
    const T inz = nz > 1 ? (T)1 / (T)nz : (T)0;
    for (int k = 0; k < nz; ++k) {
        T rk = (T)0;
        const int a = S.id[k][tid];
        if (nz > 1) {
            const T *La = tabL + a * N;
            const T dk = S.dl[k][tid];
            T s = (T)0;
            for (int k2 = 0; k2 < nz; ++k2) {
                if (k2 == k) continue;
                s = s + ldg(La + S.id[k2][tid]) * (dk - S.dl[k2][tid]);
            }
            rk = -(s * inz);
        }
        S.lap[k][tid] = rk;
        const long long fo = (long long)a * Vs;
        if (ERR) {
            const T p0v = ldg(P.p0 + fo + i), v0 = S.cen[k][tid], r0v = ldg(P.r0in + fo + i);
            const T sr = r0v + rk;
            T e = ((T)12 * (p0v - v0) + ((T)6 * dt) * sr) * ((T)1 / (T)15);
            const T trial = p0v + (dt * (T)0.5) * sr;
            if (trial < (T)0 || trial > (T)1) e = (T)0;
            if (e != (T)0) {
                const T w = rph * fmaxf(fabsf(p0v), fabsf(v0)) + aph;
                const T q = e / w;
                esum += (double)(q * q);
                nc++;
            }
        } else {
            T c = S.val[k][tid] + b1c * rk;
            if (PROJ) {
                if (c < (T)0) { c = (T)0; changed = true; }
                if (c >= (T)1 && (c > best || (c == best && a < bestid))) { best = c; bestid = a; }
                ssum = ssum + c;
            }
            (P.out + fo)[i32] = c;
        }
    }
    if (ERR) {
        ecnt += (nc > 0 ? nc : 2);
        if (KC) {
            const long long o = (long long)N * Vs + i;
            const T un = ldg(P.p0 + o), un1 = cc, rn = ldg(P.r0in + o);
            const T e = ((T)12 * (un - un1) + ((T)6 * dt) * (rn + rc)) * ((T)1 / (T)15);
            const T w = (T)P.r_c * fmaxf(fabsf(un + (T)g.cref), fabsf(un1 + (T)g.cref)) + (T)P.a_c;
            const T q = e / w;
            esum += (double)(q * q);
            ecnt += 1;
        }
        return true;
    }
    if (PROJ) {
        if (bestid >= 0) { changed = true; ssum = (T)1; }
        if (!(ssum > (T)0)) raise_flag(P.flag, FLAG_SIMPLEX);
    }
    const T inv = (ssum > (T)0) ? (T)1 / ssum : (T)1;
    const bool fix = R0OUT && P.fix_first && changed;
    int kr = 0;
    int curid = nz > 0 ? S.id[0][tid] : -1;
#pragma unroll 4
    for (int a = 0; a < N; ++a) {
        const long long fo = (long long)a * Vs;
        T w = (P.out + fo)[i32];
        if (PROJ) w = (bestid >= 0) ? ((a == bestid) ? (T)1 : (T)0) : w * inv;
        if (R0OUT) {
            T r = (T)0;
            if (a == curid) { r = S.lap[kr][tid]; kr++; curid = kr < nz ? S.id[kr][tid] : -1; }
            if (fix) r = (w - ldg(P.in + fo + i)) * ib1;
            (P.r0out + fo)[i32] = r;
        }
        (P.out + fo)[i32] = w;
    }
    if (KC) {
        const long long o = (long long)N * Vs + i;
        // the small increments are summed first: c is rounded once per stage
        T d = b1c * rc;
        if (HR0) d = d + b0c * ldg(P.r0in + o);
        if (HP0) d = d + a0c * (ldg(P.p0 + o) - cc);
        if (HP2) d = d + a2c * (ldg(P.p2 + o) - cc);
        const T acc = cc + d;
        if (!isfinite(acc)) raise_flag(P.flag, FLAG_NONFINITE);
        if (R0OUT) P.r0out[o] = rc;
        P.out[o] = acc;
    }
    return true;
}

template <int DIM, int KC, unsigned SIG>
__global__ void __launch_bounds__(BLOCK, 4)
big_kernel(const __grid_constant__ Geom g, const __grid_constant__ Pass<float> P, const float *__restrict__ tabA,
           const float *__restrict__ tabB, const float *__restrict__ tabL, const signed char *__restrict__ ptype)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    if (pass_skipped(P.flag)) return;
    ListSmem<float> &S = *reinterpret_cast<ListSmem<float> *>(smem_raw);
    const int tid = threadIdx.x;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int x = blockIdx.x * TX + (tid % TX);
    const int y = blockIdx.y * TY + (tid / TX);
    const int z = blockIdx.z;
    double esum = 0.0;
    long long ecnt = 0;
    if (x < g.nx && y < g.ny) {
        const long long i = ((long long)z * g.ny + y) * g.nx + x;
        long long off64[6];
        int ghost[6];
        face_offsets(g, x, y, z, off64, ghost);
        PlainLoader<DIM> ld;
        int off[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            off[f] = ghost[f] ? 0 : (int)off64[f];
            ld.inb[f] = (int)i + off[f];
        }
        ld.ic = (int)i;
        ld.Vs = (int)g.Vs;
        ld.nph = g.N;
        ld.in = P.in;
        ld.p0 = P.p0;
        ld.p2 = P.p2;
        ld.r0 = P.r0in;
        if (!big_cell<DIM, KC, SIG>(g, P, ld, S, tid, i, off, ghost, tabA, tabB, tabL, ptype, esum, ecnt)) {
            esum = 0.0;
            ecnt = 0;
            wide_cell<float, DIM, KC>(&g, &P, tabA, tabB, tabL, ptype, x, y, z, &esum, &ecnt);
        }
    }
    if (SIG & SIG_ERR) block_partials(esum, ecnt, P.part_sum, P.part_cnt, bid, P.part_n);
    if (P.count_step) count_step_done(P.flag);
}

// FP32 fast path with plain global loads (any grid, 2D or 3D).
template <int DIM, int KC, unsigned SIG, int NMAX, bool MASK>
__device__ __forceinline__ void fast_body(const Geom &g, const Pass<float> &P, const float *__restrict__ tabA,
                                          const float *__restrict__ tabB, const float *__restrict__ tabL,
                                          const signed char *__restrict__ ptype)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    if (pass_skipped(P.flag)) return;
    ListSmem<float> &S = *reinterpret_cast<ListSmem<float> *>(smem_raw);
    const int tid = threadIdx.x;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int x = blockIdx.x * TX + (tid % TX);
    const int y = blockIdx.y * TY + (tid / TX);
    const int z = blockIdx.z;
    double esum = 0.0;
    long long ecnt = 0;
    const bool here = x < g.nx && y < g.ny;
    const unsigned am = MASK ? __ballot_sync(0xffffffffu, here) : 0xffffffffu;
    if (here) {
        const long long i = ((long long)z * g.ny + y) * g.nx + x;
        long long off64[6];
        int ghost[6];
        face_offsets(g, x, y, z, off64, ghost);
        PlainLoader<DIM> ld;
        int off[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            off[f] = ghost[f] ? 0 : (int)off64[f];
            ld.inb[f] = (int)i + off[f];
        }
        ld.ic = (int)i;
        ld.Vs = (int)g.Vs;
        ld.nph = g.N;
        ld.in = P.in;
        ld.p0 = P.p0;
        ld.p2 = P.p2;
        ld.r0 = P.r0in;
        bool over = false;
        if constexpr (MASK)
            masked_cell<DIM, KC, SIG, true, (NMAX + 31) / 32>(g, P, S, tid, i, off, ghost, tabA, tabB, tabL, ptype,
                                                              esum, ecnt, am, over);
        else if constexpr (PF_DENSE_ROLLED || (SIG & (SIG_ERR | SIG_Z | SIG_O2 | SIG_EMB)) != 0)
            masked_cell<DIM, KC, SIG, false, (NMAX + 31) / 32>(g, P, S, tid, i, off, ghost, tabA, tabB, tabL, ptype,
                                                               esum, ecnt, am, over);
        else
            over = !fast_cell<DIM, KC, SIG, NMAX>(g, P, ld, S, tid, i, off, ghost, tabA, tabB, tabL, ptype, esum,
                                                  ecnt);
        if (over) {
            esum = 0.0;
            ecnt = 0;
            wide_cell<float, DIM, KC>(&g, &P, tabA, tabB, tabL, ptype, x, y, z, &esum, &ecnt);
        }
    }
    if (SIG & (SIG_ERR | SIG_EMB)) block_partials(esum, ecnt, P.part_sum, P.part_cnt, bid, P.part_n);
    if (P.count_step) count_step_done(P.flag);
}

template <int DIM, int KC, unsigned SIG, int NMAX, bool MASK = false>
__global__ void __launch_bounds__(BLOCK, MASK ? PF_MASK_MINB : PF_FAST_MINB)
fast_kernel(const __grid_constant__ Geom g, const __grid_constant__ Pass<float> P, const float *__restrict__ tabA,
            const float *__restrict__ tabB, const float *__restrict__ tabL, const signed char *__restrict__ ptype)
{
    fast_body<DIM, KC, SIG, NMAX, MASK>(g, P, tabA, tabB, tabL, ptype);
}

// The same pass with its description read from device memory (device-driven
// adaptive steps; see cell_kernel_d).
template <int DIM, int KC, unsigned SIG, int NMAX>
__global__ void __launch_bounds__(BLOCK, PF_FAST_MINB)
fast_kernel_d(const __grid_constant__ Geom g, const Pass<float> *__restrict__ Pd, const float *__restrict__ tabA,
              const float *__restrict__ tabB, const float *__restrict__ tabL, const signed char *__restrict__ ptype)
{
    __shared__ Pass<float> Ps;
    if (threadIdx.x == 0) Ps = *Pd;
    __syncthreads();
    fast_body<DIM, KC, SIG, NMAX, false>(g, Ps, tabA, tabB, tabL, ptype);
}

// FP32 fast path with TMA staging, warp-specialised: warps 0..7 compute the
// 32 x 8 tile, warp 8 is the producer that streams phase planes into the
// ring (waiting on each slot's "empty" barrier, one arrival per consumer
// warp) and the consumers wait on the slot's "full" barrier.  3D only, tiles
// fully inside the domain in x and y (nx % 32 == 0, ny % 8 == 0).
constexpr int TMA_BLOCK = BLOCK + 32;

template <int KC, unsigned SIG>
__global__ void __launch_bounds__(TMA_BLOCK, 3)
tma_kernel(const __grid_constant__ Geom g, const __grid_constant__ Pass<float> P, const __grid_constant__ TmaMaps M,
           const float *__restrict__ tabA, const float *__restrict__ tabB, const float *__restrict__ tabL,
           const signed char *__restrict__ ptype)
{
    constexpr bool ERR = (SIG & SIG_ERR) != 0;
    constexpr bool HP0 = (SIG & SIG_P0) != 0 || ERR;
    constexpr bool HP2 = (SIG & SIG_P2) != 0;
    constexpr bool HR0 = (SIG & SIG_R0IN) != 0 || ERR;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // [pad to 1024 B | TmaSmem | ListSmem]: TMA destinations must be 128-byte
    // aligned; the launch reserves 1 KB for the pad
    unsigned char *sbase = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    TmaSmem &Q = *reinterpret_cast<TmaSmem *>(sbase);
    ListSmem<float> &S = *reinterpret_cast<ListSmem<float> *>(sbase + sizeof(TmaSmem));
    if (pass_skipped(P.flag)) return;
    const int tid = threadIdx.x;
    const int N = g.N;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z = blockIdx.z;
    const bool zin = z > 0 && z < g.nz - 1;
    if (tid == 0) {
#pragma unroll
        for (int r = 0; r < TMA_R; ++r) {
            mbar_init(&Q.full[r], 1);
            mbar_init(&Q.empty[r], BLOCK / 32);
        }
        mbar_fence_init();
    }
    __syncthreads();
    double esum = 0.0;
    long long ecnt = 0;
    int timeout = 0;
    if (tid >= BLOCK) {
        // ---- producer warp: one elected lane issues every copy -------------
        if (tid == BLOCK) {
            const unsigned pt = (unsigned)(TX * TY * sizeof(float));
            const unsigned bytes = (zin ? 3u : 1u) * pt + (HP0 ? pt : 0u) + (HP2 ? pt : 0u) + (HR0 ? pt : 0u);
            int issued = 0;
            for (int a = 0; a < N; ++a) {
                const int r = a % TMA_R;
                // a slot that its consumers never released: stop issuing (no
                // copy may land in a slot that is still being read)
                if (a >= TMA_R && !mbar_wait(&Q.empty[r], (unsigned)(((a / TMA_R) - 1) & 1))) {
                    timeout = 1;
                    break;
                }
                fence_proxy_async();
                mbar_expect_tx(&Q.full[r], bytes);
                if (zin) tma_load4(&Q.in[r][0][0][0], &M.in3, x0, y0, z - 1, a, &Q.full[r]);
                else tma_load4(&Q.in[r][1][0][0], &M.in1, x0, y0, z, a, &Q.full[r]);
                if (HP0) tma_load4(&Q.p0[r][0][0], &M.p0, x0, y0, z, a, &Q.full[r]);
                if (HP2) tma_load4(&Q.p2[r][0][0], &M.p2, x0, y0, z, a, &Q.full[r]);
                if (HR0) tma_load4(&Q.r0[r][0][0], &M.r0, x0, y0, z, a, &Q.full[r]);
                issued = a + 1;
            }
            // the block's shared memory must outlive every copy issued into
            // it: wait (bounded) until the last copy of each slot has landed
            for (int a = issued - TMA_R > 0 ? issued - TMA_R : 0; a < issued; ++a)
                if (!mbar_wait(&Q.full[a % TMA_R], (unsigned)((a / TMA_R) & 1))) timeout = 1;
        }
    } else {
        // ---- consumer warps: one cell per thread ---------------------------
        const int tx = tid % TX, ty = tid / TX;
        const int x = x0 + tx, y = y0 + ty;
        const long long i = ((long long)z * g.ny + y) * g.nx + x;
        long long off64[6];
        int ghost[6];
        face_offsets(g, x, y, z, off64, ghost);
        TmaLoader ld;
#pragma unroll
        for (int f = 0; f < 6; ++f) ld.off[f] = ghost[f] ? 0 : (int)off64[f];
        ld.Q = &Q;
        ld.pin = P.in + i;
        ld.tx = tx;
        ld.ty = ty;
        ld.zin = zin;
        ld.ok = true;
        if (!fast_cell<3, KC, SIG, 32>(g, P, ld, S, tid, i, ld.off, ghost, tabA, tabB, tabL, ptype, esum, ecnt)) {
            esum = 0.0;
            ecnt = 0;
            wide_cell<float, 3, KC>(&g, &P, tabA, tabB, tabL, ptype, x, y, z, &esum, &ecnt);
        }
        if (!ld.ok) timeout = 1;
    }
    if (timeout) raise_flag(P.flag, FLAG_TIMEOUT);
    if (ERR) block_partials(esum, ecnt, P.part_sum, P.part_cnt, bid, P.part_n);
    if (P.count_step) count_step_done(P.flag);
}

// Signature of a pass as used by the engine's dispatcher.
template <typename T>
inline unsigned pass_signature(const Pass<T> &P)
{
    if (P.mode == MODE_ERR) return P.r0out ? (SIG_ERR | SIG_R0OUT) : SIG_ERR;
    if (P.mode == MODE_RHS) return SIG_RHS;
    unsigned s = 0;
    if (P.p0) s |= SIG_P0;
    if (P.p2) s |= SIG_P2;
    if (P.r0in) s |= SIG_R0IN;
    if (P.r0out) s |= SIG_R0OUT;
    if (P.project) s |= SIG_PROJECT;
    if (P.zout) s |= SIG_Z;
    if (P.out2) s |= SIG_O2;
    if (P.embedded_err) {
        if (!P.zout) return SIG_GENERIC;
        s |= SIG_EMB;
    }
    return s;
}

}  // namespace pfk
