// pf_engine.cu -- host engine and C ABI of libpf (see include/pf.h).
//
// The engine owns five device state vectors per handle (cell-record layout,
// see pf_kernels.cuh) and drives the fused stage pass for every integrator of
// Sec. 3.2 of Seiz & Takaki (arXiv 2601.16522), the error estimate and norm of
// Sec. 3.3 (deterministic two-level FP64 reduction) and the PID controller
// with bias.  Only scalars cross the host/device boundary per adaptive step.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/pf.h"
#include "pf_internal.h"

using pfk::Geom;
using pfk::Pass;

namespace {

const double kPi = 3.14159265358979323846;
constexpr int NBUF = 5;
constexpr size_t PF_FLAG_BYTES = 4 * sizeof(int);   // device status words (pfk::raise_flag)

// ---------------------------------------------------------------------------
// auxiliary kernels: layout conversion and reductions
// ---------------------------------------------------------------------------

// ABI layout (FP64: N phase fields at phi, field stride V; the concentration
// at c) -> engine layout (T, field stride Vs).  phi and c may be device
// memory or page-locked host memory reached through its device mapping.
template <typename T>
__global__ void pack_kernel(const double *__restrict__ phi, const double *__restrict__ c, T *__restrict__ dst,
                            long long V, long long Vs, int N, int NF, double cref)
{
    const long long n = V * NF;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const long long f = k / V;
        const long long i = k - f * V;
        dst[f * Vs + i] = (T)(f < N ? phi[k] : c[i] - cref);
    }
}

// engine layout -> ABI layout (phi and c as for pack_kernel; c may be null)
template <typename T>
__global__ void unpack_kernel(const T *__restrict__ src, double *__restrict__ phi, double *__restrict__ c, long long V,
                              long long Vs, int N, int NF, double cref)
{
    const long long n = V * NF;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const long long f = k / V;
        const long long i = k - f * V;
        const double v = (double)src[f * Vs + i];
        if (f < N) phi[k] = v;
        else if (c) c[i] = v + cref;
    }
}

// Slot storage (pf_slots.cuh layout).  Dense ABI layout -> slots: a cell's
// nonzero values (after rounding to FP32) in ascending phase order; a cell
// with more than NSLOT raises FLAG_NZ_OVERFLOW (the state cannot be held).
__global__ void slot_pack_dense(const double *__restrict__ phi, const double *__restrict__ c, float *__restrict__ dst,
                                long long V, int Vs, int N, int K, double cref, int *flag)
{
    unsigned short *ids = reinterpret_cast<unsigned short *>(dst + (long long)pfk::NSLOT * Vs);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
        int cnt = 0;
        for (int a = 0; a < N; ++a) {
            const float v = (float)phi[(long long)a * V + i];
            if (v == 0.0f) continue;
            if (cnt < pfk::NSLOT) {
                dst[(long long)cnt * Vs + i] = v;
                ids[(long long)cnt * Vs + i] = (unsigned short)a;
            }
            cnt++;
        }
        if (cnt > pfk::NSLOT) atomicOr(flag, pfk::FLAG_NZ_OVERFLOW);
        for (int k = cnt; k < pfk::NSLOT; ++k) {
            dst[(long long)k * Vs + i] = 0.0f;
            ids[(long long)k * Vs + i] = (unsigned short)pfk::SLOT_EMPTY;
        }
        if (K) dst[(long long)pfk::SLOT_C_PLANES * Vs + i] = (float)(c[i] - cref);
    }
}

// Slot form of the ABI (n_in planes of values and of int ids, id < 0 empty)
// -> slots: the entries with a nonzero FP32 value, sorted by id.  More than
// NSLOT of them, an id outside 0..N-1 or a repeated id raises
// FLAG_NZ_OVERFLOW.
__global__ void slot_pack_slots(const double *__restrict__ vals, const int *__restrict__ idin, int n_in,
                                const double *__restrict__ c, float *__restrict__ dst, long long V, int Vs, int N,
                                int K, double cref, int *flag)
{
    unsigned short *ids = reinterpret_cast<unsigned short *>(dst + (long long)pfk::NSLOT * Vs);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
        float sv[pfk::NSLOT];
        int sid[pfk::NSLOT];
        int cnt = 0;
        bool bad = false;
        for (int k = 0; k < n_in; ++k) {
            const int a = idin[(long long)k * V + i];
            if (a < 0) continue;
            const float v = (float)vals[(long long)k * V + i];
            if (v == 0.0f) continue;
            if (a >= N || cnt >= pfk::NSLOT) { bad = true; break; }
            // insertion in ascending id order
            int j = cnt;
            while (j > 0 && sid[j - 1] > a) { sid[j] = sid[j - 1]; sv[j] = sv[j - 1]; --j; }
            if (j > 0 && sid[j - 1] == a) { bad = true; break; }
            sid[j] = a;
            sv[j] = v;
            cnt++;
        }
        if (bad) { atomicOr(flag, pfk::FLAG_NZ_OVERFLOW); cnt = 0; }
        for (int k = 0; k < pfk::NSLOT; ++k) {
            dst[(long long)k * Vs + i] = k < cnt ? sv[k] : 0.0f;
            ids[(long long)k * Vs + i] = (unsigned short)(k < cnt ? sid[k] : (int)pfk::SLOT_EMPTY);
        }
        if (K) dst[(long long)pfk::SLOT_C_PLANES * Vs + i] = (float)(c[i] - cref);
    }
}

// Slots -> dense ABI layout (c may be null).
__global__ void slot_unpack_dense(const float *__restrict__ src, double *__restrict__ phi, double *__restrict__ c,
                                  long long V, int Vs, int N, int K, double cref)
{
    const unsigned short *ids = reinterpret_cast<const unsigned short *>(src + (long long)pfk::NSLOT * Vs);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
        for (int a = 0; a < N; ++a) phi[(long long)a * V + i] = 0.0;
        for (int k = 0; k < pfk::NSLOT; ++k) {
            const unsigned a = ids[(long long)k * Vs + i];
            if (a >= (unsigned)N) break;
            phi[(long long)a * V + i] = (double)src[(long long)k * Vs + i];
        }
        if (K && c) c[i] = (double)src[(long long)pfk::SLOT_C_PLANES * Vs + i] + cref;
    }
}

// Slots -> slot form of the ABI (NSLOT planes of values and ids, -1 empty).
__global__ void slot_unpack_slots(const float *__restrict__ src, double *__restrict__ vals, int *__restrict__ idout,
                                  double *__restrict__ c, long long V, int Vs, int N, int K, double cref)
{
    const unsigned short *ids = reinterpret_cast<const unsigned short *>(src + (long long)pfk::NSLOT * Vs);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
        for (int k = 0; k < pfk::NSLOT; ++k) {
            const unsigned a = ids[(long long)k * Vs + i];
            const bool used = a < (unsigned)N;
            vals[(long long)k * V + i] = used ? (double)src[(long long)k * Vs + i] : 0.0;
            idout[(long long)k * V + i] = used ? (int)a : -1;
        }
        if (K && c) c[i] = (double)src[(long long)pfk::SLOT_C_PLANES * Vs + i] + cref;
    }
}

// Per-phase totals of a slot state: sum (FP64 atomics, so the last bits
// depend on the order the blocks run in) and maximum (on the encodings of
// the nonnegative values, exact) of every phase.
__global__ void slot_phase_totals(const float *__restrict__ src, long long V, int Vs, int N, double *vol,
                                  unsigned long long *mx)
{
    const unsigned short *ids = reinterpret_cast<const unsigned short *>(src + (long long)pfk::NSLOT * Vs);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x)
        for (int k = 0; k < pfk::NSLOT; ++k) {
            const unsigned a = ids[(long long)k * Vs + i];
            if (a >= (unsigned)N) break;
            const double v = (double)src[(long long)k * Vs + i];
            atomicAdd(vol + a, v);
            if (v > 0.0) atomicMax(mx + a, (unsigned long long)__double_as_longlong(v));
        }
}

// Self-test of the bounded device waits: one thread waits on a shared-memory
// mbarrier that no thread arrives on, with the poll loop of the TMA kernels
// and a caller-given limit; it must give up, raise FLAG_TIMEOUT and return.
__global__ void wait_selftest_kernel(int *flag, unsigned polls)
{
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        pfk::mbar_init(&bar, 1);
        pfk::mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!pfk::mbar_wait(&bar, 0u, polls)) atomicOr(flag, pfk::FLAG_TIMEOUT);
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(pfk::smem_u32(&bar)) : "memory");
    }
}

// Fixed-order sum of the per-block error partials (one block of 256 threads).
// n: the number of partials, or (pn non-null) at most n, the count the error
// pass recorded (its block count depends on the kernel that ran).
__global__ void finalize_err_kernel(const double *__restrict__ ps, const long long *__restrict__ pc, int n,
                                    double *out_sum, long long *out_cnt, const int *pn = nullptr)
{
    if (pn && *pn < n) n = *pn;
    __shared__ double ss[256];
    __shared__ long long sc[256];
    double s = 0.0;
    long long c = 0;
    for (int k = threadIdx.x; k < n; k += 256) { s += ps[k]; c += pc[k]; }
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int o = 128; o >= 1; o >>= 1) {
        if ((int)threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            sc[threadIdx.x] += sc[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { *out_sum = ss[0]; *out_cnt = sc[0]; }
}

// Occupancy words of an FP32 state (masked storage): bit b of word w of cell
// i (plane w) is set where phase 32 w + b is nonzero.
__global__ void mask_kernel(const float *__restrict__ u, unsigned *__restrict__ m, long long V, long long Vs, int N)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
        for (int w = 0; 32 * w < N; ++w) {
            unsigned bits = 0u;
            for (int b = 0; b < 32 && 32 * w + b < N; ++b)
                if (u[(long long)(32 * w + b) * Vs + i] != 0.0f) bits |= 1u << b;
            m[(long long)w * Vs + i] = bits;
        }
    }
}

// Per-field totals: block (b, f) sums / maximises field f over a fixed cell range.
template <typename T>
__global__ void totals_kernel(const T *__restrict__ u, long long V, long long Vs, double *psum, double *pmax)
{
    const int f = blockIdx.y;
    const long long chunk = (V + gridDim.x - 1) / gridDim.x;
    const long long lo = blockIdx.x * chunk;
    const long long hi = lo + chunk < V ? lo + chunk : V;
    double s = 0.0, m = -1e300;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double v = (double)u[(long long)f * Vs + i];
        s += v;
        m = v > m ? v : m;
    }
    __shared__ double ss[256], sm[256];
    ss[threadIdx.x] = s;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = 128; o >= 1; o >>= 1) {
        if ((int)threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            sm[threadIdx.x] = sm[threadIdx.x] > sm[threadIdx.x + o] ? sm[threadIdx.x] : sm[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        psum[(long long)f * gridDim.x + blockIdx.x] = ss[0];
        pmax[(long long)f * gridDim.x + blockIdx.x] = sm[0];
    }
}


// Stage 1 from a stored RHS: recompute sweep (1) or store-and-reread (0).
#ifndef PF_FIRST_RECOMPUTE
#define PF_FIRST_RECOMPUTE 1
#endif

// RKL stage 1 from a stored RHS (reuse of F(u^{n+1}) of the previous error
// sweep as F(u^n)): u1 = S(u^n + b1 F) with the simplex projection of
// Sec. 3.1 in the stage kernels' order (clamp, largest value >= 1 with ties
// to the lowest id, division by the sum), and the RKL2 first-stage fix
// F <- (S(u1) - u^n) / b1 in every phase of a cell where S acted (fix != 0).
// The stored RHS is updated in place (each thread reads and writes only its
// own cell).  Pass 1 writes the unprojected values to out; pass 2 rereads
// them (the same thread wrote them).
template <typename T>
__global__ void first_from_rhs_kernel(const T *__restrict__ in, T *out, T *r0, long long V, long long Vs, int N, int K,
                                      double b1, int fix, int *flag)
{
    if (pfk::pass_skipped(flag)) return;
    const T one = (T)1, b1c = (T)b1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
        bool changed = false;
        T best = (T)-1, ssum = (T)0;
        int bestid = -1, nnz = 0;
        for (int a = 0; a < N; ++a) {
            const long long o = (long long)a * Vs + i;
            T acc = one * in[o];
            acc = acc + b1c * r0[o];
            if (acc < (T)0) { acc = (T)0; changed = true; }
            if (acc >= (T)1 && acc > best) { best = acc; bestid = a; }
            if (acc != (T)0) nnz++;
            ssum = ssum + acc;
            out[o] = acc;
        }
        if (bestid >= 0) {
            if (!(best == (T)1 && nnz == 1)) changed = true;
            ssum = (T)1;
        }
        if (!(ssum > (T)0)) pfk::raise_flag(flag, pfk::FLAG_SIMPLEX);
        const bool fx = fix && changed;
        for (int a = 0; a < N; ++a) {
            const long long o = (long long)a * Vs + i;
            T w = out[o];
            if (bestid >= 0) w = (a == bestid) ? (T)1 : (T)0;
            else if (ssum > (T)0) w = w / ssum;
            out[o] = w;
            if (fx) r0[o] = (w - in[o]) / b1c;
        }
        if (K) {
            const long long o = (long long)N * Vs + i;
            T acc = one * in[o];
            acc = acc + b1c * r0[o];
            if (!isfinite(acc)) pfk::raise_flag(flag, pfk::FLAG_NONFINITE);
            out[o] = acc;
        }
    }
}

// The same stage without storing the unprojected values: a first sweep over
// the phases gathers the projection's sum and decisions, a second sweep
// recomputes each value from u^n and F and writes it (u^n and F are read
// twice, the output once).
template <typename T>
__global__ void __launch_bounds__(256)
first_from_rhs_recompute_kernel(const T *__restrict__ in, T *out, T *r0, long long V, long long Vs, int N, int K,
                                double b1, int fix, int *flag)
{
    if (pfk::pass_skipped(flag)) return;
    const T one = (T)1, b1c = (T)b1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
        bool changed = false;
        T best = (T)-1, ssum = (T)0;
        int bestid = -1, nnz = 0;
#pragma unroll 8
        for (int a = 0; a < N; ++a) {
            const long long o = (long long)a * Vs + i;
            T x = one * in[o];
            x = x + b1c * r0[o];
            if (x < (T)0) { x = (T)0; changed = true; }
            if (x >= (T)1 && x > best) { best = x; bestid = a; }
            if (x != (T)0) nnz++;
            ssum = ssum + x;
        }
        if (bestid >= 0) {
            if (!(best == (T)1 && nnz == 1)) changed = true;
            ssum = (T)1;
        }
        if (!(ssum > (T)0)) pfk::raise_flag(flag, pfk::FLAG_SIMPLEX);
        const bool fx = fix && changed;
#pragma unroll 8
        for (int a = 0; a < N; ++a) {
            const long long o = (long long)a * Vs + i;
            const T v = in[o];
            T x = one * v;
            x = x + b1c * r0[o];
            if (x < (T)0) x = (T)0;
            T w;
            if (bestid >= 0) w = (a == bestid) ? (T)1 : (T)0;
            else w = (ssum > (T)0) ? x / ssum : x;
            out[o] = w;
            if (fx) r0[o] = (w - v) / b1c;
        }
        if (K) {
            const long long o = (long long)N * Vs + i;
            T x = one * in[o];
            x = x + b1c * r0[o];
            if (!isfinite(x)) pfk::raise_flag(flag, pfk::FLAG_NONFINITE);
            out[o] = x;
        }
    }
}

// Energy functional of Eq. energy, one cell per thread, accumulated in FP64.
// The gradients are forward differences across the +x, +y, +z faces (a
// zero-gradient ghost across a non-periodic face).  Only phases that are
// nonzero at the cell or at one of those three neighbours contribute (every
// other term is an exact zero); they are listed in ascending order, up to
// EMAX of them, and a cell with more counts as an overflow.  Per cell:
//   e = sum_{a>b} (-A_ab grad phi_a . grad phi_b + B_ab phi_a phi_b)
//     + sum_a phi_a mu^2 / (2 k_a)                     (K = 1, KKS, Sec. 2)
constexpr int EMAX = 32;

// x != 0 taken without the FP64 pipe (GB300's FP64 rate is a small fraction
// of its FP32 rate): FP32 values are compared in FP32, FP64 values by their
// encoding with the sign bit dropped (the same answer for every value).
__device__ __forceinline__ bool nonzero_value(float x) { return x != 0.0f; }
__device__ __forceinline__ bool nonzero_value(double x) { return (__double_as_longlong(x) << 1) != 0; }

template <typename T>
__global__ void __launch_bounds__(256)
energy_kernel(const Geom g, const T *__restrict__ u, const double *__restrict__ A, const double *__restrict__ B,
              const signed char *__restrict__ ptype, double dx, double *ps, long long *pc)
{
    unsigned char id[EMAX];
    double ph[EMAX], gr[EMAX][3];
    double esum = 0.0;
    long long over = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.V; i += stride) {
        const int x = (int)(i % g.nx);
        const int y = (int)((i / g.nx) % g.ny);
        const int z = (int)(i / ((long long)g.nx * g.ny));
        long long off[6];
        int ghost[6];
        pfk::face_offsets(g, x, y, z, off, ghost);
        int n = 0;
        bool full = false;
        for (int a = 0; a < g.N; ++a) {
            const T *f = u + (long long)a * g.Vs + i;
            const T vt = f[0];
            T wt[3] = {vt, vt, vt};
            bool any = nonzero_value(vt);
            for (int ax = 0; ax < g.dim; ++ax) {
                if (!ghost[2 * ax + 1]) wt[ax] = f[off[2 * ax + 1]];
                any = any || nonzero_value(wt[ax]);
            }
            if (!any) continue;
            // equal values have a zero difference: no FP64 division for them
            const double v = (double)vt;
            double d[3] = {0.0, 0.0, 0.0};
            for (int ax = 0; ax < g.dim; ++ax)
                if (wt[ax] != vt) d[ax] = __dsub_rn((double)wt[ax], v) / dx;
            if (n == EMAX) { full = true; break; }
            id[n] = (unsigned char)a;
            ph[n] = v;
            gr[n][0] = d[0]; gr[n][1] = d[1]; gr[n][2] = d[2];
            ++n;
        }
        if (full) { ++over; continue; }
        double e = 0.0;
        for (int p = 0; p < n; ++p) {
            const long long ra = (long long)id[p] * g.N;
            for (int q = 0; q < p; ++q) {
                double gg = 0.0;
                for (int ax = 0; ax < g.dim; ++ax) gg = __dadd_rn(gg, __dmul_rn(gr[p][ax], gr[q][ax]));
                e = __dsub_rn(e, __dmul_rn(A[ra + id[q]], gg));
                e = __dadd_rn(e, __dmul_rn(__dmul_rn(B[ra + id[q]], ph[p]), ph[q]));
            }
        }
        if (g.K) {
            double num = (double)u[(long long)g.N * g.Vs + i], den = 0.0;
            for (int p = 0; p < n; ++p) {
                const int t = ptype[id[p]];
                num = __dsub_rn(num, __dmul_rn(ph[p], g.c0[t]));
                den = __dadd_rn(den, __dmul_rn(ph[p], g.invk[t]));
            }
            const double mu = num / den;
            for (int p = 0; p < n; ++p) {
                const int t = ptype[id[p]];
                e = __dadd_rn(e, __dmul_rn(ph[p], __dmul_rn(mu, mu) / __dmul_rn(2.0, g.k[t])));
            }
        }
        esum = __dadd_rn(esum, e);
    }
    pfk::block_partials(esum, over, ps, pc, blockIdx.x);
}
}  // namespace

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------

// Caller-supplied device allocator (pf_set_allocator).
struct AllocHook {
    pf_alloc_fn alloc = nullptr;
    pf_free_fn free = nullptr;
    void *ctx = nullptr;
};

struct pf_handle {
    int dev = 0;
    AllocHook hook;                    // allocator captured at pf_create (empty: stream-ordered CUDA)
    std::vector<std::pair<void *, size_t>> allocs;   // every device allocation and its size
    long long footprint = 0;           // pf_footprint of the parameters (batch admission)
    std::vector<Pass<float>> *collect = nullptr;   // batch mode: FP32 passes recorded, not launched
    bool in_batch = false;
    cudaStream_t stream = nullptr;
    int prec = 64;
    size_t esize = 8;
    Geom g{};
    int N = 0, K = 0, NP = 0;
    long long V = 0, Vs = 0;
    int grid = 1;                      // blocks per pass (= error partials)
    std::vector<int> ptype;
    std::vector<double> A, B, L;
    void *dA = nullptr, *dB = nullptr, *dL = nullptr;
    double *dAB64 = nullptr;           // A then B in FP64 (energy functional)
    signed char *dptype = nullptr;
    void *buf[NBUF] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int iu = 0;                        // buffer holding u^n
    size_t vec_bytes = 0;
    double *staging = nullptr;         // (N + K) * V doubles (set/get/rhs)
    unsigned char *dnz = nullptr;
    double *part_sum = nullptr;
    long long *part_cnt = nullptr;
    double *dres = nullptr;            // [0] error sum
    long long *dcnt = nullptr;
    int *dflag = nullptr;
    int *dpartn = nullptr;             // error partials written by the last error pass
    int *dcrowd = nullptr;             // crowded cells recorded by a two-cell pass (FP32)
    double *tot_sum = nullptr, *tot_max = nullptr;
    int tot_blocks = 0;
    bool slots = false;                // per-cell phase slots (pf_slots.cuh layout)
    bool masked = false;               // masked storage: occupancy-word planes after the fields
    int nw = 0;                        // occupancy words per cell (masked storage)
    bool tma_ok = false;               // tensor maps built: TMA-staged kernels available
    bool tma = false;                  // TMA-staged FP32 kernels in use
    CUtensorMap m3[NBUF], m1[NBUF];    // per buffer: 3-plane and 1-plane boxes
    double t = 0.0;
    bool has_state = false;
    double dte = 0.0;
    double dx = 1.0;
    // launch accounting and optional per-pass event timing
    long long launches = 0;
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_kind;          // kind of the pass bracketed by events 2k, 2k+1
    int ev_used = 0;
    double prof_ms[PF_NPASS_KINDS] = {0};
    long long prof_n[PF_NPASS_KINDS] = {0};
    int cur_kind = PF_PASS_OTHER;
    // CUDA graph of `period` full fixed steps (replayed while the step size,
    // stage count and buffer rotation are unchanged)
    cudaGraphExec_t gexec = nullptr;
    int g_integ = -1, g_s = -1, g_iu = -1, g_period = 0;
    std::vector<int> g_seq;            // buffer holding u^n after each step of the period
    double g_dt = 0.0;
    long long g_evals = 0, g_launches = 0;
    long long graph_replays = 0;
    // controller (Sec. 3.3)
    double b = 0.9, E1 = 0.0, E2 = 0.0, dt1 = 0.0, dt2 = 0.0;
    int nhist = 0;
    double dt_next = 0.0;
    // device-driven adaptive RKL steps: control block, pass descriptions, graph
    void *dl_ctl = nullptr, *dl_desc = nullptr;
    cudaGraph_t dl_graph = nullptr;
    cudaGraphExec_t dl_exec = nullptr;
    int dl_integ = -1;
    // reuse of F(u^{n+1}) as the next step's F(u^n) (PF_STEP_REUSE_RHS):
    // buffer rhs_buf holds the raw RHS of the state in buffer rhs_iu
    bool reuse_on = false, rhs_valid = false;
    int rhs_buf = -1, rhs_iu = -1;
    int rhs_pending = -1;              // buffer the last error sweep wrote F(u^{n+1}) into
};

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? PF_OK : PF_EDEVICE; }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no -lcuda).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 4D map (x, y, z, field) of one FP32 state buffer with a 32 x 8 x boxz x 1 box.
bool make_map(CUtensorMap *m, void *base, const pfk::Geom &g, int boxz)
{
    auto enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)g.NF};
    const cuuint64_t strides[3] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.nx * g.ny * 4, (cuuint64_t)g.Vs * 4};
    const cuuint32_t box[4] = {(cuuint32_t)pfk::TX, (cuuint32_t)pfk::TY, (cuuint32_t)boxz, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void *vec(pf_handle *h, int k) { return h->buf[k]; }

// Fold recorded event pairs into the per-kind totals (synchronises).
int prof_flush(pf_handle *h)
{
    if (h->ev_used == 0) return PF_OK;
    if (cudaEventSynchronize(h->ev_pool[2 * (h->ev_used - 1) + 1]) != cudaSuccess) return PF_EDEVICE;
    for (int k = 0; k < h->ev_used; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev_pool[2 * k], h->ev_pool[2 * k + 1]) != cudaSuccess) return PF_EDEVICE;
        h->prof_ms[h->ev_kind[k]] += ms;
        h->prof_n[h->ev_kind[k]] += 1;
    }
    h->ev_used = 0;
    return PF_OK;
}

int prof_begin(pf_handle *h)
{
    if (!h->prof_on) return PF_OK;
    if (h->ev_used * 2 + 2 > (int)h->ev_pool.size()) {
        int st = prof_flush(h);
        if (st) return st;
    }
    h->ev_kind[h->ev_used] = h->cur_kind;
    return cudaEventRecord(h->ev_pool[2 * h->ev_used], h->stream) == cudaSuccess ? PF_OK : PF_EDEVICE;
}

int prof_end(pf_handle *h)
{
    if (!h->prof_on) return PF_OK;
    if (cudaEventRecord(h->ev_pool[2 * h->ev_used + 1], h->stream) != cudaSuccess) return PF_EDEVICE;
    h->ev_used++;
    return PF_OK;
}

int buf_index(const pf_handle *h, const void *p)
{
    for (int k = 0; k < NBUF; ++k) if (h->buf[k] == p) return k;
    return -1;
}

// Occupancy-mask plane of a state vector (masked storage): Vs words after
// the NP fields.
unsigned *mask_plane(const pf_handle *h, const void *vecp)
{
    return vecp ? (unsigned *)((char *)const_cast<void *>(vecp) + (size_t)h->Vs * h->NP * h->esize) : nullptr;
}

// Pass signatures that have a masked instantiation.
bool masked_sig(unsigned s)
{
    using namespace pfk;
    return s == SIG_PROJECT || s == (SIG_P2 | SIG_PROJECT) || s == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT) ||
           s == (SIG_R0OUT | SIG_PROJECT) || s == SIG_ERR || s == (SIG_P0 | SIG_PROJECT) ||
           s == (SIG_O2 | SIG_PROJECT) || s == (SIG_Z | SIG_PROJECT) || s == (SIG_Z | SIG_O2 | SIG_PROJECT) ||
           s == (SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT);
}

// After a pass that wrote a state vector without maintaining its mask, mark
// every phase of it as possibly nonzero.
int invalidate_mask(pf_handle *h, const void *vecp)
{
    if (!vecp || buf_index(h, vecp) < 0) return PF_OK;
    return cudaMemsetAsync(mask_plane(h, vecp), 0xff, sizeof(unsigned) * (size_t)h->Vs * h->nw, h->stream) ==
                   cudaSuccess ? PF_OK : PF_EDEVICE;
}

template <typename T>
int run_pass(pf_handle *h, const Pass<T> &P)
{
    // the kernels evaluate the combination as v + a0 (p0 - v) + a2 (p2 - v)
    if (P.mode == pfk::MODE_STAGE &&
        fabs(P.a1 + (P.p0 ? P.a0 : 0.0) + (P.p2 ? P.a2 : 0.0) - 1.0) > 1e-12)
        return PF_EINVAL;
    if constexpr (sizeof(T) == 4) {
        // batch mode: the pass is recorded for a packed launch
        if (h->collect) {
            h->collect->push_back(P);
            return PF_OK;
        }
    }
    int st = prof_begin(h);
    if (st) return st;
    pfk::TmaMaps tm;
    const pfk::TmaMaps *tmp = nullptr;
    if (h->tma && P.mode != pfk::MODE_RHS) {
        const int ki = buf_index(h, P.in), k0 = P.p0 ? buf_index(h, P.p0) : 0, k2 = P.p2 ? buf_index(h, P.p2) : 0,
                  kr = P.r0in ? buf_index(h, P.r0in) : 0;
        if (ki >= 0 && k0 >= 0 && k2 >= 0 && kr >= 0) {
            tm.in3 = h->m3[ki];
            tm.in1 = h->m1[ki];
            tm.p0 = h->m1[k0];
            tm.p2 = h->m1[k2];
            tm.r0 = h->m1[kr];
            tmp = &tm;
        }
    }
    if (h->masked && P.mode != pfk::MODE_RHS && masked_sig(pfk::pass_signature(P))) {
        Pass<T> Q = P;
        Q.m_in = mask_plane(h, P.in);
        Q.m_p0 = mask_plane(h, P.p0);
        Q.m_p2 = mask_plane(h, P.p2);
        Q.m_r0 = mask_plane(h, P.r0in);
        Q.m_out = P.mode == pfk::MODE_ERR ? nullptr : mask_plane(h, P.out);
        Q.m_r0out = mask_plane(h, P.r0out);
        Q.m_zin = mask_plane(h, P.zin);
        Q.m_zout = mask_plane(h, P.zout);
        Q.m_out2 = mask_plane(h, P.out2);
        Q.m_q2in = mask_plane(h, P.q2in);
        Q.m_uw = mask_plane(h, P.uw);
        int e = pfk::launch_stage<T>(h->g, Q, h->stream, (const T *)h->dA, (const T *)h->dB, (const T *)h->dL,
                                     h->dptype, nullptr);
        h->launches++;
        if (e != 0) return PF_EDEVICE;
        return prof_end(h);
    }
    int nk = 1;
    int e = pfk::launch_stage<T>(h->g, P, h->stream, (const T *)h->dA, (const T *)h->dB, (const T *)h->dL,
                                 h->dptype, tmp, &nk);
    h->launches += nk;
    if (e != 0) return PF_EDEVICE;
    if (h->masked && P.mode != pfk::MODE_RHS) {
        // a dense pass (generic kernel) wrote these vectors: their masks are stale
        const void *outs[] = {P.out, P.r0out, P.zout, P.out2};
        for (const void *o : outs)
            if ((st = invalidate_mask(h, o))) return st;
    }
    return prof_end(h);
}

template <typename T>
Pass<T> blank_pass(pf_handle *h)
{
    Pass<T> P;
    memset(&P, 0, sizeof(P));
    P.mode = pfk::MODE_STAGE;
    P.project = 1;
    P.a1 = 1.0;
    P.flag = h->dflag;
    P.part_n = h->dpartn;
    P.crowd = h->dcrowd;
    P.part_sum = h->part_sum;
    P.part_cnt = h->part_cnt;
    return P;
}

// ---- Gershgorin reading of the stable Euler step (Sec. 3.2) ---------------
double gershgorin_dt_e(const pf_handle *h, const pf_params *p)
{
    const int N = h->N;
    const double d4 = 4.0 * p->dim / (p->dx * p->dx);
    double lphi = 0.0, lmax = 0.0;
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            if (a == b) continue;
            const double v = h->L[a * N + b] * (h->A[a * N + b] * d4 - h->B[a * N + b]);
            if (v > lphi) lphi = v;
            if (h->L[a * N + b] > lmax) lmax = h->L[a * N + b];
        }
    double lam = lphi;
    if (h->K) {
        bool used[2] = {false, false};
        for (int a = 0; a < N; ++a) used[h->ptype[a]] = true;
        double kmax = 0.0, c0max = -1e300, c0min = 1e300, Dmax = 0.0;
        for (int t = 0; t < 2; ++t) {
            if (!used[t]) continue;
            kmax = fmax(kmax, p->k[t]);
            c0max = fmax(c0max, p->c0[t]);
            c0min = fmin(c0min, p->c0[t]);
            Dmax = fmax(Dmax, p->D[t]);
        }
        const double dc0 = c0max - c0min;
        const double chem = lmax * kmax * dc0 * c0max;       // chemical driving-force term
        const double lc = d4 * Dmax * (1.0 + dc0 / 2.0);     // concentration diffusion
        lam = fmax(lphi + chem, lc);
    }
    return 2.0 / lam;
}

// ---- RKL coefficients (Meyer et al. 2012/2014, Legendre basis) ------------
__host__ __device__ double rkl2_b(int j)
{
    if (j < 2) return 1.0 / 3.0;
    const double jj = (double)j;
    return (jj * jj + jj - 2.0) / (2.0 * jj * (jj + 1.0));
}

// Smallest odd stage count whose RKL stability bound with 0.9 dt_e covers dt.
__host__ __device__ int sts_stages(int integ, double dt, double dte)
{
    const double dte9 = 0.9 * dte;
    for (int s = (integ == PF_RKL2) ? 3 : 1;; s += 2) {
        const double ds = (double)s;
        const double bound = (integ == PF_RKL2) ? (ds * ds + ds - 2.0) / 4.0 * dte9 : (ds * ds + ds) / 2.0 * dte9;
        if (bound >= dt || s > 1000001) return s;
    }
}

__host__ __device__ double sts_max_dt(int integ, int s, double dte)
{
    const double ds = (double)s;
    return ((integ == PF_RKL2) ? (ds * ds + ds - 2.0) / 4.0 : (ds * ds + ds) / 2.0) * 0.9 * dte;
}

int method_order(int integ)
{
    switch (integ) {
    case PF_FEULER: return 1;
    case PF_SSP2: return 2;
    case PF_SSP104: return 4;
    case PF_RKL1: return 1;
    default: return 2;
    }
}

// Embedded weights for SSP(10)4: minimum-norm solution of the order-3
// conditions over the first nine stages (the scheme's own weights are all
// 1/10 and already minimal, so the last stage is left out of the embedding).
void ssp104_embedded(double bh[10])
{
    double Am[10][10] = {{0}}, c[10];
    for (int i = 1; i < 5; ++i)
        for (int j = 0; j < i; ++j) Am[i][j] = 1.0 / 6.0;
    for (int j = 0; j < 5; ++j) Am[5][j] = 0.4 / 6.0;
    for (int i = 6; i < 10; ++i) {
        for (int j = 0; j < 10; ++j) Am[i][j] = Am[i - 1][j];
        Am[i][i - 1] += 1.0 / 6.0;
    }
    for (int i = 0; i < 10; ++i) {
        c[i] = 0.0;
        for (int j = 0; j < 10; ++j) c[i] += Am[i][j];
    }
    double M[4][10];
    const double g[4] = {1.0, 0.5, 1.0 / 3.0, 1.0 / 6.0};
    for (int i = 0; i < 10; ++i) {
        double ac = 0.0;
        for (int j = 0; j < 10; ++j) ac += Am[i][j] * c[j];
        const bool use = i < 9;
        M[0][i] = use ? 1.0 : 0.0;
        M[1][i] = use ? c[i] : 0.0;
        M[2][i] = use ? c[i] * c[i] : 0.0;
        M[3][i] = use ? ac : 0.0;
    }
    double G[4][5];
    for (int r = 0; r < 4; ++r) {
        for (int q = 0; q < 4; ++q) {
            double s = 0.0;
            for (int i = 0; i < 10; ++i) s += M[r][i] * M[q][i];
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
            const double f = G[r][col] / G[col][col];
            for (int q = 0; q < 5; ++q) G[r][q] -= f * G[col][q];
        }
    }
    double y[4];
    for (int r = 0; r < 4; ++r) y[r] = G[r][4] / G[r][r];
    for (int i = 0; i < 10; ++i) {
        double s = 0.0;
        for (int r = 0; r < 4; ++r) s += M[r][i] * y[r];
        bh[i] = s;
    }
}

// ---- PID controller with bias (Sec. 3.3, Soderlind 2006 form) --------------
struct CtrlState {
    double b, E1, E2, dt1, dt2;
    int nhist;
};

// One controller update on the state of the last accepted steps; the host
// loop and the device-driven loop share it.  Returns the next step size.
__host__ __device__ double pid_bias(CtrlState &c, double err, double dt, int P, int *accept)
{
    const double k1 = 1.25, k2 = 0.5, k3 = -0.6, k4 = 0.25, k5 = 0.0;
    const double ex = 1.0 / (double)(P + 1);
    double E = err / c.b;
    if (E < 1e-10) E = 1e-10;
    double F = pow(E, -k1 * ex);
    if (c.nhist >= 1) F = F * pow(c.E1, -k2 * ex) * pow(dt / c.dt1, k4);
    if (c.nhist >= 2) F = F * pow(c.E2, -k3 * ex) * pow(c.dt1 / c.dt2, k5);
    const int acc = err < 1.0;
    if (acc) {
        c.E2 = c.E1;
        c.E1 = E;
        c.dt2 = c.dt1;
        c.dt1 = dt;
        if (c.nhist < 2) c.nhist++;
        const double nb = sqrt(c.b);
        c.b = nb > 0.98 ? 0.98 : nb;
    } else {
        const double nb = c.b * c.b;
        c.b = nb < 0.1 ? 0.1 : nb;
        if (F > 1.0) F = pow(E, -k1 * ex);
    }
    *accept = acc;
    return dt * (1.0 + 5.0 * atan((F - 1.0) / 5.0));
}

double controller(pf_handle *h, double err, double dt, int P, int *accept)
{
    CtrlState c{h->b, h->E1, h->E2, h->dt1, h->dt2, h->nhist};
    const double r = pid_bias(c, err, dt, P, accept);
    h->b = c.b;
    h->E1 = c.E1;
    h->E2 = c.E2;
    h->dt1 = c.dt1;
    h->dt2 = c.dt2;
    h->nhist = c.nhist;
    return r;
}

void reset_controller(pf_handle *h)
{
    h->b = 0.9;
    h->E1 = h->E2 = h->dt1 = h->dt2 = 0.0;
    h->nhist = 0;
    h->dt_next = 0.0;
}

int grid_for(long long n) { long long b = (n + 255) / 256; return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096); }

// ---- one step ---------------------------------------------------------------
// Runs the stages of one step of size dt with s stages from buf[iu].  On
// return *out is the buffer index holding the candidate u^{n+1}; when
// want_err is set, the error partials of Sec. 3.3 are in part_sum/part_cnt.
template <typename T>
int do_step(pf_handle *h, int integ, double dt, int s, const pf_tol *tol, bool want_err, int *out, long long *evals)
{
    const int U = h->iu;
    int w[NBUF - 1], nw = 0;
    for (int k = 0; k < NBUF; ++k) if (k != U) w[nw++] = k;
    int st;
    auto B = [&](int k) { return (T *)vec(h, k); };

    if (integ == PF_FEULER) {
        h->cur_kind = PF_PASS_EULER;
        Pass<T> P = blank_pass<T>(h);
        P.in = B(U); P.out = B(w[0]); P.a1 = 1.0; P.b1 = dt;
        P.count_step = !want_err;
        if ((st = run_pass<T>(h, P))) return st;
        *out = w[0];
        *evals += 1;
        return PF_OK;
    }
    if (integ == PF_SSP2) {
        // Alg. ssp2: s-1 Euler substeps of dt/(s-1), then the final combination
        int q1 = w[0], q3 = w[1];
        h->cur_kind = PF_PASS_SSP;
        const double hs = dt / (double)(s - 1);
        int cur = U;
        for (int k = 1; k <= s - 1; ++k) {
            Pass<T> P = blank_pass<T>(h);
            P.in = B(cur); P.out = B(q1); P.a1 = 1.0; P.b1 = hs;
            if ((st = run_pass<T>(h, P))) return st;
            cur = q1;
            int t = q1; q1 = q3; q3 = t;
        }
        Pass<T> P = blank_pass<T>(h);
        P.in = B(cur); P.p0 = B(U);
        P.a0 = 1.0 / (double)s; P.a1 = (double)(s - 1) / (double)s; P.b1 = dt / (double)s;
        P.out = B(q1);
        P.count_step = !want_err;
        if ((st = run_pass<T>(h, P))) return st;
        *out = q1;
        *evals += s;
        return PF_OK;
    }
    if (integ == PF_SSP104) {
        // Ketcheson (2008) low-storage SSP(10,4) with an extra stage buffer and
        // the embedded accumulator z = u^n + dt sum bh_i F_i (Sec. 3.3).  The
        // register q2 is kept divided by 2/5 so that every combination is
        // affine: after stage 5 q2 = u^n/10 + 9 q1/10 and q1 <- 6 q2 - 5 q1;
        // the result is 2 q2/5 + 3 q1/5 + dt F(q1)/10 (the same method).
        double bh[10];
        ssp104_embedded(bh);
        int q1 = w[0], q3 = w[1], q2 = w[2], zb = w[3];
        h->cur_kind = PF_PASS_SSP;
        const double h6 = dt / 6.0;
        int cur = U;
        for (int k = 1; k <= 9; ++k) {
            Pass<T> P = blank_pass<T>(h);
            P.in = B(cur); P.a1 = 1.0; P.b1 = h6;
            if (want_err) { P.zin = (k == 1) ? B(U) : B(zb); P.zout = B(zb); P.bz = dt * bh[k - 1]; }
            if (k == 5) {
                P.out2 = B(q2); P.q2in = B(U);
                P.m25 = 0.1; P.m15 = 6.0;
            }
            P.out = B(q1);
            if ((st = run_pass<T>(h, P))) return st;
            cur = q1;
            int t = q1; q1 = q3; q3 = t;
        }
        Pass<T> P = blank_pass<T>(h);
        P.in = B(cur); P.p0 = B(q2); P.a0 = 0.4; P.a1 = 0.6; P.b1 = dt / 10.0;
        P.out = B(q1);
        P.count_step = !want_err;
        if (want_err) {
            P.zin = B(zb); P.zout = B(zb); P.bz = dt * bh[9]; P.embedded_err = 1; P.uw = B(U);
            P.r_phi = tol->r_phi; P.a_phi = tol->a_phi; P.r_c = tol->r_c; P.a_c = tol->a_c;
        }
        if ((st = run_pass<T>(h, P))) return st;
        *out = q1;
        *evals += 10;
        return PF_OK;
    }
    // RKL1 / RKL2 (Eq. sts), ring of three stage buffers plus F(u^n)
    const bool o2 = (integ == PF_RKL2);
    // F(u^n) kept by the previous accepted step's error sweep (reuse)
    const bool reuse = h->reuse_on && h->rhs_valid && h->rhs_iu == U && h->rhs_buf >= 0 && h->rhs_buf != U;
    int ring[3] = {w[0], w[1], w[2]};
    int r0 = w[3];
    if (reuse) {
        r0 = h->rhs_buf;
        int n = 0;
        for (int k = 0; k < NBUF; ++k) if (k != U && k != r0) ring[n++] = k;
    }
    const double ds = (double)s;
    const double w1 = o2 ? 4.0 / (ds * ds + ds - 2.0) : 2.0 / (ds * ds + ds);
    const double mt1 = o2 ? rkl2_b(1) * w1 : w1;
    if (reuse) {
        // stage 1 from the stored F(u^n): no RHS evaluation; the stored RHS is
        // consumed (replaced by the effective one where the fix applies)
        h->cur_kind = PF_PASS_STS_FIRST;
        if ((st = prof_begin(h))) return st;
        if (PF_FIRST_RECOMPUTE)
            first_from_rhs_recompute_kernel<T><<<grid_for(h->V), 256, 0, h->stream>>>(
                B(U), B(ring[0]), B(r0), h->V, h->Vs, h->N, h->K, mt1 * dt, o2 ? 1 : 0, h->dflag);
        else
            first_from_rhs_kernel<T><<<grid_for(h->V), 256, 0, h->stream>>>(B(U), B(ring[0]), B(r0), h->V, h->Vs,
                                                                             h->N, h->K, mt1 * dt, o2 ? 1 : 0, h->dflag);
        h->launches++;
        if (cudaGetLastError() != cudaSuccess) return PF_EDEVICE;
        if ((st = prof_end(h))) return st;
        h->rhs_valid = false;
    } else {
        h->cur_kind = PF_PASS_STS_FIRST;
        Pass<T> P = blank_pass<T>(h);
        P.in = B(U); P.a1 = 1.0; P.b1 = mt1 * dt; P.out = B(ring[0]); P.r0out = B(r0); P.fix_first = o2 ? 1 : 0;
        P.count_step = !want_err && s == 1;
        if ((st = run_pass<T>(h, P))) return st;
    }
    h->cur_kind = o2 ? PF_PASS_RKL2 : PF_PASS_RKL1;
    for (int j = 2; j <= s; ++j) {
        const double dj = (double)j;
        double mu, nu, mt, gt;
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
        Pass<T> P = blank_pass<T>(h);
        P.in = B(ring[(j - 2) % 3]);
        P.p2 = (j == 2) ? B(U) : B(ring[(j - 3) % 3]);
        P.a1 = mu; P.a2 = nu; P.b1 = mt * dt;
        if (o2) { P.p0 = B(U); P.a0 = (1.0 - mu) - nu; P.r0in = B(r0); P.b0 = gt * dt; }
        P.out = B(ring[(j - 1) % 3]);
        P.count_step = !want_err && j == s;
        if ((st = run_pass<T>(h, P))) return st;
    }
    const int fin = ring[(s - 1) % 3];
    *evals += reuse ? s - 1 : s;
    h->rhs_pending = -1;
    if (want_err) {
        // Sommeijer estimate with F(u^{n+1}) (Sec. 3.3): one more RHS sweep;
        // with reuse it also keeps F(u^{n+1}) in a stage buffer it no longer needs
        h->cur_kind = PF_PASS_STS_ERR;
        Pass<T> P = blank_pass<T>(h);
        P.mode = pfk::MODE_ERR;
        P.in = B(fin); P.p0 = B(U); P.r0in = B(r0); P.dt = dt; P.project = 0;
        P.r_phi = tol->r_phi; P.a_phi = tol->a_phi; P.r_c = tol->r_c; P.a_c = tol->a_c;
        if (h->reuse_on) {
            h->rhs_pending = ring[(s + 1) % 3];
            P.r0out = B(h->rhs_pending);
        }
        if ((st = run_pass<T>(h, P))) return st;
        *evals += 1;
    }
    *out = fin;
    return PF_OK;
}

// Device flags -> status: a non-positive simplex sum is an instability; more
// nontrivial phases in one cell than the kernel's list holds is unsupported.
__host__ __device__ int flag_status(int flag)
{
    if (flag & pfk::FLAG_NZ_OVERFLOW) return PF_EINVAL;
    if (flag & pfk::FLAG_TIMEOUT) return PF_ETIMEOUT;
    return PF_EUNSTABLE;
}

int read_error(pf_handle *h, double *err)
{
    h->cur_kind = PF_PASS_OTHER;
    int pst = prof_begin(h);
    if (pst) return pst;
    finalize_err_kernel<<<1, 256, 0, h->stream>>>(h->part_sum, h->part_cnt, h->grid, h->dres, h->dcnt, h->dpartn);
    h->launches++;
    if (cudaGetLastError() != cudaSuccess) return PF_EDEVICE;
    if ((pst = prof_end(h))) return pst;
    double s;
    long long c;
    int flag;
    if (cudaMemcpyAsync(&s, h->dres, sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) return PF_EDEVICE;
    if (cudaMemcpyAsync(&c, h->dcnt, sizeof(long long), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) return PF_EDEVICE;
    if (cudaMemcpyAsync(&flag, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) return PF_EDEVICE;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return PF_EDEVICE;
    if (flag) return flag_status(flag);
    *err = c > 0 ? sqrt(s / (double)c) : 0.0;
    return PF_OK;
}

int check_flag(pf_handle *h, int *failed_step = nullptr)
{
    int w[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(w, h->dflag, PF_FLAG_BYTES, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) return PF_EDEVICE;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return PF_EDEVICE;
    if (failed_step) *failed_step = w[3];
    return w[0] ? flag_status(w[0]) : PF_OK;
}

// Capture full fixed steps of size dt with s stages into a graph until the
// buffer holding u^n is the one it started from (so the graph can be
// replayed); nothing executes during capture.  Returns false (and leaves the
// handle unchanged) when capture is not possible.
template <typename T>
bool capture_fixed_steps(pf_handle *h, int integ, double dt, int s)
{
    if (h->gexec && h->g_integ == integ && h->g_s == s && h->g_dt == dt && h->g_iu == h->iu) return true;
    if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
    const int iu0 = h->iu;
    const long long l0 = h->launches;
    long long ev = 0;
    int period = 0;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    bool ok = true;
    std::vector<int> seq;
    do {
        int cand = -1;
        if (do_step<T>(h, integ, dt, s, nullptr, false, &cand, &ev) != PF_OK) { ok = false; break; }
        h->iu = cand;
        seq.push_back(cand);
        period++;
    } while (h->iu != iu0 && period < 12);
    if (cudaStreamEndCapture(h->stream, &graph) != cudaSuccess) ok = false;
    ok = ok && graph && h->iu == iu0;
    h->iu = iu0;
    const long long nl = h->launches - l0;
    h->launches = l0;
    cudaGraphExec_t exec = nullptr;
    if (ok && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) ok = false;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        cudaGetLastError();
        return false;
    }
    h->gexec = exec;
    h->g_integ = integ;
    h->g_s = s;
    h->g_dt = dt;
    h->g_iu = iu0;
    h->g_period = period;
    h->g_seq = seq;
    h->g_evals = ev;
    h->g_launches = nl;
    return true;
}

// ---------------------------------------------------------------------------
// Device-driven adaptive RKL steps (PF_STEP_DEVICE_LOOP).  Every decision of
// the adaptive loop of Sec. 3.2/3.3 -- the output-time clip, the stage count,
// each stage's buffers and coefficients, the error norm, the PID controller
// with bias and accept/reject -- is taken on the GPU by single-thread
// kernels, and the attempts run as one CUDA graph with two conditional WHILE
// nodes (attempts; stages 2..s).  A launch carries up to DL_CAP attempts, so
// the host waits once per launch instead of once per attempt.  Every WHILE
// ends: the attempt loop after DL_CAP attempts per launch, the stage loop
// after s <= max_stages stages.
// ---------------------------------------------------------------------------
constexpr int DL_CAP = 256;

template <typename P>
bool dmalloc(pf_handle *h, P **p, size_t bytes);
void dfree(pf_handle *h, void *p);

struct DevCtl {
    // inputs, set by the host for each pf_step call
    double t_end, dte, tol[4];
    int integ, max_stages, order, trace_cap;
    int kpp;                         // kernels each pass launches
    long long max_attempts;          // 0: no limit
    double *tr_dt, *tr_err;
    int *tr_s, *tr_acc;
    void *buf[NBUF];
    // loop state (read back by the host after every launch)
    double t, dt, hs, hlast, elast;
    double b, E1, E2, dt1, dt2;
    int nhist, iu, s, j, last, status, ntr;
    long long evals, acc_n, rej_n, attempts, launch_attempts, launches;
};

// The four buffers other than u^n in index order: three RKL stage buffers
// and F(u^n) (the assignment do_step uses).
__host__ __device__ inline void dl_buffers(int iu, int w[NBUF - 1])
{
    int n = 0;
    for (int k = 0; k < NBUF; ++k) if (k != iu) w[n++] = k;
}

__global__ void dl_begin(DevCtl *c, cudaGraphConditionalHandle hout)
{
    c->launch_attempts = 0;
    c->launches += 1;
    const bool go = c->status == PF_OK && c->t < c->t_end && (c->max_attempts == 0 || c->attempts < c->max_attempts);
    cudaGraphSetConditional(hout, go ? 1u : 0u);
}

// Stage 1: step size (clipped to the output time), stage count, description.
template <typename T>
__global__ void dl_first(DevCtl *c, Pass<T> *d, cudaGraphConditionalHandle hin)
{
    const bool o2 = c->integ == PF_RKL2;
    const double rem = c->t_end - c->t;
    double hs = c->dt;
    int last = 0;
    if (hs >= rem * (1.0 - 1e-9)) { hs = rem; last = 1; }
    int s = sts_stages(c->integ, hs, c->dte);
    if (s > c->max_stages) {
        s = c->max_stages | 1;
        hs = sts_max_dt(c->integ, s, c->dte);
        last = 0;
    }
    c->hs = hs;
    c->s = s;
    c->last = last;
    c->j = 2;
    int w[NBUF - 1];
    dl_buffers(c->iu, w);
    const double ds = (double)s;
    const double w1 = o2 ? 4.0 / (ds * ds + ds - 2.0) : 2.0 / (ds * ds + ds);
    const double mt1 = o2 ? rkl2_b(1) * w1 : w1;
    Pass<T> P = d[3];
    P.in = (const T *)c->buf[c->iu];
    P.a1 = 1.0;
    P.b1 = mt1 * hs;
    P.out = (T *)c->buf[w[0]];
    P.r0out = (T *)c->buf[w[3]];
    P.fix_first = o2 ? 1 : 0;
    d[0] = P;
    cudaGraphSetConditional(hin, s >= 2 ? 1u : 0u);
}

// Stage j >= 2 of Eq. sts: coefficients and the ring of stage buffers.
template <typename T>
__global__ void dl_stage(DevCtl *c, Pass<T> *d, cudaGraphConditionalHandle hin)
{
    const bool o2 = c->integ == PF_RKL2;
    const int j = c->j, s = c->s;
    const double hs = c->hs, ds = (double)s, dj = (double)j;
    const double w1 = o2 ? 4.0 / (ds * ds + ds - 2.0) : 2.0 / (ds * ds + ds);
    double mu, nu, mt, gt;
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
    int w[NBUF - 1];
    dl_buffers(c->iu, w);
    Pass<T> P = d[3];
    P.in = (const T *)c->buf[w[(j - 2) % 3]];
    P.p2 = (j == 2) ? (const T *)c->buf[c->iu] : (const T *)c->buf[w[(j - 3) % 3]];
    P.a1 = mu;
    P.a2 = nu;
    P.b1 = mt * hs;
    if (o2) {
        P.p0 = (const T *)c->buf[c->iu];
        P.a0 = (1.0 - mu) - nu;
        P.r0in = (const T *)c->buf[w[3]];
        P.b0 = gt * hs;
    }
    P.out = (T *)c->buf[w[(j - 1) % 3]];
    d[1] = P;
    c->j = j + 1;
    cudaGraphSetConditional(hin, (j + 1 <= s) ? 1u : 0u);
}

// The error sweep's description (Sommeijer estimate with F(u^{n+1})).
template <typename T>
__global__ void dl_err(DevCtl *c, Pass<T> *d)
{
    int w[NBUF - 1];
    dl_buffers(c->iu, w);
    Pass<T> P = d[3];
    P.mode = pfk::MODE_ERR;
    P.in = (const T *)c->buf[w[(c->s - 1) % 3]];
    P.p0 = (const T *)c->buf[c->iu];
    P.r0in = (const T *)c->buf[w[3]];
    P.dt = c->hs;
    P.project = 0;
    P.r_phi = c->tol[0];
    P.a_phi = c->tol[1];
    P.r_c = c->tol[2];
    P.a_c = c->tol[3];
    d[2] = P;
}

// Error norm, controller, accept/reject, trace; continue or end the launch.
__global__ void dl_ctrl(DevCtl *c, const double *dres, const long long *dcnt, const int *dflag,
                        cudaGraphConditionalHandle hout)
{
    c->attempts++;
    c->launch_attempts++;
    c->evals += c->s + 1;
    // planning kernels and passes of stages 1..s and the error sweep, the
    // norm and this kernel
    c->launches += ((long long)c->s + 1) * (1 + c->kpp) + 2;
    int st = PF_OK;
    const int flag = *dflag;
    double err = 0.0;
    if (flag) {
        st = flag_status(flag);
    } else {
        const long long n = *dcnt;
        err = n > 0 ? sqrt(*dres / (double)n) : 0.0;
        if (!isfinite(err)) st = PF_EUNSTABLE;
    }
    if (st == PF_OK) {
        CtrlState cs{c->b, c->E1, c->E2, c->dt1, c->dt2, c->nhist};
        int acc = 0;
        const double dtn = pid_bias(cs, err, c->hs, c->order, &acc);
        c->b = cs.b;
        c->E1 = cs.E1;
        c->E2 = cs.E2;
        c->dt1 = cs.dt1;
        c->dt2 = cs.dt2;
        c->nhist = cs.nhist;
        if (c->ntr < c->trace_cap) {
            c->tr_dt[c->ntr] = c->hs;
            c->tr_s[c->ntr] = c->s;
            c->tr_err[c->ntr] = err;
            c->tr_acc[c->ntr] = acc;
            c->ntr++;
        }
        c->hlast = c->hs;
        c->elast = err;
        if (acc) {
            int w[NBUF - 1];
            dl_buffers(c->iu, w);
            c->iu = w[(c->s - 1) % 3];
            c->t = c->last ? c->t_end : c->t + c->hs;
            c->acc_n++;
        } else {
            c->rej_n++;
            if (c->rej_n > 100000) st = PF_EUNSTABLE;
        }
        c->dt = dtn;
    }
    c->status = st;
    const bool go = st == PF_OK && c->t < c->t_end && c->launch_attempts < DL_CAP &&
                    (c->max_attempts == 0 || c->attempts < c->max_attempts);
    cudaGraphSetConditional(hout, go ? 1u : 0u);
}

void free_devloop(pf_handle *h)
{
    if (h->dl_exec) cudaGraphExecDestroy(h->dl_exec);
    if (h->dl_graph) cudaGraphDestroy(h->dl_graph);
    h->dl_exec = nullptr;
    h->dl_graph = nullptr;
    h->dl_integ = -1;
}

// Capture the launches fn() makes on the handle's stream into `graph`
// (after the nodes deps); *leaves receives the last captured nodes.
template <class F>
bool capture_to(pf_handle *h, cudaGraph_t graph, const cudaGraphNode_t *deps, size_t ndeps,
                std::vector<cudaGraphNode_t> *leaves, F fn)
{
    if (cudaStreamBeginCaptureToGraph(h->stream, graph, deps, nullptr, ndeps, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
        return false;
    bool ok = fn();
    if (ok && leaves) {
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t *d = nullptr;
        size_t n = 0;
        ok = cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, nullptr, &d, nullptr, &n) == cudaSuccess && n > 0;
        if (ok) leaves->assign(d, d + n);
    }
    cudaGraph_t g = nullptr;
    const bool ended = cudaStreamEndCapture(h->stream, &g) == cudaSuccess;
    return ok && ended;
}

bool add_while(cudaGraph_t graph, const cudaGraphNode_t *dep, size_t ndep, cudaGraphConditionalHandle hc,
               cudaGraphNode_t *node, cudaGraph_t *body)
{
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = hc;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (cudaGraphAddNode(node, graph, dep, nullptr, ndep, &cp) != cudaSuccess) return false;
    *body = cp.conditional.phGraph_out[0];
    return true;
}

// Build (once per integrator) the graph: begin -> WHILE(attempts){ plan and
// stage 1 -> WHILE(stages 2..s){ plan, stage } -> error sweep, norm,
// controller }.  The kernels are captured straight into the conditional
// nodes' body graphs; every body sets its own node's condition.
template <typename T>
int build_devloop(pf_handle *h, int integ)
{
    if (h->dl_exec && h->dl_integ == integ) return PF_OK;
    free_devloop(h);
    if (!h->dl_ctl && !dmalloc(h, &h->dl_ctl, sizeof(DevCtl))) return PF_ENOMEM;
    if (!h->dl_desc && !dmalloc(h, &h->dl_desc, 4 * sizeof(Pass<double>))) return PF_ENOMEM;
    DevCtl *ctl = (DevCtl *)h->dl_ctl;
    Pass<T> *desc = (Pass<T> *)h->dl_desc;
    const Pass<T> base = blank_pass<T>(h);
    if (cudaMemcpyAsync(desc + 3, &base, sizeof(base), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        return PF_EDEVICE;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return PF_EDEVICE;
    const unsigned body_sig = integ == PF_RKL2 ? (pfk::SIG_P0 | pfk::SIG_P2 | pfk::SIG_R0IN | pfk::SIG_PROJECT)
                                               : (pfk::SIG_P2 | pfk::SIG_PROJECT);
    const T *A = (const T *)h->dA, *B = (const T *)h->dB, *L = (const T *)h->dL;
    cudaStream_t st = h->stream;
    cudaGraph_t top = nullptr, outer = nullptr, inner = nullptr;
    cudaGraphConditionalHandle hout = 0, hin = 0;
    cudaGraphNode_t nw, ni;
    std::vector<cudaGraphNode_t> lb, la;
    bool ok = cudaGraphCreate(&top, 0) == cudaSuccess &&
              cudaGraphConditionalHandleCreate(&hout, top, 0, cudaGraphCondAssignDefault) == cudaSuccess;
    ok = ok && capture_to(h, top, nullptr, 0, &lb, [&] {
        dl_begin<<<1, 1, 0, st>>>(ctl, hout);
        return cudaGetLastError() == cudaSuccess;
    });
    ok = ok && add_while(top, lb.data(), lb.size(), hout, &nw, &outer);
    ok = ok && cudaGraphConditionalHandleCreate(&hin, outer, 0, 0) == cudaSuccess;
    ok = ok && capture_to(h, outer, nullptr, 0, &la, [&] {
        dl_first<T><<<1, 1, 0, st>>>(ctl, desc, hin);
        return cudaGetLastError() == cudaSuccess &&
               pfk::launch_stage_d<T>(h->g, pfk::SIG_R0OUT | pfk::SIG_PROJECT, desc + 0, st, A, B, L, h->dptype) == 0;
    });
    ok = ok && add_while(outer, la.data(), la.size(), hin, &ni, &inner);
    ok = ok && capture_to(h, inner, nullptr, 0, nullptr, [&] {
        dl_stage<T><<<1, 1, 0, st>>>(ctl, desc, hin);
        return cudaGetLastError() == cudaSuccess &&
               pfk::launch_stage_d<T>(h->g, body_sig, desc + 1, st, A, B, L, h->dptype) == 0;
    });
    ok = ok && capture_to(h, outer, &ni, 1, nullptr, [&] {
        dl_err<T><<<1, 1, 0, st>>>(ctl, desc);
        if (cudaGetLastError() != cudaSuccess) return false;
        if (pfk::launch_stage_d<T>(h->g, pfk::SIG_ERR, desc + 2, st, A, B, L, h->dptype) != 0) return false;
        finalize_err_kernel<<<1, 256, 0, st>>>(h->part_sum, h->part_cnt, h->grid, h->dres, h->dcnt, h->dpartn);
        dl_ctrl<<<1, 1, 0, st>>>(ctl, h->dres, h->dcnt, h->dflag, hout);
        return cudaGetLastError() == cudaSuccess;
    });
    cudaGraphExec_t exec = nullptr;
    ok = ok && cudaGraphInstantiate(&exec, top, 0) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        if (top) cudaGraphDestroy(top);
        return PF_EDEVICE;
    }
    h->dl_graph = top;
    h->dl_exec = exec;
    h->dl_integ = integ;
    return PF_OK;
}

// Adaptive RKL1/RKL2 to t_end through the device-driven graph.
template <typename T>
int devloop(pf_handle *h, int integ, double t_end, const pf_tol *tol, const pf_step_opts *o, pf_stats *stats)
{
    int st = build_devloop<T>(h, integ);
    if (st) return st;
    DevCtl c;
    memset(&c, 0, sizeof(c));
    c.t_end = t_end;
    c.dte = h->dte;
    c.tol[0] = tol->r_phi;
    c.tol[1] = tol->a_phi;
    c.tol[2] = tol->r_c;
    c.tol[3] = tol->a_c;
    c.integ = integ;
    c.max_stages = o->max_stages > 0 ? o->max_stages : 1001;
    c.order = method_order(integ);
    c.kpp = pfk::kernels_per_pass_d<T>(h->g);
    c.max_attempts = o->max_attempts;
    c.trace_cap = o->trace_cap > 0 ? o->trace_cap : 0;
    for (int k = 0; k < NBUF; ++k) c.buf[k] = h->buf[k];
    c.t = h->t;
    c.dt = h->dt_next > 0.0 ? h->dt_next : (o->dt0 > 0.0 ? o->dt0 : 0.9 * h->dte);
    c.b = h->b;
    c.E1 = h->E1;
    c.E2 = h->E2;
    c.dt1 = h->dt1;
    c.dt2 = h->dt2;
    c.nhist = h->nhist;
    c.iu = h->iu;
    void *trbuf = nullptr;
    if (c.trace_cap > 0) {
        const size_t n = (size_t)c.trace_cap;
        if (!dmalloc(h, &trbuf, n * (2 * sizeof(double) + 2 * sizeof(int)))) return PF_ENOMEM;
        c.tr_dt = (double *)trbuf;
        c.tr_err = c.tr_dt + n;
        c.tr_s = (int *)(c.tr_err + n);
        c.tr_acc = c.tr_s + n;
    }
    DevCtl *dctl = (DevCtl *)h->dl_ctl;
    st = PF_OK;
    if (cudaMemsetAsync(h->dflag, 0, PF_FLAG_BYTES, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(dctl, &c, sizeof(c), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        st = PF_EDEVICE;
    long long prev_attempts = -1;
    while (st == PF_OK) {
        if (cudaGraphLaunch(h->dl_exec, h->stream) != cudaSuccess ||
            cudaMemcpyAsync(&c, dctl, sizeof(c), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess) {
            st = PF_EDEVICE;
            break;
        }
        if (c.status != PF_OK) { st = c.status; break; }
        if (!(c.t < t_end) || (c.max_attempts > 0 && c.attempts >= c.max_attempts)) break;
        if (c.attempts == prev_attempts) { st = PF_EDEVICE; break; }   // a launch that made no attempt
        prev_attempts = c.attempts;
    }
    if (trbuf) {
        const size_t n = (size_t)c.ntr;
        bool okc = true;
        if (o->trace_dt) okc = okc && cudaMemcpyAsync(o->trace_dt, c.tr_dt, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream) == cudaSuccess;
        if (o->trace_err) okc = okc && cudaMemcpyAsync(o->trace_err, c.tr_err, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream) == cudaSuccess;
        if (o->trace_s) okc = okc && cudaMemcpyAsync(o->trace_s, c.tr_s, n * sizeof(int), cudaMemcpyDeviceToHost, h->stream) == cudaSuccess;
        if (o->trace_acc) okc = okc && cudaMemcpyAsync(o->trace_acc, c.tr_acc, n * sizeof(int), cudaMemcpyDeviceToHost, h->stream) == cudaSuccess;
        dfree(h, trbuf);
        if (cudaStreamSynchronize(h->stream) != cudaSuccess || !okc) st = st ? st : PF_EDEVICE;
    }
    if (o->trace_len) *o->trace_len = c.ntr;
    h->t = c.t;
    h->iu = c.iu;
    h->b = c.b;
    h->E1 = c.E1;
    h->E2 = c.E2;
    h->dt1 = c.dt1;
    h->dt2 = c.dt2;
    h->nhist = c.nhist;
    h->dt_next = c.dt;
    h->launches += c.launches;
    if (stats) {
        stats->rhs_evals = c.evals;
        stats->steps_accepted = c.acc_n;
        stats->steps_rejected = c.rej_n;
        stats->t = h->t;
        stats->dt_last = c.hlast;
        stats->err_last = c.elast;
        stats->dt_e = h->dte;
        stats->dt_next = h->dt_next;
        stats->kernel_launches = c.launches;
    }
    return st;
}

// Size *hs (in: the proposal), stage count and "lands on t_end" flag of the
// next attempt (Sec. 3.2 stage rule; Sec. 5 output times): an adaptive
// proposal within 1e-9 of the remaining time rem is stretched onto it; fixed
// step kfix + 1 of nfix, the last shortened onto t_end; an RKL step needing
// more than max_stages stages is refused (fixed) or cut to the largest step
// max_stages (rounded up to odd) allows (adaptive).
int plan_attempt(const pf_handle *h, int integ, bool adaptive, double rem, long long kfix, long long nfix,
                 int ssp_stages, int max_stages, double *hs, int *s, bool *last)
{
    const bool sts = (integ == PF_RKL1 || integ == PF_RKL2);
    *last = false;
    if (adaptive) {
        if (*hs >= rem * (1.0 - 1e-9)) { *hs = rem; *last = true; }
    } else {
        *last = (kfix + 1 >= nfix);
        if (*last) *hs = rem;
    }
    *s = 1;
    if (sts) {
        *s = sts_stages(integ, *hs, h->dte);
        if (*s > max_stages && !adaptive) return PF_EINVAL;
        if (*s > max_stages) {
            *s = max_stages | 1;
            *hs = sts_max_dt(integ, *s, h->dte);
            *last = false;
        }
    } else if (integ == PF_SSP2) {
        *s = ssp_stages;
    } else if (integ == PF_SSP104) {
        *s = 10;
    }
    return PF_OK;
}

template <typename T>
int step_loop(pf_handle *h, int integ, double t_end, const pf_tol *tol, const pf_step_opts *o, pf_stats *stats)
{
    const bool adaptive = !(o->dt_mult > 0.0);
    const bool sts = (integ == PF_RKL1 || integ == PF_RKL2);
    if (adaptive && (integ == PF_FEULER || integ == PF_SSP2)) return PF_EINVAL;
    if (adaptive && !tol) return PF_EINVAL;
    if (integ == PF_SSP2 && o->ssp_stages < 2) return PF_EINVAL;
    if (o->flags & PF_STEP_DEVICE_LOOP) {
        // the descriptor-driven kernels cover FP64 and FP32 dense storage with N <= 32
        if (!(adaptive && sts) || !h->stream || h->prof_on || (o->flags & PF_STEP_REUSE_RHS) || h->masked ||
            !(sizeof(T) == 8 || h->N <= 32) || h->Vs >= 0x7fffffffLL || h->g.simplex != pfk::SIMPLEX_STANDARD ||
            h->slots)
            return PF_EINVAL;
        h->rhs_valid = false;
        return devloop<T>(h, integ, t_end, tol, o, stats);
    }
    // the pointwise first stage of the reuse path applies the standard S only
    if ((o->flags & PF_STEP_REUSE_RHS) && (h->g.simplex != pfk::SIMPLEX_STANDARD || h->slots)) return PF_EINVAL;
    // slot storage: the passes of FE, SSP(s)2, RKL1 and RKL2
    if (h->slots && integ == PF_SSP104) return PF_EINVAL;
    const int max_stages = o->max_stages > 0 ? o->max_stages : 1001;
    long long evals = 0, acc_n = 0, rej_n = 0, attempts = 0;
    const long long launches0 = h->launches;
    double dt = adaptive ? (h->dt_next > 0.0 ? h->dt_next : (o->dt0 > 0.0 ? o->dt0 : 0.9 * h->dte)) : o->dt_mult * h->dte;
    double hlast = 0.0, elast = 0.0;
    int ntr = 0, status = PF_OK;
    // fixed steps: step k ends at t0 + k dt (no drift); the last is shortened
    // to land exactly on t_end (Sec. 5, output at target times)
    const double t0 = h->t;
    long long nfix = 0, kfix = 0;
    if (!adaptive) {
        nfix = (long long)ceil((t_end - t0) / dt - 1e-9);
        if (nfix < 1) nfix = 1;
    }
    if (cudaMemsetAsync(h->dflag, 0, PF_FLAG_BYTES, h->stream) != cudaSuccess) return PF_EDEVICE;
    // reuse of F(u^{n+1}): adaptive RKL steps in dense storage only
    h->reuse_on = (o->flags & PF_STEP_REUSE_RHS) && adaptive && sts && !h->masked;
    if (!h->reuse_on) h->rhs_valid = false;
    const bool graphs = !adaptive && h->stream != nullptr && !h->prof_on && !(o->flags & PF_STEP_NO_GRAPH) &&
                        o->max_attempts == 0 && o->trace_cap == 0;
    // fixed steps: the buffer holding u^n after each step, so that a failure
    // found at the end of the call can be traced back to the last good step
    const int iu0 = h->iu;
    std::vector<signed char> iu_hist;
    while (h->t < t_end) {
        if (o->max_attempts > 0 && attempts >= o->max_attempts) break;
        // replay whole groups of full fixed steps from a CUDA graph
        if (graphs && nfix - 1 - kfix >= 8) {
            const int s_full = sts ? sts_stages(integ, dt, h->dte)
                                   : (integ == PF_SSP2 ? o->ssp_stages : (integ == PF_SSP104 ? 10 : 1));
            if (!(sts && s_full > max_stages) && capture_fixed_steps<T>(h, integ, dt, s_full)) {
                const long long groups = (nfix - 1 - kfix) / h->g_period;
                for (long long r = 0; r < groups; ++r)
                    if (cudaGraphLaunch(h->gexec, h->stream) != cudaSuccess) { status = PF_EDEVICE; break; }
                if (status) break;
                for (long long r = 0; r < groups; ++r)
                    for (int b : h->g_seq) iu_hist.push_back((signed char)b);
                kfix += groups * h->g_period;
                attempts += groups * h->g_period;
                acc_n += groups * h->g_period;
                evals += groups * h->g_evals;
                h->launches += groups * h->g_launches;
                h->graph_replays += groups;
                h->t = t0 + (double)kfix * dt;
                hlast = dt;
                continue;
            }
        }
        double hs = dt;
        bool last = false;
        int s = 1;
        if ((status = plan_attempt(h, integ, adaptive, t_end - h->t, kfix, nfix, o->ssp_stages, max_stages, &hs, &s,
                                   &last)))
            break;
        int cand = -1;
        if ((status = do_step<T>(h, integ, hs, s, tol, adaptive, &cand, &evals))) break;
        attempts++;
        double err = 0.0;
        int acc = 1;
        if (adaptive) {
            if ((status = read_error(h, &err))) break;
            if (!isfinite(err)) { status = PF_EUNSTABLE; break; }
            dt = controller(h, err, hs, method_order(integ), &acc);
        }
        if (o->trace_cap > ntr) {
            if (o->trace_dt) o->trace_dt[ntr] = hs;
            if (o->trace_s) o->trace_s[ntr] = s;
            if (o->trace_err) o->trace_err[ntr] = err;
            if (o->trace_acc) o->trace_acc[ntr] = acc;
            ntr++;
        }
        hlast = hs;
        elast = err;
        if (acc) {
            h->iu = cand;
            if (!adaptive) {
                kfix++;
                h->t = last ? t_end : t0 + (double)kfix * dt;
                iu_hist.push_back((signed char)cand);
            }
            else h->t = last ? t_end : h->t + hs;
            acc_n++;
            if (h->reuse_on && h->rhs_pending >= 0) {
                h->rhs_valid = true;
                h->rhs_buf = h->rhs_pending;
                h->rhs_iu = cand;
            }
        } else {
            h->rhs_valid = false;
            rej_n++;
            if (rej_n > 100000) { status = PF_EUNSTABLE; break; }
        }
    }
    if (status == PF_OK) {
        int failed = 0;
        status = check_flag(h, &failed);
        if (status != PF_OK && !adaptive) {
            // a pass of fixed step `failed` (1-based) raised a flag and every
            // later pass did nothing: return the state after the last good
            // step, which that step's passes read but did not overwrite
            const long long good = failed > 0 ? failed - 1 : 0;
            if (good <= (long long)iu_hist.size()) {
                h->iu = good > 0 ? iu_hist[good - 1] : iu0;
                h->t = good >= nfix ? t_end : t0 + (double)good * dt;
                acc_n = good;
            }
        }
    }
    if (adaptive) h->dt_next = dt;
    if (o->trace_len) *o->trace_len = ntr;
    if (stats) {
        stats->rhs_evals = evals;
        stats->steps_accepted = acc_n;
        stats->steps_rejected = rej_n;
        stats->t = h->t;
        stats->dt_last = hlast;
        stats->err_last = elast;
        stats->dt_e = h->dte;
        stats->dt_next = h->dt_next;
        stats->kernel_launches = h->launches - launches0;
    }
    return status;
}


// An address through which kernels reach p: device and managed memory as
// is, page-locked host memory through its device mapping; null for pageable
// host memory (whose transfers go through the staging buffer).
const void *device_view(const void *p)
{
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
    if (a.type == cudaMemoryTypeHost && a.devicePointer) return a.devicePointer;
    return nullptr;
}

template <typename T>
int set_state_t(pf_handle *h, const double *phi_dev, const double *c_dev)
{
    if (h->slots) {
        if (cudaMemsetAsync(h->dflag, 0, PF_FLAG_BYTES, h->stream) != cudaSuccess) return PF_EDEVICE;
        slot_pack_dense<<<grid_for(h->V), 256, 0, h->stream>>>(phi_dev, c_dev, (float *)h->buf[h->iu], h->V,
                                                              (int)h->Vs, h->N, h->K, h->g.cref, h->dflag);
        h->launches++;
        if (cudaGetLastError() != cudaSuccess) return PF_EDEVICE;
        return check_flag(h);
    }
    pack_kernel<T><<<grid_for(h->V * h->NP), 256, 0, h->stream>>>(phi_dev, c_dev, (T *)h->buf[h->iu], h->V, h->Vs,
                                                                    h->N, h->NP, h->g.cref);
    h->launches++;
    if (h->masked) {
        mask_kernel<<<grid_for(h->V), 256, 0, h->stream>>>((const float *)h->buf[h->iu], mask_plane(h, h->buf[h->iu]),
                                                           h->V, h->Vs, h->N);
        h->launches++;
    }
    return cuda_status(cudaGetLastError());
}

template <typename T>
int get_state_t(pf_handle *h, double *phi_dev, double *c_dev)
{
    if (h->slots) {
        slot_unpack_dense<<<grid_for(h->V), 256, 0, h->stream>>>((const float *)h->buf[h->iu], phi_dev, c_dev, h->V,
                                                                (int)h->Vs, h->N, h->K, h->g.cref);
        h->launches++;
        return cuda_status(cudaGetLastError());
    }
    unpack_kernel<T><<<grid_for(h->V * h->NP), 256, 0, h->stream>>>((const T *)h->buf[h->iu], phi_dev, c_dev, h->V,
                                                                      h->Vs, h->N, h->NP, h->g.cref);
    h->launches++;
    return cuda_status(cudaGetLastError());
}

// RHS of the current state into the staging buffer (rhs true; allocated by
// the caller) and/or N_z per cell into nz_dev.
template <typename T>
int rhs_t(pf_handle *h, unsigned char *nz_dev, bool rhs)
{
    if (rhs && !h->staging) return PF_EINVAL;
    // slot passes write only the listed phases' entries
    if (rhs && h->slots &&
        cudaMemsetAsync(h->staging, 0, sizeof(double) * (size_t)h->NP * h->V, h->stream) != cudaSuccess)
        return PF_EDEVICE;
    h->cur_kind = PF_PASS_RHS;
    Pass<T> P = blank_pass<T>(h);
    P.mode = pfk::MODE_RHS;
    P.in = (const T *)h->buf[h->iu];
    P.rhs_pm = rhs ? h->staging : nullptr;
    P.nz_out = nz_dev;
    P.project = 0;
    return run_pass<T>(h, P);
}

template <typename T>
int totals_t(pf_handle *h)
{
    dim3 grid(h->tot_blocks, h->NP);
    totals_kernel<T><<<grid, 256, 0, h->stream>>>((const T *)h->buf[h->iu], h->V, h->Vs, h->tot_sum, h->tot_max);
    h->launches++;
    return cuda_status(cudaGetLastError());
}

// Device memory comes from the caller's allocator hook when one was set
// (pf_set_allocator, captured at pf_create), else from the stream-ordered
// allocator on the handle's stream: creating and destroying handles then
// does not synchronise the device, so other simulations keep running while
// one is set up or torn down.  Every allocation is recorded with its size
// and released through the same route.
template <typename P>
bool dmalloc(pf_handle *h, P **p, size_t bytes)
{
    void *q = nullptr;
    if (h->hook.alloc) {
        q = h->hook.alloc(bytes, (void *)h->stream, h->hook.ctx);
        if (!q) return false;
    } else if (cudaMallocAsync(&q, bytes, h->stream) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    h->allocs.push_back(std::make_pair(q, bytes));
    *p = static_cast<P *>(q);
    return true;
}

void dfree(pf_handle *h, void *p)
{
    if (!p) return;
    for (size_t k = 0; k < h->allocs.size(); ++k)
        if (h->allocs[k].first == p) {
            const size_t bytes = h->allocs[k].second;
            h->allocs.erase(h->allocs.begin() + k);
            if (h->hook.free) h->hook.free(p, bytes, (void *)h->stream, h->hook.ctx);
            else cudaFreeAsync(p, h->stream);
            return;
        }
}

int ensure_staging(pf_handle *h)
{
    if (h->staging) return PF_OK;
    if (!dmalloc(h, &h->staging, sizeof(double) * (size_t)h->NP * h->V)) return PF_ENOMEM;
    return PF_OK;
}

void free_all(pf_handle *h)
{
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    if (h->dl_exec) cudaGraphExecDestroy(h->dl_exec);
    if (h->dl_graph) cudaGraphDestroy(h->dl_graph);
    h->dl_exec = nullptr;
    h->dl_graph = nullptr;
    for (cudaEvent_t ev : h->ev_pool) cudaEventDestroy(ev);
    h->ev_pool.clear();
    // the stream's work must be done before a caller's allocator reuses the memory
    cudaStreamSynchronize(h->stream);
    while (!h->allocs.empty()) dfree(h, h->allocs.back().first);
    cudaStreamSynchronize(h->stream);
}

// Process-wide allocator hook for the handles created next (pf_set_allocator).
std::mutex g_hook_lock;
AllocHook g_hook;

// Process-wide autotuning results: problem shape -> kernel variant (PF_KVAR_*).
typedef std::tuple<int, int, int, int, int, int, int> TuneKey;   // prec, dim, nx, ny, nz, N, K
std::mutex g_tune_lock;
std::map<TuneKey, int> g_tune;

TuneKey tune_key(const pf_handle *h)
{
    return TuneKey(h->prec, h->g.dim, h->g.nx, h->g.ny, h->g.nz, h->N, h->K);
}

int tuned_choice(const pf_handle *h)
{
    std::lock_guard<std::mutex> guard(g_tune_lock);
    auto it = g_tune.find(tune_key(h));
    return it == g_tune.end() ? -1 : it->second;
}

// Kernel variant of the FP32 dense passes (PF_KVAR_*) applied to a handle.
void set_variant(pf_handle *h, int v)
{
    h->tma = h->tma_ok && v == PF_KVAR_TMA;
    h->g.kvar = v == PF_KVAR_TWO_CELL ? pfk::KVAR_TWO_CELL : pfk::KVAR_ONE_CELL;
}

int current_variant(const pf_handle *h)
{
    return h->tma ? PF_KVAR_TMA : (h->g.kvar == pfk::KVAR_TWO_CELL ? PF_KVAR_TWO_CELL : PF_KVAR_ONE_CELL);
}

// Average time of the RKL2-body pass signature on the current state with
// kernel variant v (inputs u^n for every operand, output into a work buffer;
// no state change).
double time_rkl2_pass(pf_handle *h, int v, int reps)
{
    const int keep = current_variant(h);
    set_variant(h, v);
    const int U = h->iu, W = (h->iu + 1) % NBUF;
    Pass<float> P = blank_pass<float>(h);
    P.in = (float *)h->buf[U]; P.p0 = (float *)h->buf[U]; P.p2 = (float *)h->buf[U]; P.r0in = (float *)h->buf[U];
    P.a0 = -0.5; P.a1 = 1.5; P.a2 = 0.0; P.b1 = 0.0; P.b0 = 0.0;
    P.out = (float *)h->buf[W];
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double ms = -1.0;
    bool ok = true;
    for (int r = 0; r < 2 && ok; ++r) ok = run_pass<float>(h, P) == PF_OK;
    cudaEventRecord(e0, h->stream);
    for (int r = 0; r < reps && ok; ++r) ok = run_pass<float>(h, P) == PF_OK;
    cudaEventRecord(e1, h->stream);
    if (ok && cudaEventSynchronize(e1) == cudaSuccess) {
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        ms = t / reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaMemsetAsync(h->dflag, 0, PF_FLAG_BYTES, h->stream);
    set_variant(h, keep);
    return ms;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

const char *pf_strerror(int s)
{
    switch (s) {
    case PF_OK: return "ok";
    case PF_EINVAL: return "invalid argument";
    case PF_ENOMEM: return "out of memory";
    case PF_EUNSTABLE: return "unstable (non-finite error norm, bad simplex sum or too many rejections)";
    case PF_ETIMEOUT: return "device wait timed out";
    case PF_EDEVICE: return "CUDA error";
    case PF_ESTATE: return "no state set";
    default: return "unknown status";
    }
}

int pf_create(const pf_params *p, void *cuda_stream, pf_handle **out)
{
    if (!p || !out) return PF_EINVAL;
    *out = nullptr;
    if (p->dim != 2 && p->dim != 3) return PF_EINVAL;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || (p->dim == 2 && p->nz != 1)) return PF_EINVAL;
    if (!(p->dx > 0.0) || !(p->W > 0.0)) return PF_EINVAL;
    if (!isfinite(p->c_ref)) return PF_EINVAL;
    if (p->n_phases < 2 || !p->phase_type || !p->gamma || (!p->mobility && !p->L_override)) return PF_EINVAL;
    if (p->has_conc != 0 && p->has_conc != 1) return PF_EINVAL;
    if (p->precision != 32 && p->precision != 64) return PF_EINVAL;
    const int NP = p->n_phases + p->has_conc;
    const bool slots = (p->options & PF_OPT_SLOTS) != 0;
    if (slots ? p->n_phases > pfk::SLOT_MAXN : NP > 128) return PF_EINVAL;
    if (slots && (p->precision != 32 || (p->options & (PF_OPT_MASKED | PF_OPT_MOBILITY_SIMPLEX)))) return PF_EINVAL;
    for (int f = 0; f < 6; ++f) {
        if (f >= 2 * p->dim) break;
        const int o = f ^ 1;
        if (p->bc_phi[f] != PF_BC_PERIODIC && p->bc_phi[f] != PF_BC_NEUMANN) return PF_EINVAL;
        if (p->bc_c[f] < 0 || p->bc_c[f] > 2) return PF_EINVAL;
        const bool per = p->bc_phi[f] == PF_BC_PERIODIC;
        if (per != (p->bc_phi[o] == PF_BC_PERIODIC)) return PF_EINVAL;
        if (p->has_conc && per != (p->bc_c[f] == PF_BC_PERIODIC)) return PF_EINVAL;
    }
    for (int a = 0; a < p->n_phases; ++a)
        if (p->phase_type[a] != 0 && p->phase_type[a] != 1) return PF_EINVAL;
    if (p->has_conc)
        for (int t = 0; t < 2; ++t) if (!(p->k[t] > 0.0)) return PF_EINVAL;

    pf_handle *h = new (std::nothrow) pf_handle();
    if (!h) return PF_ENOMEM;
    if (cudaGetDevice(&h->dev) != cudaSuccess) { delete h; return PF_EDEVICE; }
    {
        std::lock_guard<std::mutex> guard(g_hook_lock);
        h->hook = g_hook;
    }
    pf_footprint(p, &h->footprint);
    h->stream = (cudaStream_t)cuda_stream;
    h->prec = p->precision;
    h->esize = p->precision == 64 ? 8 : 4;
    const int N = p->n_phases;
    h->N = N;
    h->K = p->has_conc;
    h->NP = NP;
    h->V = (long long)p->nx * p->ny * p->nz;
    h->ptype.assign(p->phase_type, p->phase_type + N);
    h->A.resize(N * N);
    h->B.resize(N * N);
    h->L.resize(N * N);
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            const double g = p->gamma[a * N + b];
            // Sec. 2: A = 4 W gamma / pi, B = 4 gamma / (pi W), L = pi M / (4 W)
            h->A[a * N + b] = 4.0 * p->W * g / kPi;
            h->B[a * N + b] = 4.0 * g / (kPi * p->W);
            h->L[a * N + b] = p->L_override ? p->L_override[a * N + b] : kPi * p->mobility[a * N + b] / (4.0 * p->W);
        }
    Geom &g = h->g;
    g.nx = p->nx; g.ny = p->ny; g.nz = p->nz; g.dim = p->dim;
    h->Vs = (h->V + 63) / 64 * 64;
    g.V = h->V; g.Vs = h->Vs; g.N = N; g.K = h->K; g.NF = NP;
    g.tiles_x = (p->nx + pfk::TX - 1) / pfk::TX;
    g.tiles_y = (p->ny + pfk::TY - 1) / pfk::TY;
    // FP32 storage keeps c - c_ref (pf_params.c_ref); c0 and the Dirichlet
    // values are shifted with it, which leaves mu = (c - sum phi c0) / (sum phi / k)
    // and every difference of psi unchanged
    g.cref = (h->prec == 32 && h->K) ? p->c_ref : 0.0;
    g.simplex = (p->options & PF_OPT_MOBILITY_SIMPLEX) ? pfk::SIMPLEX_MOBILITY : pfk::SIMPLEX_STANDARD;
    g.slots = slots ? 1 : 0;
    h->slots = slots;
    // slot passes index a slot plane with 32-bit offsets
    if (slots && (long long)pfk::NSLOT * h->Vs >= 0x7fffffffLL) { delete h; return PF_EINVAL; }
    for (int f = 0; f < 6; ++f) {
        g.bc_phi[f] = p->bc_phi[f];
        g.bc_c[f] = p->bc_c[f];
        g.cdir[f] = p->c_dirichlet[f] - g.cref;
    }
    g.dx2 = p->dx * p->dx;
    h->dx = p->dx;
    for (int t = 0; t < 2; ++t) {
        const double k = h->K ? p->k[t] : 1.0;
        g.k[t] = k;
        g.c0[t] = p->c0[t] - g.cref;
        g.invk[t] = 1.0 / k;
        g.Dk[t] = p->D[t] / k;
    }
    h->dte = gershgorin_dt_e(h, p);

    int st = PF_OK;
    int bps = (h->prec == 64) ? pfk::prepare_stage<double>() : pfk::prepare_stage<float>();
    if (bps <= 0) { delete h; return PF_EINVAL; }
    if ((long long)g.tiles_x * g.tiles_y * p->nz > 0x7fffffffLL || p->nz > 65535) { delete h; return PF_EINVAL; }
    // error partials: one per block of the largest tiling an error pass may use
    h->grid = (int)std::max((long long)g.tiles_x * g.tiles_y, pfk::vec_tiles(g)) * p->nz;
    h->tot_blocks = (int)((h->V + 4095) / 4096 < 1024 ? (h->V + 4095) / 4096 : 1024);
    if (h->tot_blocks < 1) h->tot_blocks = 1;

    if (p->options & PF_OPT_MASKED) {
        // masked storage: FP32, one occupancy word per 32 phases and cell
        if (p->precision != 32 || p->n_phases > 128 || g.simplex != pfk::SIMPLEX_STANDARD) {
            delete h;
            return PF_EINVAL;
        }
        h->masked = true;
        h->nw = (p->n_phases + 31) / 32;
    }
    h->vec_bytes = slots ? sizeof(float) * (size_t)h->Vs * pfk::slot_planes(h->K)
                         : (size_t)h->Vs * NP * h->esize + sizeof(unsigned) * (size_t)h->Vs * h->nw;
    bool ok = true;
    for (int k = 0; k < NBUF && ok; ++k) ok = dmalloc(h, &h->buf[k], h->vec_bytes);
    ok = ok && dmalloc(h, &h->dA, h->esize * N * N);
    ok = ok && dmalloc(h, &h->dB, h->esize * N * N);
    ok = ok && dmalloc(h, &h->dL, h->esize * N * N);
    ok = ok && dmalloc(h, &h->dptype, N);
    if (!slots) ok = ok && dmalloc(h, &h->dAB64, sizeof(double) * 2 * N * N);   // energy (dense storage)
    ok = ok && dmalloc(h, &h->part_sum, sizeof(double) * h->grid);
    ok = ok && dmalloc(h, &h->part_cnt, sizeof(long long) * h->grid);
    ok = ok && dmalloc(h, &h->dres, sizeof(double));
    ok = ok && dmalloc(h, &h->dcnt, sizeof(long long));
    ok = ok && dmalloc(h, &h->dflag, PF_FLAG_BYTES);
    ok = ok && dmalloc(h, &h->dpartn, sizeof(int));
    if (h->prec == 32)   // two entries of bookkeeping + one entry (block, 256-bit mask) per block
        ok = ok && dmalloc(h, &h->dcrowd, sizeof(int) * (2 + (size_t)h->grid * (1 + pfk::VCELLS / 32)));
    ok = ok && dmalloc(h, &h->tot_sum, sizeof(double) * h->tot_blocks * NP);
    ok = ok && dmalloc(h, &h->tot_max, sizeof(double) * h->tot_blocks * NP);
    if (!ok) { cudaGetLastError(); free_all(h); delete h; return PF_ENOMEM; }
    // coefficient tables in the storage precision
    std::vector<signed char> pt(N);
    for (int a = 0; a < N; ++a) pt[a] = (signed char)h->ptype[a];
    std::vector<float> fa(h->A.begin(), h->A.end()), fb(h->B.begin(), h->B.end()), fl(h->L.begin(), h->L.end());
    if (slots && N >= 2) {
        // one value off the diagonal of every table (grain growth with equal
        // gamma and M): the slot passes read it from the constants, which is
        // the same FP32 value (same bits) the gather would return
        bool same = true;
        for (int a = 0; a < N && same; ++a)
            for (int b = 0; b < N && same; ++b)
                if (a != b)
                    same = memcmp(&fa[a * N + b], &fa[1], sizeof(float)) == 0 &&
                           memcmp(&fb[a * N + b], &fb[1], sizeof(float)) == 0 &&
                           memcmp(&fl[a * N + b], &fl[1], sizeof(float)) == 0;
        h->g.uni = same ? 1 : 0;
        h->g.uA = fa[1];
        h->g.uB = fb[1];
        h->g.uL = fl[1];
    }
    const void *ta = h->prec == 64 ? (const void *)h->A.data() : (const void *)fa.data();
    const void *tb = h->prec == 64 ? (const void *)h->B.data() : (const void *)fb.data();
    const void *tl = h->prec == 64 ? (const void *)h->L.data() : (const void *)fl.data();
    st |= cudaMemcpyAsync(h->dA, ta, h->esize * N * N, cudaMemcpyHostToDevice, h->stream);
    st |= cudaMemcpyAsync(h->dB, tb, h->esize * N * N, cudaMemcpyHostToDevice, h->stream);
    st |= cudaMemcpyAsync(h->dL, tl, h->esize * N * N, cudaMemcpyHostToDevice, h->stream);
    st |= cudaMemcpyAsync(h->dptype, pt.data(), N, cudaMemcpyHostToDevice, h->stream);
    if (h->dAB64) {
        st |= cudaMemcpyAsync(h->dAB64, h->A.data(), sizeof(double) * N * N, cudaMemcpyHostToDevice, h->stream);
        st |= cudaMemcpyAsync(h->dAB64 + (size_t)N * N, h->B.data(), sizeof(double) * N * N, cudaMemcpyHostToDevice,
                              h->stream);
    }
    st |= cudaMemsetAsync(h->dflag, 0, PF_FLAG_BYTES, h->stream);
    if (h->dcrowd) st |= cudaMemsetAsync(h->dcrowd, 0, 2 * sizeof(int), h->stream);
    if (h->masked)
        for (int k = 0; k < NBUF; ++k)
            st |= cudaMemsetAsync(mask_plane(h, h->buf[k]), 0xff, sizeof(unsigned) * (size_t)h->Vs * h->nw,
                                  h->stream);
    st |= cudaStreamSynchronize(h->stream);
    if (st != 0) { free_all(h); delete h; return PF_EDEVICE; }
    // TMA-staged FP32 kernels: full 32 x 8 tiles, 3D, 5..32 phases
    if (h->prec == 32 && !h->masked && !slots && p->dim == 3 && N > 4 && N <= 32 && p->nx % pfk::TX == 0 &&
        p->ny % pfk::TY == 0 &&
        p->nz >= 3 && h->Vs < 0x7fffffffLL) {
        bool ok = true;
        for (int k = 0; k < NBUF && ok; ++k)
            ok = make_map(&h->m3[k], h->buf[k], g, 3) && make_map(&h->m1[k], h->buf[k], g, 1);
        h->tma_ok = ok;
    }
    // kernel variant: forced by an option, else a tuned choice for this shape,
    // else the two-cell kernel (the one-cell kernel where it does not apply)
    int variant = PF_KVAR_TWO_CELL;
    if (p->options & PF_OPT_ONE_CELL) variant = PF_KVAR_ONE_CELL;
    else if ((p->options & PF_OPT_TMA) && h->tma_ok) variant = PF_KVAR_TMA;
    else if (h->prec == 32) {
        const int tuned = tuned_choice(h);
        if (tuned >= 0 && (tuned != PF_KVAR_TMA || h->tma_ok)) variant = tuned;
    }
    set_variant(h, variant);
    *out = h;
    return PF_OK;
}

int pf_footprint(const pf_params *p, long long *bytes)
{
    if (!p || !bytes) return PF_EINVAL;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->n_phases < 2 || (p->precision != 32 && p->precision != 64))
        return PF_EINVAL;
    const long long V = (long long)p->nx * p->ny * p->nz;
    const long long Vs = (V + 63) / 64 * 64;
    const long long NF = p->n_phases + (p->has_conc ? 1 : 0);
    const long long es = p->precision == 64 ? 8 : 4;
    const long long vt = (long long)((p->nx + 2 * pfk::VTX - 1) / (2 * pfk::VTX)) * ((p->ny + pfk::VTY - 1) / pfk::VTY);
    const long long tiles = std::max((long long)((p->nx + pfk::TX - 1) / pfk::TX) * ((p->ny + pfk::TY - 1) / pfk::TY), vt) *
                            p->nz;
    const long long tot_blocks = (V + 4095) / 4096 < 1024 ? ((V + 4095) / 4096 > 0 ? (V + 4095) / 4096 : 1) : 1024;
    const bool slots = (p->options & PF_OPT_SLOTS) != 0;
    long long b = slots ? (long long)NBUF * pfk::slot_planes(p->has_conc ? 1 : 0) * Vs * 4   // slot vectors
                        : (long long)NBUF * NF * Vs * es;                                    // state vectors
    if (p->options & PF_OPT_MASKED) b += (long long)NBUF * ((p->n_phases + 31) / 32) * Vs * 4;   // occupancy words
    if (!slots) b += NF * V * 8;                           // ABI staging buffer (allocated on first set/get)
    b += 3LL * p->n_phases * p->n_phases * es + p->n_phases;   // coefficient tables, phase types
    if (!slots) b += 2LL * p->n_phases * p->n_phases * 8;  // FP64 A and B for the energy functional
    b += tiles * 16 + 2 * tot_blocks * NF * 8 + 64;       // reduction partials
    if (p->precision == 32) b += 4 * (2 + tiles * (1 + pfk::VCELLS / 32));   // crowded-cell record
    *bytes = b;
    return PF_OK;
}

int pf_destroy(pf_handle *h)
{
    if (!h) return PF_OK;
    if (h->in_batch) return PF_EINVAL;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return PF_OK;
}

int pf_selftest_wait(void *cuda_stream, unsigned polls)
{
    if (polls == 0 || polls > pfk::TMA_SPIN) return PF_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int *d = nullptr;
    if (cudaMallocAsync((void **)&d, sizeof(int), s) != cudaSuccess) return PF_ENOMEM;
    int hflag = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        wait_selftest_kernel<<<1, 32, 0, s>>>(d, polls);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, d, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(d, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || e != cudaSuccess) return PF_EDEVICE;
    return (hflag & pfk::FLAG_TIMEOUT) ? PF_ETIMEOUT : PF_OK;
}

int pf_get_controller(pf_handle *h, pf_controller *out)
{
    if (!h || !out) return PF_EINVAL;
    out->b = h->b;
    out->E1 = h->E1;
    out->E2 = h->E2;
    out->dt1 = h->dt1;
    out->dt2 = h->dt2;
    out->dt_next = h->dt_next;
    out->nhist = h->nhist;
    return PF_OK;
}

int pf_set_controller(pf_handle *h, const pf_controller *in)
{
    if (!h || !in) return PF_EINVAL;
    if (!h->has_state) return PF_ESTATE;
    const double v[] = {in->b, in->E1, in->E2, in->dt1, in->dt2, in->dt_next};
    for (double x : v)
        if (!isfinite(x) || x < 0.0) return PF_EINVAL;
    if (in->b < 0.1 || in->b > 0.98 || in->nhist < 0 || in->nhist > 2) return PF_EINVAL;
    h->b = in->b;
    h->E1 = in->E1;
    h->E2 = in->E2;
    h->dt1 = in->dt1;
    h->dt2 = in->dt2;
    h->dt_next = in->dt_next;
    h->nhist = in->nhist;
    return PF_OK;
}

int pf_dt_e(pf_handle *h, double *dte)
{
    if (!h || !dte) return PF_EINVAL;
    *dte = h->dte;
    return PF_OK;
}

int pf_set_state(pf_handle *h, const double *phi, const double *c, double t, int ptr_is_device)
{
    if (!h || !phi || (h->K && !c) || h->in_batch) return PF_EINVAL;
    int st;
    const double *vphi = (const double *)device_view(phi), *vc = h->K ? (const double *)device_view(c) : nullptr;
    if (vphi && (!h->K || vc)) {
        // device or page-locked host memory: the layout conversion reads it directly
        st = (h->prec == 64) ? set_state_t<double>(h, vphi, vc) : set_state_t<float>(h, vphi, vc);
        if (st) return st;
    } else {
        if ((st = ensure_staging(h))) return st;
        const size_t nphi = sizeof(double) * (size_t)h->N * h->V;
        const cudaMemcpyKind kind = ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        double *sc = h->staging + (size_t)h->N * h->V;
        if (cudaMemcpyAsync(h->staging, phi, nphi, kind, h->stream) != cudaSuccess) return PF_EDEVICE;
        if (h->K && cudaMemcpyAsync(sc, c, sizeof(double) * h->V, kind, h->stream) != cudaSuccess) return PF_EDEVICE;
        st = (h->prec == 64) ? set_state_t<double>(h, h->staging, sc) : set_state_t<float>(h, h->staging, sc);
        if (st) return st;
    }
    if (!ptr_is_device && cudaStreamSynchronize(h->stream) != cudaSuccess) return PF_EDEVICE;
    h->t = t;
    h->has_state = true;
    h->rhs_valid = false;
    reset_controller(h);
    return PF_OK;
}

int pf_set_state_slots(pf_handle *h, const double *vals, const int *ids, int n_in, const double *c, double t,
                       int ptr_is_device)
{
    if (!h || !h->slots || !vals || !ids || n_in < 1 || (h->K && !c) || h->in_batch) return PF_EINVAL;
    const double *dv = (const double *)device_view(vals), *dc = h->K ? (const double *)device_view(c) : nullptr;
    const int *di = (const int *)device_view(ids);
    std::vector<void *> tmp;
    auto stage = [&](const void *src, size_t bytes) -> const void * {
        void *q = nullptr;
        if (!dmalloc(h, &q, bytes)) return nullptr;
        tmp.push_back(q);
        if (cudaMemcpyAsync(q, src, bytes, ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            h->stream) != cudaSuccess)
            return nullptr;
        return q;
    };
    int st = PF_OK;
    // pageable host memory goes through temporary device copies
    if (!dv) dv = (const double *)stage(vals, sizeof(double) * (size_t)n_in * h->V);
    if (!di) di = (const int *)stage(ids, sizeof(int) * (size_t)n_in * h->V);
    if (h->K && !dc) dc = (const double *)stage(c, sizeof(double) * (size_t)h->V);
    if (!dv || !di || (h->K && !dc)) st = PF_ENOMEM;
    if (!st && cudaMemsetAsync(h->dflag, 0, PF_FLAG_BYTES, h->stream) != cudaSuccess) st = PF_EDEVICE;
    if (!st) {
        slot_pack_slots<<<grid_for(h->V), 256, 0, h->stream>>>(dv, di, n_in, dc, (float *)h->buf[h->iu], h->V,
                                                              (int)h->Vs, h->N, h->K, h->g.cref, h->dflag);
        h->launches++;
        st = cudaGetLastError() == cudaSuccess ? check_flag(h) : PF_EDEVICE;
    }
    cudaStreamSynchronize(h->stream);
    for (void *q : tmp) dfree(h, q);
    if (st) return st;
    h->t = t;
    h->has_state = true;
    h->rhs_valid = false;
    reset_controller(h);
    return PF_OK;
}

int pf_get_state_slots(pf_handle *h, double *vals, int *ids, double *c, double *t, int ptr_is_device)
{
    if (!h || !h->slots || !vals || !ids) return PF_EINVAL;
    if (!h->has_state) return PF_ESTATE;
    double *dv = (double *)device_view(vals), *dc = (c && h->K) ? (double *)device_view(c) : nullptr;
    int *di = (int *)device_view(ids);
    const size_t nv = sizeof(double) * (size_t)pfk::NSLOT * h->V, ni = sizeof(int) * (size_t)pfk::NSLOT * h->V;
    double *tv = nullptr, *tc = nullptr;
    int *ti = nullptr;
    int st = PF_OK;
    if (!dv && !dmalloc(h, &tv, nv)) st = PF_ENOMEM;
    if (!st && !di && !dmalloc(h, &ti, ni)) st = PF_ENOMEM;
    if (!st && c && h->K && !dc && !dmalloc(h, &tc, sizeof(double) * h->V)) st = PF_ENOMEM;
    if (!st) {
        slot_unpack_slots<<<grid_for(h->V), 256, 0, h->stream>>>((const float *)h->buf[h->iu], dv ? dv : tv,
                                                                di ? di : ti, (c && h->K) ? (dc ? dc : tc) : nullptr,
                                                                h->V, (int)h->Vs, h->N, h->K, h->g.cref);
        h->launches++;
        if (cudaGetLastError() != cudaSuccess) st = PF_EDEVICE;
    }
    const cudaMemcpyKind kind = ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (!st && tv && cudaMemcpyAsync(vals, tv, nv, kind, h->stream) != cudaSuccess) st = PF_EDEVICE;
    if (!st && ti && cudaMemcpyAsync(ids, ti, ni, kind, h->stream) != cudaSuccess) st = PF_EDEVICE;
    if (!st && tc && cudaMemcpyAsync(c, tc, sizeof(double) * h->V, kind, h->stream) != cudaSuccess) st = PF_EDEVICE;
    if (t) *t = h->t;
    if ((tv || ti || tc || !ptr_is_device) && cudaStreamSynchronize(h->stream) != cudaSuccess && !st) st = PF_EDEVICE;
    if (tv) dfree(h, tv);
    if (ti) dfree(h, ti);
    if (tc) dfree(h, tc);
    return st;
}

int pf_get_state(pf_handle *h, double *phi, double *c, unsigned char *nz, double *t, int ptr_is_device)
{
    if (!h) return PF_EINVAL;
    if (!h->has_state) return PF_ESTATE;
    int st;
    const cudaMemcpyKind kind = ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    double *vphi = phi ? (double *)device_view(phi) : nullptr;
    double *vc = (c && h->K) ? (double *)device_view(c) : nullptr;
    if (phi && vphi && (!c || !h->K || vc)) {
        // device or page-locked host memory: the layout conversion writes it directly
        st = (h->prec == 64) ? get_state_t<double>(h, vphi, vc) : get_state_t<float>(h, vphi, vc);
        if (st) return st;
    } else if (phi || c) {
        if ((st = ensure_staging(h))) return st;
        double *sc = h->staging + (size_t)h->N * h->V;
        st = (h->prec == 64) ? get_state_t<double>(h, h->staging, sc) : get_state_t<float>(h, h->staging, sc);
        if (st) return st;
        if (phi && cudaMemcpyAsync(phi, h->staging, sizeof(double) * (size_t)h->N * h->V, kind, h->stream) != cudaSuccess)
            return PF_EDEVICE;
        if (c && h->K && cudaMemcpyAsync(c, sc, sizeof(double) * h->V, kind, h->stream) != cudaSuccess)
            return PF_EDEVICE;
    }
    if (nz) {
        if (!h->dnz && !dmalloc(h, &h->dnz, h->V)) return PF_ENOMEM;
        // N_z only: the RHS values are not stored
        st = (h->prec == 64) ? rhs_t<double>(h, h->dnz, false) : rhs_t<float>(h, h->dnz, false);
        if (st) return st;
        if (cudaMemcpyAsync(nz, h->dnz, h->V, kind, h->stream) != cudaSuccess) return PF_EDEVICE;
    }
    if (t) *t = h->t;
    if (!ptr_is_device && cudaStreamSynchronize(h->stream) != cudaSuccess) return PF_EDEVICE;
    return PF_OK;
}

int pf_rhs(pf_handle *h, double *rhs_phi, double *rhs_c, unsigned char *nz, int ptr_is_device)
{
    if (!h || !rhs_phi) return PF_EINVAL;
    if (!h->has_state) return PF_ESTATE;
    int st;
    if ((st = ensure_staging(h))) return st;
    if (nz && !h->dnz && !dmalloc(h, &h->dnz, h->V)) return PF_ENOMEM;
    if (cudaMemsetAsync(h->dflag, 0, PF_FLAG_BYTES, h->stream) != cudaSuccess) return PF_EDEVICE;
    st = (h->prec == 64) ? rhs_t<double>(h, nz ? h->dnz : nullptr, true)
                         : rhs_t<float>(h, nz ? h->dnz : nullptr, true);
    if (st) return st;
    const cudaMemcpyKind kind = ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (cudaMemcpyAsync(rhs_phi, h->staging, sizeof(double) * (size_t)h->N * h->V, kind, h->stream) != cudaSuccess)
        return PF_EDEVICE;
    if (rhs_c && h->K &&
        cudaMemcpyAsync(rhs_c, h->staging + (size_t)h->N * h->V, sizeof(double) * h->V, kind, h->stream) != cudaSuccess)
        return PF_EDEVICE;
    if (nz && cudaMemcpyAsync(nz, h->dnz, h->V, kind, h->stream) != cudaSuccess) return PF_EDEVICE;
    return check_flag(h);
}

int pf_step(pf_handle *h, pf_integrator integ, double t_end, const pf_tol *tol, const pf_step_opts *opts,
            pf_stats *stats)
{
    if (!h || h->in_batch) return PF_EINVAL;
    if (!h->has_state) return PF_ESTATE;
    if ((int)integ < PF_FEULER || (int)integ > PF_RKL2) return PF_EINVAL;
    if (!(t_end >= h->t)) return PF_EINVAL;
    pf_step_opts o;
    memset(&o, 0, sizeof(o));
    o.ssp_stages = 5;
    if (opts) o = *opts;
    return (h->prec == 64) ? step_loop<double>(h, integ, t_end, tol, &o, stats)
                           : step_loop<float>(h, integ, t_end, tol, &o, stats);
}

int pf_profile(pf_handle *h, int enable, double *ms, long long *launches)
{
    if (!h) return PF_EINVAL;
    if (enable && h->ev_pool.empty()) {
        const int cap = 4096;
        h->ev_pool.resize(2 * cap);
        h->ev_kind.resize(cap);
        for (auto &ev : h->ev_pool)
            if (cudaEventCreate(&ev) != cudaSuccess) return PF_EDEVICE;
    }
    int st = prof_flush(h);
    if (st) return st;
    if (ms)
        for (int k = 0; k < PF_NPASS_KINDS; ++k) ms[k] = h->prof_ms[k];
    if (launches)
        for (int k = 0; k < PF_NPASS_KINDS; ++k) launches[k] = h->prof_n[k];
    if (enable >= 0) {
        for (int k = 0; k < PF_NPASS_KINDS; ++k) { h->prof_ms[k] = 0.0; h->prof_n[k] = 0; }
        h->prof_on = enable != 0;
    }
    return PF_OK;
}

long long pf_launch_count(pf_handle *h) { return h ? h->launches : -1; }

int pf_autotune(pf_handle *h, int *choice, double *ms)
{
    if (!h) return PF_EINVAL;
    if (!h->has_state) return PF_ESTATE;
    if (ms)
        for (int v = 0; v < PF_KVAR_COUNT; ++v) ms[v] = -1.0;
    int c = current_variant(h);
    if (h->prec == 32 && !h->masked && !h->slots) {
        const bool ok[PF_KVAR_COUNT] = {pfk::vec_eligible(h->g), true, h->tma_ok};
        double best = -1.0;
        for (int v = 0; v < PF_KVAR_COUNT; ++v) {
            if (!ok[v]) continue;
            const double t = time_rkl2_pass(h, v, 5);
            if (t < 0.0) return PF_EDEVICE;
            if (ms) ms[v] = t;
            if (best < 0.0 || t < best) { best = t; c = v; }
        }
        std::lock_guard<std::mutex> guard(g_tune_lock);
        g_tune[tune_key(h)] = c;
    }
    set_variant(h, c);
    if (choice) *choice = c;
    return check_flag(h);
}

// pf_reduce on slot storage: per-phase sums and maxima by atomics over the
// slots (N doubles each), the concentration by the fixed-order partials.
int reduce_slots(pf_handle *h, double *mass_c, double *vol_phi, int *grains_alive)
{
    const int N = h->N;
    double *vol = h->tot_sum;
    unsigned long long *mx = reinterpret_cast<unsigned long long *>(h->tot_max);
    double *cs = h->tot_sum + N, *cm = h->tot_max + N;      // N + tot_blocks <= tot_blocks * NP
    if (cudaMemsetAsync(vol, 0, sizeof(double) * N, h->stream) != cudaSuccess) return PF_EDEVICE;
    if (cudaMemsetAsync(mx, 0, sizeof(double) * N, h->stream) != cudaSuccess) return PF_EDEVICE;
    const float *u = (const float *)h->buf[h->iu];
    slot_phase_totals<<<grid_for(h->V), 256, 0, h->stream>>>(u, h->V, (int)h->Vs, N, vol, mx);
    h->launches++;
    if (h->K) {
        dim3 grid(h->tot_blocks, 1);
        totals_kernel<float><<<grid, 256, 0, h->stream>>>(u + (size_t)pfk::SLOT_C_PLANES * h->Vs, h->V, h->Vs, cs, cm);
        h->launches++;
    }
    if (cudaGetLastError() != cudaSuccess) return PF_EDEVICE;
    std::vector<double> v(N), c(h->tot_blocks);
    std::vector<unsigned long long> m(N);
    if (cudaMemcpyAsync(v.data(), vol, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return PF_EDEVICE;
    if (cudaMemcpyAsync(m.data(), mx, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return PF_EDEVICE;
    if (h->K && cudaMemcpyAsync(c.data(), cs, sizeof(double) * h->tot_blocks, cudaMemcpyDeviceToHost, h->stream) !=
                    cudaSuccess)
        return PF_EDEVICE;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return PF_EDEVICE;
    const double dv = pow(h->dx, h->g.dim);
    int alive = 0;
    for (int a = 0; a < N; ++a) {
        if (vol_phi) vol_phi[a] = v[a] * dv;
        double mv;
        memcpy(&mv, &m[a], sizeof(double));
        if (mv >= 0.5) alive++;
    }
    if (mass_c) {
        double tot = 0.0;
        for (int b = 0; b < h->tot_blocks; ++b) tot += c[b];
        *mass_c = h->K ? (tot + (double)h->V * h->g.cref) * dv : 0.0;
    }
    if (grains_alive) *grains_alive = alive;
    return PF_OK;
}

int pf_reduce(pf_handle *h, double *mass_c, double *vol_phi, int *grains_alive)
{
    if (!h) return PF_EINVAL;
    if (!h->has_state) return PF_ESTATE;
    if (h->slots) return reduce_slots(h, mass_c, vol_phi, grains_alive);
    int st = (h->prec == 64) ? totals_t<double>(h) : totals_t<float>(h);
    if (st) return st;
    std::vector<double> s((size_t)h->tot_blocks * h->NP), m((size_t)h->tot_blocks * h->NP);
    if (cudaMemcpyAsync(s.data(), h->tot_sum, sizeof(double) * s.size(), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return PF_EDEVICE;
    if (cudaMemcpyAsync(m.data(), h->tot_max, sizeof(double) * m.size(), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return PF_EDEVICE;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return PF_EDEVICE;
    const double dv = pow(h->dx, h->g.dim);
    int alive = 0;
    for (int f = 0; f < h->NP; ++f) {
        double tot = 0.0, mx = -1e300;
        for (int b = 0; b < h->tot_blocks; ++b) {
            tot += s[(size_t)f * h->tot_blocks + b];
            mx = fmax(mx, m[(size_t)f * h->tot_blocks + b]);
        }
        if (f < h->N) {
            if (vol_phi) vol_phi[f] = tot * dv;
            if (mx >= 0.5) alive++;
        } else if (mass_c) {
            *mass_c = (tot + (double)h->V * h->g.cref) * dv;     // the state holds c - cref
        }
    }
    if (mass_c && !h->K) *mass_c = 0.0;
    if (grains_alive) *grains_alive = alive;
    return PF_OK;
}

int pf_energy(pf_handle *h, double *F)
{
    if (!h || !F || h->slots) return PF_EINVAL;
    if (!h->has_state) return PF_ESTATE;
    const long long want = (h->V + 255) / 256;
    const int nblk = (int)(want < h->grid ? want : h->grid);
    if (h->prec == 64)
        energy_kernel<double><<<nblk, 256, 0, h->stream>>>(h->g, (const double *)h->buf[h->iu], h->dAB64,
                                                          h->dAB64 + (size_t)h->N * h->N, h->dptype, h->dx,
                                                          h->part_sum, h->part_cnt);
    else
        energy_kernel<float><<<nblk, 256, 0, h->stream>>>(h->g, (const float *)h->buf[h->iu], h->dAB64,
                                                         h->dAB64 + (size_t)h->N * h->N, h->dptype, h->dx,
                                                         h->part_sum, h->part_cnt);
    h->launches++;
    finalize_err_kernel<<<1, 256, 0, h->stream>>>(h->part_sum, h->part_cnt, nblk, h->dres, h->dcnt);
    h->launches++;
    if (cudaGetLastError() != cudaSuccess) return PF_EDEVICE;
    double sum = 0.0;
    long long over = 0;
    if (cudaMemcpyAsync(&sum, h->dres, sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return PF_EDEVICE;
    if (cudaMemcpyAsync(&over, h->dcnt, sizeof(long long), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return PF_EDEVICE;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return PF_EDEVICE;
    if (over) return PF_EINVAL;
    *F = sum * pow(h->dx, h->g.dim);
    return PF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched stepping (pf_batch_*): continuous batching of many simulations on
// one stream.  Every round each running request takes one step or adaptive
// attempt; the FP32 passes of the requests that can be packed are recorded
// (do_step in collect mode) and issued wave by wave, one packed launch per
// pass kind and wave; the error partials and device flags of all requests
// are folded and read back in one transfer; the controller and the
// bookkeeping of step_loop then run per request on the host.
// ---------------------------------------------------------------------------
namespace {

struct BatchReq {
    pf_handle *h = nullptr;
    int integ = 0;
    double t_end = 0.0;
    pf_tol tol{};
    pf_step_opts o{};
    bool adaptive = false, packed = false, done = false;
    int status = PF_OK;
    double dt = 0.0, t0 = 0.0;
    long long nfix = 0, kfix = 0;
    int max_stages = 1001;
    long long acc_n = 0, rej_n = 0, evals = 0, launches = 0;
    double hlast = 0.0, elast = 0.0;
    // the attempt of the current round
    std::vector<Pass<float>> passes;
    int cand = -1, s = 1;
    double hs = 0.0;
    bool last = false;
};

// Per request: where its error partials and status words are.
struct BatchGather {
    const double *ps;
    const long long *pc;
    const int *pn;
    int cap;
    int *flag;
};

// One block per request: the error partials folded in the order of
// finalize_err_kernel (so the norm equals the single-handle one bit for
// bit), the status words read and cleared for the next round.
__global__ void batch_gather_kernel(const BatchGather *__restrict__ gs, double *out)
{
    const BatchGather G = gs[blockIdx.x];
    __shared__ double ss[256];
    __shared__ long long sc[256];
    int n = G.cap;
    if (G.pn && *G.pn < n) n = *G.pn;
    double s = 0.0;
    long long c = 0;
    for (int k = threadIdx.x; k < n; k += 256) { s += G.ps[k]; c += G.pc[k]; }
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int o = 128; o >= 1; o >>= 1) {
        if ((int)threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            sc[threadIdx.x] += sc[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double *o = out + 4 * blockIdx.x;
        o[0] = ss[0];
        o[1] = (double)sc[0];
        o[2] = (double)G.flag[0];
        o[3] = (double)G.flag[3];
        G.flag[0] = G.flag[1] = G.flag[2] = G.flag[3] = 0;
    }
}

template <typename T>
bool grow(T **dev, T **host, size_t *cap, size_t want)
{
    if (want <= *cap) return true;
    size_t c = *cap ? *cap : 64;
    while (c < want) c *= 2;
    if (*dev) cudaFree(*dev);
    if (*host) cudaFreeHost(*host);
    *dev = nullptr;
    *host = nullptr;
    *cap = 0;
    if (cudaMalloc((void **)dev, sizeof(T) * c) != cudaSuccess) { cudaGetLastError(); return false; }
    if (cudaMallocHost((void **)host, sizeof(T) * c) != cudaSuccess) { cudaGetLastError(); return false; }
    *cap = c;
    return true;
}

bool packable(const pf_handle *h, int integ)
{
    return h->prec == 32 && !h->masked && !h->slots && !h->tma && h->g.kvar == pfk::KVAR_TWO_CELL &&
           pfk::vec_eligible(h->g) && integ != PF_SSP104 && h->g.simplex == pfk::SIMPLEX_STANDARD;
}

}  // namespace

struct pf_batch {
    int dev = 0;
    cudaStream_t stream = nullptr;
    long long max_bytes = 0, used = 0;
    std::vector<BatchReq> slots;       // h == nullptr: free slot
    pfk::VecInst *dtab = nullptr, *htab = nullptr;
    size_t tcap = 0;
    int *dstart = nullptr, *hstart = nullptr;
    size_t scap = 0;
    BatchGather *dg = nullptr, *hg = nullptr;
    size_t gcap = 0;
    double *dout = nullptr, *hout = nullptr;
    size_t ocap = 0;
    int *ddone = nullptr;
};

namespace {

// Bookkeeping of step_loop after one attempt of a request (packed path).
void batch_after(BatchReq &r, int flag, double sum, double cnt)
{
    pf_handle *h = r.h;
    r.hlast = r.hs;
    if (flag) {
        r.done = true;
        r.status = flag_status(flag);
        return;
    }
    int acc = 1;
    if (r.adaptive) {
        const double err = cnt > 0.0 ? sqrt(sum / cnt) : 0.0;
        r.elast = err;
        if (!isfinite(err)) {
            r.done = true;
            r.status = PF_EUNSTABLE;
            return;
        }
        r.dt = controller(h, err, r.hs, method_order(r.integ), &acc);
        h->dt_next = r.dt;
    }
    if (acc) {
        h->iu = r.cand;
        if (!r.adaptive) {
            r.kfix++;
            h->t = r.last ? r.t_end : r.t0 + (double)r.kfix * r.dt;
        } else {
            h->t = r.last ? r.t_end : h->t + r.hs;
        }
        r.acc_n++;
    } else {
        r.rej_n++;
        if (r.rej_n > 100000) {
            r.done = true;
            r.status = PF_EUNSTABLE;
            return;
        }
    }
    if (!(h->t < r.t_end)) r.done = true;
}

int batch_round(pf_batch *b)
{
    std::vector<int> act;
    size_t npass = 0, maxw = 0;
    for (size_t k = 0; k < b->slots.size(); ++k) {
        BatchReq &r = b->slots[k];
        if (!r.h || r.done) continue;
        pf_handle *h = r.h;
        r.hs = r.dt;
        int st = plan_attempt(h, r.integ, r.adaptive, r.t_end - h->t, r.kfix, r.nfix, r.o.ssp_stages, r.max_stages,
                              &r.hs, &r.s, &r.last);
        r.passes.clear();
        if (!st) {
            const pf_tol *tol = r.adaptive ? &r.tol : nullptr;
            long long ev = 0;
            const long long l0 = h->launches;
            if (r.packed) {
                // the passes are recorded for the packed launches below
                h->collect = &r.passes;
                st = do_step<float>(h, r.integ, r.hs, r.s, tol, r.adaptive, &r.cand, &ev);
                h->collect = nullptr;
            } else {
                // launched now on the handle's stream; the batch's stream waits for them
                st = (h->prec == 64) ? do_step<double>(h, r.integ, r.hs, r.s, tol, r.adaptive, &r.cand, &ev)
                                     : do_step<float>(h, r.integ, r.hs, r.s, tol, r.adaptive, &r.cand, &ev);
                if (!st && h->stream != b->stream) {
                    cudaEvent_t e;
                    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return PF_EDEVICE;
                    cudaEventRecord(e, h->stream);
                    cudaStreamWaitEvent(b->stream, e, 0);
                    cudaEventDestroy(e);
                }
            }
            r.launches += h->launches - l0;
            r.evals += ev;
        }
        if (st) { r.done = true; r.status = st; continue; }
        npass += r.passes.size();
        maxw = std::max(maxw, r.passes.size());
        act.push_back((int)k);
    }
    if (act.empty()) return PF_OK;
    if (!grow(&b->dtab, &b->htab, &b->tcap, npass) || !grow(&b->dstart, &b->hstart, &b->scap, npass) ||
        !grow(&b->dg, &b->hg, &b->gcap, act.size()) || !grow(&b->dout, &b->hout, &b->ocap, 4 * act.size()))
        return PF_ENOMEM;
    // waves: the w-th pass of every request; one packed launch per pass kind
    struct Launch { int dim, K; unsigned sig; size_t toff; int n, blocks; };
    std::vector<Launch> launches;
    size_t toff = 0;
    for (size_t w = 0; w < maxw; ++w) {
        std::map<std::tuple<int, int, unsigned>, std::vector<int>> groups;
        for (int k : act) {
            BatchReq &r = b->slots[k];
            if (w < r.passes.size())
                groups[std::make_tuple(r.h->g.dim, r.h->K, pfk::pass_signature(r.passes[w]))].push_back(k);
        }
        for (auto &gr : groups) {
            Launch l{std::get<0>(gr.first), std::get<1>(gr.first), std::get<2>(gr.first), toff, 0, 0};
            for (int k : gr.second) {
                BatchReq &r = b->slots[k];
                pfk::VecInst &I = b->htab[toff];
                I.g = r.h->g;
                I.P = r.passes[w];
                I.A = (const float *)r.h->dA;
                I.B = (const float *)r.h->dB;
                I.L = (const float *)r.h->dL;
                I.ptype = r.h->dptype;
                I.nblk = (int)(pfk::vec_tiles(r.h->g) * r.h->g.nz);
                b->hstart[toff] = l.blocks;
                l.blocks += I.nblk;
                l.n++;
                toff++;
                r.launches += 2;
            }
            launches.push_back(l);
        }
    }
    if (cudaMemcpyAsync(b->dtab, b->htab, sizeof(pfk::VecInst) * toff, cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(b->dstart, b->hstart, sizeof(int) * toff, cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
        return PF_EDEVICE;
    for (const Launch &l : launches) {
        bool ok = false;
        const int e = pfk::launch_packed(l.dim, l.K, l.sig, b->dtab + l.toff, b->dstart + l.toff, l.n, l.blocks,
                                         b->ddone, b->stream, &ok);
        if (!ok || e != 0) return PF_EDEVICE;
    }
    // error partials and status words of every request, one transfer
    for (size_t j = 0; j < act.size(); ++j) {
        const pf_handle *h = b->slots[act[j]].h;
        b->hg[j] = BatchGather{h->part_sum, h->part_cnt, h->dpartn, h->grid, h->dflag};
    }
    if (cudaMemcpyAsync(b->dg, b->hg, sizeof(BatchGather) * act.size(), cudaMemcpyHostToDevice, b->stream) !=
        cudaSuccess)
        return PF_EDEVICE;
    batch_gather_kernel<<<(unsigned)act.size(), 256, 0, b->stream>>>(b->dg, b->dout);
    if (cudaGetLastError() != cudaSuccess) return PF_EDEVICE;
    if (cudaMemcpyAsync(b->hout, b->dout, sizeof(double) * 4 * act.size(), cudaMemcpyDeviceToHost, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return PF_EDEVICE;
    for (size_t j = 0; j < act.size(); ++j) {
        const double *o = b->hout + 4 * j;
        batch_after(b->slots[act[j]], (int)o[2], o[0], o[1]);
    }
    return PF_OK;
}

}  // namespace

extern "C" {

int pf_set_allocator(pf_alloc_fn alloc, pf_free_fn free_fn, void *ctx)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) return PF_EINVAL;
    std::lock_guard<std::mutex> guard(g_hook_lock);
    g_hook.alloc = alloc;
    g_hook.free = free_fn;
    g_hook.ctx = alloc ? ctx : nullptr;
    return PF_OK;
}

int pf_batch_create(long long max_bytes, void *cuda_stream, pf_batch **out)
{
    if (!out || max_bytes <= 0) return PF_EINVAL;
    *out = nullptr;
    pf_batch *b = new (std::nothrow) pf_batch();
    if (!b) return PF_ENOMEM;
    if (cudaGetDevice(&b->dev) != cudaSuccess) { delete b; return PF_EDEVICE; }
    b->stream = (cudaStream_t)cuda_stream;
    b->max_bytes = max_bytes;
    if (cudaMalloc((void **)&b->ddone, sizeof(int)) != cudaSuccess) { cudaGetLastError(); delete b; return PF_ENOMEM; }
    if (cudaMemsetAsync(b->ddone, 0, sizeof(int), b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaFree(b->ddone);
        delete b;
        return PF_EDEVICE;
    }
    *out = b;
    return PF_OK;
}

int pf_batch_admit(pf_batch *b, pf_handle *h, pf_integrator integ, double t_end, const pf_tol *tol,
                   const pf_step_opts *opts, int *slot)
{
    if (!b || !h || !slot) return PF_EINVAL;
    if (!h->has_state) return PF_ESTATE;
    if (h->in_batch || h->dev != b->dev) return PF_EINVAL;
    if ((int)integ < PF_FEULER || (int)integ > PF_RKL2) return PF_EINVAL;
    if (!(t_end >= h->t)) return PF_EINVAL;
    BatchReq r;
    memset(&r.o, 0, sizeof(r.o));
    r.o.ssp_stages = 5;
    if (opts) r.o = *opts;
    r.adaptive = !(r.o.dt_mult > 0.0);
    if (r.adaptive && (integ == PF_FEULER || integ == PF_SSP2)) return PF_EINVAL;
    if (r.adaptive && !tol) return PF_EINVAL;
    if (integ == PF_SSP2 && r.o.ssp_stages < 2) return PF_EINVAL;
    if (h->footprint > b->max_bytes - b->used) return PF_ENOMEM;
    r.h = h;
    r.integ = integ;
    r.t_end = t_end;
    if (tol) r.tol = *tol;
    r.max_stages = r.o.max_stages > 0 ? r.o.max_stages : 1001;
    r.packed = packable(h, integ);
    if (r.adaptive) {
        r.dt = h->dt_next > 0.0 ? h->dt_next : (r.o.dt0 > 0.0 ? r.o.dt0 : 0.9 * h->dte);
    } else {
        r.dt = r.o.dt_mult * h->dte;
        r.t0 = h->t;
        r.nfix = (long long)ceil((t_end - r.t0) / r.dt - 1e-9);
        if (r.nfix < 1) r.nfix = 1;
    }
    {
        // the batch's stream waits for the handle's earlier work
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return PF_EDEVICE;
        cudaError_t e = cudaEventRecord(ev, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, ev, 0);
        cudaEventDestroy(ev);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->dflag, 0, PF_FLAG_BYTES, b->stream);
        if (e != cudaSuccess) return PF_EDEVICE;
        h->reuse_on = false;
        h->rhs_valid = false;
    }
    if (!(h->t < t_end)) r.done = true;
    h->in_batch = true;
    b->used += h->footprint;
    int k = 0;
    while (k < (int)b->slots.size() && b->slots[k].h) ++k;
    if (k == (int)b->slots.size()) b->slots.emplace_back();
    b->slots[k] = r;
    *slot = k;
    return PF_OK;
}

int pf_batch_run(pf_batch *b, int rounds, int *n_active)
{
    if (!b || rounds < 1) return PF_EINVAL;
    for (int i = 0; i < rounds; ++i) {
        bool any = false;
        for (const BatchReq &r : b->slots) any = any || (r.h && !r.done);
        if (!any) break;
        const int st = batch_round(b);
        if (st) return st;
    }
    if (n_active) {
        int n = 0;
        for (const BatchReq &r : b->slots) n += (r.h && !r.done) ? 1 : 0;
        *n_active = n;
    }
    return PF_OK;
}

int pf_batch_result(pf_batch *b, int slot, int *done, int *status, pf_stats *stats)
{
    if (!b || !done || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].h) return PF_EINVAL;
    BatchReq &r = b->slots[slot];
    *done = r.done ? 1 : 0;
    if (!r.done) return PF_OK;
    pf_handle *h = r.h;
    if (status) *status = r.status;
    if (stats) {
        stats->rhs_evals = r.evals;
        stats->steps_accepted = r.acc_n;
        stats->steps_rejected = r.rej_n;
        stats->t = h->t;
        stats->dt_last = r.hlast;
        stats->err_last = r.elast;
        stats->dt_e = h->dte;
        stats->dt_next = r.adaptive ? h->dt_next : 0.0;
        stats->kernel_launches = r.launches;
    }
    // the handle's stream is ordered after the batch's work on it
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(ev, b->stream);
        cudaStreamWaitEvent(h->stream, ev, 0);
        cudaEventDestroy(ev);
    }
    h->in_batch = false;
    b->used -= h->footprint;
    r = BatchReq();
    return PF_OK;
}

int pf_batch_destroy(pf_batch *b)
{
    if (!b) return PF_OK;
    cudaStreamSynchronize(b->stream);
    for (BatchReq &r : b->slots)
        if (r.h) r.h->in_batch = false;
    if (b->dtab) cudaFree(b->dtab);
    if (b->htab) cudaFreeHost(b->htab);
    if (b->dstart) cudaFree(b->dstart);
    if (b->hstart) cudaFreeHost(b->hstart);
    if (b->dg) cudaFree(b->dg);
    if (b->hg) cudaFreeHost(b->hg);
    if (b->dout) cudaFree(b->dout);
    if (b->hout) cudaFreeHost(b->hout);
    if (b->ddone) cudaFree(b->ddone);
    delete b;
    return PF_OK;
}

}  // extern "C"
