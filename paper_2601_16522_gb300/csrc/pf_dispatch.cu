// pf_dispatch.cu -- picks the instantiation for a pass (see pf_stage_*.cu).
#include "pf_internal.h"

namespace pfk {

int launch_f64(const Geom &, const Pass<double> &, unsigned, cudaStream_t, const double *, const double *,
               const double *, const signed char *, const TmaMaps *, bool *);
int launch_f32k0(const Geom &, const Pass<float> &, unsigned, cudaStream_t, const float *, const float *,
                 const float *, const signed char *, const TmaMaps *, bool *);
int launch_f32k1(const Geom &, const Pass<float> &, unsigned, cudaStream_t, const float *, const float *,
                 const float *, const signed char *, const TmaMaps *, bool *);
int launch_m32k0(const Geom &, const Pass<float> &, unsigned, cudaStream_t, const float *, const float *,
                 const float *, const signed char *, bool *);
int launch_m32k1(const Geom &, const Pass<float> &, unsigned, cudaStream_t, const float *, const float *,
                 const float *, const signed char *, bool *);
int launchd_f64(const Geom &, unsigned, const Pass<double> *, cudaStream_t, const double *, const double *,
                const double *, const signed char *);
int launchd_f32k0(const Geom &, unsigned, const Pass<float> *, cudaStream_t, const float *, const float *,
                  const float *, const signed char *);
int launchd_f32k1(const Geom &, unsigned, const Pass<float> *, cudaStream_t, const float *, const float *,
                  const float *, const signed char *);
int launch_v32k0(const Geom &, const Pass<float> &, unsigned, cudaStream_t, const float *, const float *,
                 const float *, const signed char *, bool *);
int launch_v32k1(const Geom &, const Pass<float> &, unsigned, cudaStream_t, const float *, const float *,
                 const float *, const signed char *, bool *);
int launchd_v32k0(const Geom &, unsigned, const Pass<float> *, cudaStream_t, const float *, const float *,
                  const float *, const signed char *, bool *);
int launchd_v32k1(const Geom &, unsigned, const Pass<float> *, cudaStream_t, const float *, const float *,
                  const float *, const signed char *, bool *);
int launchp_v32k0(int, unsigned, const VecInst *, const int *, int, int, int *, cudaStream_t, bool *);
int launchp_v32k1(int, unsigned, const VecInst *, const int *, int, int, int *, cudaStream_t, bool *);
int launch_s32k0(const Geom &, const Pass<float> &, unsigned, cudaStream_t, const float *, const float *,
                 const float *, const signed char *, bool *);
int launch_s32k1(const Geom &, const Pass<float> &, unsigned, cudaStream_t, const float *, const float *,
                 const float *, const signed char *, bool *);
int prepare_v32k0();
int prepare_v32k1();
int prepare_f64();
int prepare_f32k0();
int prepare_f32k1();
int prepare_m32k0();
int prepare_m32k1();

template <>
int launch_stage<double>(const Geom &g, const Pass<double> &P, cudaStream_t st, const double *A, const double *B,
                         const double *L, const signed char *ptype, const TmaMaps *, int *nk)
{
    bool done = false;
    if (nk) *nk = 1;
    // FP64 runs every pass through the generic instantiation
    int e = launch_f64(g, P, SIG_GENERIC, st, A, B, L, ptype, nullptr, &done);
    return done ? e : (int)cudaErrorInvalidValue;
}

template <>
int launch_stage<float>(const Geom &g, const Pass<float> &P, cudaStream_t st, const float *A, const float *B,
                        const float *L, const signed char *ptype, const TmaMaps *tma, int *nk)
{
    bool done = false;
    if (nk) *nk = 1;
    if (g.slots) {
        // slot storage: only the slot instantiations read the layout; a pass
        // kind without one is refused (cudaErrorInvalidValue)
        int e = g.K ? launch_s32k1(g, P, pass_signature(P), st, A, B, L, ptype, &done)
                    : launch_s32k0(g, P, pass_signature(P), st, A, B, L, ptype, &done);
        return done ? e : (int)cudaErrorInvalidValue;
    }
    if (g.simplex != SIMPLEX_STANDARD) {
        // the mobility-weighted projection lives in the generic body only
        int e = g.K ? launch_f32k1(g, P, SIG_GENERIC, st, A, B, L, ptype, nullptr, &done)
                    : launch_f32k0(g, P, SIG_GENERIC, st, A, B, L, ptype, nullptr, &done);
        return done ? e : (int)cudaErrorInvalidValue;
    }
    if (P.m_in) {
        // masked storage: only the masked instantiations maintain the masks
        const unsigned sig = pass_signature(P);
        int e = g.K ? launch_m32k1(g, P, sig, st, A, B, L, ptype, &done)
                    : launch_m32k0(g, P, sig, st, A, B, L, ptype, &done);
        return done ? e : (int)cudaErrorInvalidValue;
    }
    if (!tma && g.kvar == KVAR_TWO_CELL && vec_eligible(g)) {
        // dense storage: the two-cell kernels take every pass they have
        const unsigned sig = pass_signature(P);
        int e = g.K ? launch_v32k1(g, P, sig, st, A, B, L, ptype, &done)
                    : launch_v32k0(g, P, sig, st, A, B, L, ptype, &done);
        if (done) {
            if (nk) *nk = 2;     // the pass and the wide pass of its crowded cells
            return e;
        }
    }
    auto go = [&](unsigned sig) {
        return g.K ? launch_f32k1(g, P, sig, st, A, B, L, ptype, tma, &done)
                   : launch_f32k0(g, P, sig, st, A, B, L, ptype, tma, &done);
    };
    int e = go(pass_signature(P));
    if (!done) e = go(SIG_GENERIC);
    return done ? e : (int)cudaErrorInvalidValue;
}

template <>
int launch_stage_d<double>(const Geom &g, unsigned sig, const Pass<double> *dP, cudaStream_t st, const double *A,
                           const double *B, const double *L, const signed char *ptype)
{
    return launchd_f64(g, sig, dP, st, A, B, L, ptype);
}

template <>
int launch_stage_d<float>(const Geom &g, unsigned sig, const Pass<float> *dP, cudaStream_t st, const float *A,
                          const float *B, const float *L, const signed char *ptype)
{
    if (g.kvar == KVAR_TWO_CELL && vec_eligible(g)) {
        bool done = false;
        int e = g.K ? launchd_v32k1(g, sig, dP, st, A, B, L, ptype, &done)
                    : launchd_v32k0(g, sig, dP, st, A, B, L, ptype, &done);
        if (done) return e;
    }
    return g.K ? launchd_f32k1(g, sig, dP, st, A, B, L, ptype) : launchd_f32k0(g, sig, dP, st, A, B, L, ptype);
}

int launch_packed(int dim, int K, unsigned sig, const VecInst *tab, const int *bstart, int n, int blocks, int *done,
                  cudaStream_t st, bool *ok)
{
    return K ? launchp_v32k1(dim, sig, tab, bstart, n, blocks, done, st, ok)
             : launchp_v32k0(dim, sig, tab, bstart, n, blocks, done, st, ok);
}

template <>
int kernels_per_pass_d<double>(const Geom &) { return 1; }

template <>
int kernels_per_pass_d<float>(const Geom &g) { return (g.kvar == KVAR_TWO_CELL && vec_eligible(g)) ? 2 : 1; }

template <>
int prepare_stage<double>() { return prepare_f64(); }

template <>
int prepare_stage<float>()
{
    const int a = prepare_f32k0(), b = prepare_f32k1(), c = prepare_m32k0(), d = prepare_m32k1();
    const int e = prepare_v32k0(), f = prepare_v32k1();
    return (a > 0 && b > 0 && c > 0 && d > 0 && e > 0 && f > 0) ? a : -1;
}

}  // namespace pfk
