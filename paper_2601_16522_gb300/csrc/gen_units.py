"""Writes the instantiation units pf_stage_*.cu (run from the repository root
after changing a kernel template's parameters or the set of pass
signatures; the written files are committed, and build.py compiles them).

pf_stage_f64.cu      FP64: the generic stage kernel, 2D/3D, K = 0/1
pf_stage_f32k{0,1}   FP32, K fixed: big_kernel (32 < N <= 250), tma_kernel and
                     fast_kernel (N <= 32, NMAX 4 or 32) per pass signature
                     (fast_kernel also for the error sweep that keeps its RHS),
                     and the generic kernel as the fallback
(each of these also holds launchd_*: the descriptor-driven passes of
device-driven adaptive RKL steps)
pf_stage_m32k{0,1}   FP32 masked storage, K fixed: fast_kernel<..., true> per
                     pass signature for N <= 4, N <= 32 and N <= 128
pf_stage_v32k{0,1}   FP32 dense storage, K fixed: vec_kernel (two cells per
                     thread, N <= 128, nx even) per pass signature followed by
                     the wide pass of its crowded cells (wide_fix_kernel), and
                     the _d forms for the device-driven adaptive RKL steps
"""
import os

HERE = os.path.dirname(os.path.abspath(__file__))

# pass signatures with specialised FP32 instantiations: Euler/SSP substep,
# RKL1 body, RKL2 body, RKL stage 1, error sweep, SSP2 final combination
SIGS = ["SIG_PROJECT", "SIG_P2 | SIG_PROJECT", "SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT",
        "SIG_R0OUT | SIG_PROJECT", "SIG_ERR", "SIG_P0 | SIG_PROJECT"]
# the dense fast kernel also has the error sweep that keeps F(u^{n+1})
FAST_SIGS = SIGS + ["SIG_ERR | SIG_R0OUT"]
# SSP(10)4 passes (one-cell rolled body, dense and masked): fixed-step stage 5,
# and the stages with the embedded accumulator
SSP_SIGS = ["SIG_O2 | SIG_PROJECT", "SIG_Z | SIG_PROJECT", "SIG_Z | SIG_O2 | SIG_PROJECT",
            "SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT"]
# passes of the device-driven adaptive RKL steps: stage 1, RKL2 body, RKL1
# body, error sweep (descriptor-driven kernels)
DSIGS = ["SIG_R0OUT | SIG_PROJECT", "SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT", "SIG_P2 | SIG_PROJECT", "SIG_ERR"]


def unit(T, kcs, fast, fname):
    tag = fname.replace('.cu', '').replace('pf_stage_', '')
    L = ["// %s -- %s instantiations of the fused stage pass." % (fname, T),
         '#include "pf_internal.h"', "", "namespace pfk {", ""]
    L.append("int launch_%s(const Geom &g, const Pass<%s> &P, unsigned sig, cudaStream_t st, const %s *A, const %s *B,"
             % (tag, T, T, T))
    L.append("             const %s *L, const signed char *ptype, const TmaMaps *tma, bool *done)" % T)
    L.append("{")
    L.append("    const dim3 grid(g.tiles_x, g.tiles_y, g.nz);")
    L.append("    *done = true;")
    prep = []
    if fast:
        kc = kcs[0]
        L.append("    const size_t smf = sizeof(ListSmem<float>);")
        L.append("    const size_t smt = 1024 + sizeof(TmaSmem) + sizeof(ListSmem<float>);")
        # SSP(10)4 passes with 33..128 phases: the rolled body the masked
        # storage uses (its results are the dense ones bit for bit)
        L.append("    if (g.N > 32 && g.N <= 128 && g.Vs < 0x7fffffffLL) {")
        for d in (2, 3):
            for sg in SSP_SIGS:
                L.append("        if (g.dim == %d && sig == (%s)) {" % (d, sg))
                L.append("            fast_kernel<%d, %d, %s, 128><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);" % (d, kc, sg))
                L.append("            return (int)cudaGetLastError();")
                L.append("        }")
                prep.append("    if (cudaFuncSetAttribute(fast_kernel<%d, %d, %s, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;" % (d, kc, sg))
        L.append("    }")
        L.append("    if (g.N > 32 && g.N <= 250 && g.Vs < 0x7fffffffLL) {")
        for d in (2, 3):
            for sg in SIGS:
                L.append("        if (g.dim == %d && sig == (%s)) {" % (d, sg))
                L.append("            big_kernel<%d, %d, %s><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);" % (d, kc, sg))
                L.append("            return (int)cudaGetLastError();")
                L.append("        }")
                prep.append("    if (cudaFuncSetAttribute(big_kernel<%d, %d, %s>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;" % (d, kc, sg))
        L.append("    }")
        L.append("    if (g.N <= 32 && g.Vs < 0x7fffffffLL) {")
        L.append("        if (tma && g.dim == 3 && g.N > 4) {")
        for sg in SIGS:
            L.append("            if (sig == (%s)) {" % sg)
            L.append("                tma_kernel<%d, %s><<<grid, TMA_BLOCK, smt, st>>>(g, P, *tma, A, B, L, ptype);" % (kc, sg))
            L.append("                return (int)cudaGetLastError();")
            L.append("            }")
            prep.append("    if (cudaFuncSetAttribute(tma_kernel<%d, %s>, cudaFuncAttributeMaxDynamicSharedMemorySize, smt) != cudaSuccess) return -1;" % (kc, sg))
        L.append("        }")
        for nmax in (4, 32):
            L.append("        if (%s) {" % ("g.N <= 4" if nmax == 4 else "g.N > 4"))
            for d in (2, 3):
                for sg in FAST_SIGS + SSP_SIGS:
                    L.append("            if (g.dim == %d && sig == (%s)) {" % (d, sg))
                    L.append("                fast_kernel<%d, %d, %s, %d><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);" % (d, kc, sg, nmax))
                    L.append("                return (int)cudaGetLastError();")
                    L.append("            }")
                    prep.append("    if (cudaFuncSetAttribute(fast_kernel<%d, %d, %s, %d>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;" % (d, kc, sg, nmax))
            L.append("        }")
        L.append("    }")
    L.append("    const size_t sm = sizeof(Smem<%s>);" % T)
    for d in (2, 3):
        for k in kcs:
            L.append("    if (g.dim == %d && g.K == %d && sig == SIG_GENERIC) {" % (d, k))
            L.append("        cell_kernel<%s, %d, %d, SIG_GENERIC><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);" % (T, d, k))
            L.append("        return (int)cudaGetLastError();")
            L.append("    }")
            prep.append("    if (cudaFuncSetAttribute(cell_kernel<%s, %d, %d, SIG_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<%s>)) != cudaSuccess) return -1;" % (T, d, k, T))
    L.append("    (void)tma;")
    L.append("    *done = false;")
    L.append("    return 0;")
    L.append("}")
    L.append("")
    # descriptor-driven passes of device-driven adaptive RKL steps
    L.append("int launchd_%s(const Geom &g, unsigned sig, const Pass<%s> *dP, cudaStream_t st, const %s *A, const %s *B,"
             % (tag, T, T, T))
    L.append("             const %s *L, const signed char *ptype)" % T)
    L.append("{")
    L.append("    const dim3 grid(g.tiles_x, g.tiles_y, g.nz);")
    if fast:
        kc = kcs[0]
        L.append("    const size_t smf = sizeof(ListSmem<float>);")
        L.append("    if (g.N <= 32 && g.Vs < 0x7fffffffLL) {")
        for nmax in (4, 32):
            L.append("        if (%s) {" % ("g.N <= 4" if nmax == 4 else "g.N > 4"))
            for d in (2, 3):
                for sg in DSIGS:
                    L.append("            if (g.dim == %d && sig == (%s)) {" % (d, sg))
                    L.append("                fast_kernel_d<%d, %d, %s, %d><<<grid, BLOCK, smf, st>>>(g, dP, A, B, L, ptype);" % (d, kc, sg, nmax))
                    L.append("                return (int)cudaGetLastError();")
                    L.append("            }")
                    prep.append("    if (cudaFuncSetAttribute(fast_kernel_d<%d, %d, %s, %d>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;" % (d, kc, sg, nmax))
            L.append("        }")
        L.append("    }")
    else:
        L.append("    const size_t sm = sizeof(Smem<%s>);" % T)
        for d in (2, 3):
            for k in kcs:
                L.append("    if (g.dim == %d && g.K == %d) {" % (d, k))
                L.append("        cell_kernel_d<%s, %d, %d, SIG_GENERIC><<<grid, BLOCK, sm, st>>>(g, dP, A, B, L, ptype);" % (T, d, k))
                L.append("        return (int)cudaGetLastError();")
                L.append("    }")
                prep.append("    if (cudaFuncSetAttribute(cell_kernel_d<%s, %d, %d, SIG_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<%s>)) != cudaSuccess) return -1;" % (T, d, k, T))
    L.append("    (void)sig;")
    L.append("    return (int)cudaErrorInvalidValue;")
    L.append("}")
    L.append("")
    L.append("int prepare_%s()" % tag)
    L.append("{")
    if fast:
        L.append("    const int smf = (int)sizeof(ListSmem<float>);")
        L.append("    const int smt = (int)(1024 + sizeof(TmaSmem) + sizeof(ListSmem<float>));")
    L += prep
    L.append("    int nb = 0;")
    L.append("    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cell_kernel<%s, 3, %d, SIG_GENERIC>, BLOCK, sizeof(Smem<%s>)) != cudaSuccess) return -1;" % (T, kcs[0], T))
    L.append("    return nb;")
    L.append("}")
    L.append("")
    L.append("}  // namespace pfk")
    return "\n".join(L) + "\n"


def munit(kc, fname):
    tag = "m32k%d" % kc
    L = ["// %s -- masked-storage instantiations of the FP32 fast pass (K = %d)." % (fname, kc),
         '#include "pf_internal.h"', "", "namespace pfk {", ""]
    L.append("int launch_%s(const Geom &g, const Pass<float> &P, unsigned sig, cudaStream_t st, const float *A," % tag)
    L.append("             const float *B, const float *L, const signed char *ptype, bool *done)")
    L.append("{")
    L.append("    const dim3 grid(g.tiles_x, g.tiles_y, g.nz);")
    L.append("    const size_t smf = sizeof(ListSmem<float>);")
    L.append("    *done = true;")
    prep = []
    L.append("    if (g.N <= 128 && g.Vs < 0x7fffffffLL) {")
    for nmax in (4, 32, 128):
        L.append("        if (%s) {" % {4: "g.N <= 4", 32: "g.N > 4 && g.N <= 32", 128: "g.N > 32"}[nmax])
        for d in (2, 3):
            for sg in SIGS + SSP_SIGS:
                L.append("            if (g.dim == %d && sig == (%s)) {" % (d, sg))
                L.append("                fast_kernel<%d, %d, %s, %d, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);" % (d, kc, sg, nmax))
                L.append("                return (int)cudaGetLastError();")
                L.append("            }")
                prep.append("    if (cudaFuncSetAttribute(fast_kernel<%d, %d, %s, %d, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;" % (d, kc, sg, nmax))
        L.append("        }")
    L.append("    }")
    L.append("    *done = false;")
    L.append("    return 0;")
    L.append("}")
    L.append("")
    L.append("int prepare_%s()" % tag)
    L.append("{")
    L.append("    const int smf = (int)sizeof(ListSmem<float>);")
    L += prep
    L.append("    return 1;")
    L.append("}")
    L.append("")
    L.append("}  // namespace pfk")
    return "\n".join(L) + "\n"


def sunit(kc, fname):
    tag = "s32k%d" % kc
    L = ["// %s -- slot-storage instantiations of the FP32 stage passes (K = %d)." % (fname, kc),
         '#include "pf_internal.h"', "", "namespace pfk {", ""]
    L.append("int launch_%s(const Geom &g, const Pass<float> &P, unsigned sig, cudaStream_t st, const float *A," % tag)
    L.append("             const float *B, const float *L, const signed char *ptype, bool *done)")
    L.append("{")
    L.append("    const dim3 grid(g.tiles_x, g.tiles_y, g.nz);")
    L.append("    *done = true;")
    for d in (2, 3):
        for sg in SIGS + ["SIG_RHS"]:
            L.append("    if (g.dim == %d && sig == (%s)) {" % (d, sg))
            L.append("        slot_kernel<%d, %d, %s><<<grid, BLOCK, 0, st>>>(g, P, A, B, L, ptype);" % (d, kc, sg))
            L.append("        return (int)cudaGetLastError();")
            L.append("    }")
    L.append("    *done = false;")
    L.append("    return 0;")
    L.append("}")
    L.append("")
    L.append("}  // namespace pfk")
    return "\n".join(L) + "\n"


def vunit(kc, fname):
    tag = "v32k%d" % kc
    L = ["// %s -- two-cell FP32 instantiations of the fused stage pass (K = %d)." % (fname, kc),
         '#include "pf_internal.h"', "", "namespace pfk {", ""]
    L.append("int launch_%s(const Geom &g, const Pass<float> &P, unsigned sig, cudaStream_t st, const float *A," % tag)
    L.append("             const float *B, const float *L, const signed char *ptype, bool *done)")
    L.append("{")
    L.append("    const dim3 grid((g.nx + 2 * VTX - 1) / (2 * VTX), (g.ny + VTY - 1) / VTY, g.nz);")
    L.append("    *done = true;")
    prep = []
    for d in (2, 3):
        for sg in FAST_SIGS:
            L.append("    if (g.dim == %d && sig == (%s)) {" % (d, sg))
            L.append("        vec_kernel<%d, %d, %s><<<grid, VBLOCK, vec_smem<%s>(), st>>>(g, P, A, B, L, ptype);" % (d, kc, sg, sg))
            L.append("        wide_fix_kernel<%d, %d><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, P, A, B, L, ptype);" % (d, kc))
            L.append("        return (int)cudaGetLastError();")
            L.append("    }")
            prep.append("    if (cudaFuncSetAttribute(vec_kernel<%d, %d, %s>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<%s>()) != cudaSuccess) return -1;" % (d, kc, sg, sg))
    L.append("    *done = false;")
    L.append("    return 0;")
    L.append("}")
    L.append("")
    L.append("int launchd_%s(const Geom &g, unsigned sig, const Pass<float> *dP, cudaStream_t st, const float *A," % tag)
    L.append("             const float *B, const float *L, const signed char *ptype, bool *done)")
    L.append("{")
    L.append("    const dim3 grid((g.nx + 2 * VTX - 1) / (2 * VTX), (g.ny + VTY - 1) / VTY, g.nz);")
    L.append("    *done = true;")
    for d in (2, 3):
        for sg in DSIGS:
            L.append("    if (g.dim == %d && sig == (%s)) {" % (d, sg))
            L.append("        vec_kernel_d<%d, %d, %s><<<grid, VBLOCK, vec_smem<%s>(), st>>>(g, dP, A, B, L, ptype);" % (d, kc, sg, sg))
            L.append("        wide_fix_kernel_d<%d, %d><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, dP, A, B, L, ptype);" % (d, kc))
            L.append("        return (int)cudaGetLastError();")
            L.append("    }")
            prep.append("    if (cudaFuncSetAttribute(vec_kernel_d<%d, %d, %s>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<%s>()) != cudaSuccess) return -1;" % (d, kc, sg, sg))
    L.append("    *done = false;")
    L.append("    return 0;")
    L.append("}")
    L.append("")
    # packed launches of several problems (batched serving)
    L.append("int launchp_%s(int dim, unsigned sig, const VecInst *tab, const int *bstart, int n, int blocks, int *done," % tag)
    L.append("             cudaStream_t st, bool *ok)")
    L.append("{")
    L.append("    *ok = true;")
    for d in (2, 3):
        for sg in FAST_SIGS:
            L.append("    if (dim == %d && sig == (%s)) {" % (d, sg))
            L.append("        packed_kernel<%d, %d, %s><<<blocks, VBLOCK, vec_smem<%s>(), st>>>(tab, bstart, n);" % (d, kc, sg, sg))
            L.append("        packed_wide_fix_kernel<%d, %d><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(tab, n, done);" % (d, kc))
            L.append("        return (int)cudaGetLastError();")
            L.append("    }")
            prep.append("    if (cudaFuncSetAttribute(packed_kernel<%d, %d, %s>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<%s>()) != cudaSuccess) return -1;" % (d, kc, sg, sg))
    L.append("    *ok = false;")
    L.append("    return 0;")
    L.append("}")
    L.append("")
    L.append("int prepare_%s()" % tag)
    L.append("{")
    L += prep
    L.append("    return 1;")
    L.append("}")
    L.append("")
    L.append("}  // namespace pfk")
    return "\n".join(L) + "\n"


def render():
    """{file name: text} of every instantiation unit."""
    return {
        "pf_stage_f64.cu": unit("double", [0, 1], False, "pf_stage_f64.cu"),
        "pf_stage_f32k0.cu": unit("float", [0], True, "pf_stage_f32k0.cu"),
        "pf_stage_f32k1.cu": unit("float", [1], True, "pf_stage_f32k1.cu"),
        "pf_stage_m32k0.cu": munit(0, "pf_stage_m32k0.cu"),
        "pf_stage_m32k1.cu": munit(1, "pf_stage_m32k1.cu"),
        "pf_stage_v32k0.cu": vunit(0, "pf_stage_v32k0.cu"),
        "pf_stage_v32k1.cu": vunit(1, "pf_stage_v32k1.cu"),
        "pf_stage_s32k0.cu": sunit(0, "pf_stage_s32k0.cu"),
        "pf_stage_s32k1.cu": sunit(1, "pf_stage_s32k1.cu"),
    }


def main():
    for name, text in render().items():
        with open(os.path.join(HERE, name), "w") as f:
            f.write(text)


if __name__ == "__main__":
    main()
