// pf_stage_s32k1.cu -- slot-storage instantiations of the FP32 stage passes (K = 1).
#include "pf_internal.h"

namespace pfk {

int launch_s32k1(const Geom &g, const Pass<float> &P, unsigned sig, cudaStream_t st, const float *A,
             const float *B, const float *L, const signed char *ptype, bool *done)
{
    const dim3 grid(g.tiles_x, g.tiles_y, g.nz);
    *done = true;
    if (g.dim == 2 && sig == (SIG_PROJECT)) {
        slot_kernel<2, 1, SIG_PROJECT><<<grid, BLOCK, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && sig == (SIG_P2 | SIG_PROJECT)) {
        slot_kernel<2, 1, SIG_P2 | SIG_PROJECT><<<grid, BLOCK, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
        slot_kernel<2, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT><<<grid, BLOCK, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && sig == (SIG_R0OUT | SIG_PROJECT)) {
        slot_kernel<2, 1, SIG_R0OUT | SIG_PROJECT><<<grid, BLOCK, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && sig == (SIG_ERR)) {
        slot_kernel<2, 1, SIG_ERR><<<grid, BLOCK, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && sig == (SIG_P0 | SIG_PROJECT)) {
        slot_kernel<2, 1, SIG_P0 | SIG_PROJECT><<<grid, BLOCK, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && sig == (SIG_RHS)) {
        slot_kernel<2, 1, SIG_RHS><<<grid, BLOCK, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && sig == (SIG_PROJECT)) {
        slot_kernel<3, 1, SIG_PROJECT><<<grid, BLOCK, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && sig == (SIG_P2 | SIG_PROJECT)) {
        slot_kernel<3, 1, SIG_P2 | SIG_PROJECT><<<grid, BLOCK, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
        slot_kernel<3, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT><<<grid, BLOCK, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && sig == (SIG_R0OUT | SIG_PROJECT)) {
        slot_kernel<3, 1, SIG_R0OUT | SIG_PROJECT><<<grid, BLOCK, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && sig == (SIG_ERR)) {
        slot_kernel<3, 1, SIG_ERR><<<grid, BLOCK, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && sig == (SIG_P0 | SIG_PROJECT)) {
        slot_kernel<3, 1, SIG_P0 | SIG_PROJECT><<<grid, BLOCK, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && sig == (SIG_RHS)) {
        slot_kernel<3, 1, SIG_RHS><<<grid, BLOCK, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    *done = false;
    return 0;
}

}  // namespace pfk
