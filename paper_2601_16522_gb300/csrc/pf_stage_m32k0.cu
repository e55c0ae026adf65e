// pf_stage_m32k0.cu -- masked-storage instantiations of the FP32 fast pass (K = 0).
#include "pf_internal.h"

namespace pfk {

int launch_m32k0(const Geom &g, const Pass<float> &P, unsigned sig, cudaStream_t st, const float *A,
             const float *B, const float *L, const signed char *ptype, bool *done)
{
    const dim3 grid(g.tiles_x, g.tiles_y, g.nz);
    const size_t smf = sizeof(ListSmem<float>);
    *done = true;
    if (g.N <= 128 && g.Vs < 0x7fffffffLL) {
        if (g.N <= 4) {
            if (g.dim == 2 && sig == (SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_PROJECT, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P2 | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_P2 | SIG_PROJECT, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_R0OUT | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_R0OUT | SIG_PROJECT, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_ERR)) {
                fast_kernel<2, 0, SIG_ERR, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_P0 | SIG_PROJECT, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_O2 | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_O2 | SIG_PROJECT, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_Z | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_Z | SIG_PROJECT, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_Z | SIG_O2 | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_Z | SIG_O2 | SIG_PROJECT, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_PROJECT, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P2 | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_P2 | SIG_PROJECT, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_R0OUT | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_R0OUT | SIG_PROJECT, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_ERR)) {
                fast_kernel<3, 0, SIG_ERR, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_P0 | SIG_PROJECT, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_O2 | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_O2 | SIG_PROJECT, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_Z | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_Z | SIG_PROJECT, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_Z | SIG_O2 | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_Z | SIG_O2 | SIG_PROJECT, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 4, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
        }
        if (g.N > 4 && g.N <= 32) {
            if (g.dim == 2 && sig == (SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_PROJECT, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P2 | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_P2 | SIG_PROJECT, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_R0OUT | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_R0OUT | SIG_PROJECT, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_ERR)) {
                fast_kernel<2, 0, SIG_ERR, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_P0 | SIG_PROJECT, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_O2 | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_O2 | SIG_PROJECT, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_Z | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_Z | SIG_PROJECT, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_Z | SIG_O2 | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_Z | SIG_O2 | SIG_PROJECT, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_PROJECT, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P2 | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_P2 | SIG_PROJECT, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_R0OUT | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_R0OUT | SIG_PROJECT, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_ERR)) {
                fast_kernel<3, 0, SIG_ERR, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_P0 | SIG_PROJECT, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_O2 | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_O2 | SIG_PROJECT, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_Z | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_Z | SIG_PROJECT, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_Z | SIG_O2 | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_Z | SIG_O2 | SIG_PROJECT, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 32, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
        }
        if (g.N > 32) {
            if (g.dim == 2 && sig == (SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_PROJECT, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P2 | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_P2 | SIG_PROJECT, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_R0OUT | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_R0OUT | SIG_PROJECT, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_ERR)) {
                fast_kernel<2, 0, SIG_ERR, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_P0 | SIG_PROJECT, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_O2 | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_O2 | SIG_PROJECT, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_Z | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_Z | SIG_PROJECT, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_Z | SIG_O2 | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_Z | SIG_O2 | SIG_PROJECT, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_PROJECT, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P2 | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_P2 | SIG_PROJECT, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_R0OUT | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_R0OUT | SIG_PROJECT, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_ERR)) {
                fast_kernel<3, 0, SIG_ERR, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_P0 | SIG_PROJECT, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_O2 | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_O2 | SIG_PROJECT, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_Z | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_Z | SIG_PROJECT, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_Z | SIG_O2 | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_Z | SIG_O2 | SIG_PROJECT, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 128, true><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
        }
    }
    *done = false;
    return 0;
}

int prepare_m32k0()
{
    const int smf = (int)sizeof(ListSmem<float>);
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_PROJECT, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_P2 | SIG_PROJECT, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_R0OUT | SIG_PROJECT, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_ERR, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_P0 | SIG_PROJECT, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_O2 | SIG_PROJECT, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_Z | SIG_PROJECT, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_Z | SIG_O2 | SIG_PROJECT, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_PROJECT, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_P2 | SIG_PROJECT, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_R0OUT | SIG_PROJECT, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_ERR, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_P0 | SIG_PROJECT, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_O2 | SIG_PROJECT, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_Z | SIG_PROJECT, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_Z | SIG_O2 | SIG_PROJECT, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_PROJECT, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_P2 | SIG_PROJECT, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_R0OUT | SIG_PROJECT, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_ERR, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_P0 | SIG_PROJECT, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_O2 | SIG_PROJECT, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_Z | SIG_PROJECT, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_Z | SIG_O2 | SIG_PROJECT, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_PROJECT, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_P2 | SIG_PROJECT, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_R0OUT | SIG_PROJECT, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_ERR, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_P0 | SIG_PROJECT, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_O2 | SIG_PROJECT, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_Z | SIG_PROJECT, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_Z | SIG_O2 | SIG_PROJECT, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_PROJECT, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_P2 | SIG_PROJECT, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_R0OUT | SIG_PROJECT, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_ERR, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_P0 | SIG_PROJECT, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_O2 | SIG_PROJECT, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_Z | SIG_PROJECT, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_Z | SIG_O2 | SIG_PROJECT, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_PROJECT, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_P2 | SIG_PROJECT, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_R0OUT | SIG_PROJECT, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_ERR, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_P0 | SIG_PROJECT, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_O2 | SIG_PROJECT, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_Z | SIG_PROJECT, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_Z | SIG_O2 | SIG_PROJECT, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    return 1;
}

}  // namespace pfk
