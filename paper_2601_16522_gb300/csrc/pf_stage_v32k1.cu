// pf_stage_v32k1.cu -- two-cell FP32 instantiations of the fused stage pass (K = 1).
#include "pf_internal.h"

namespace pfk {

int launch_v32k1(const Geom &g, const Pass<float> &P, unsigned sig, cudaStream_t st, const float *A,
             const float *B, const float *L, const signed char *ptype, bool *done)
{
    const dim3 grid((g.nx + 2 * VTX - 1) / (2 * VTX), (g.ny + VTY - 1) / VTY, g.nz);
    *done = true;
    if (g.dim == 2 && sig == (SIG_PROJECT)) {
        vec_kernel<2, 1, SIG_PROJECT><<<grid, VBLOCK, vec_smem<SIG_PROJECT>(), st>>>(g, P, A, B, L, ptype);
        wide_fix_kernel<2, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && sig == (SIG_P2 | SIG_PROJECT)) {
        vec_kernel<2, 1, SIG_P2 | SIG_PROJECT><<<grid, VBLOCK, vec_smem<SIG_P2 | SIG_PROJECT>(), st>>>(g, P, A, B, L, ptype);
        wide_fix_kernel<2, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
        vec_kernel<2, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT><<<grid, VBLOCK, vec_smem<SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>(), st>>>(g, P, A, B, L, ptype);
        wide_fix_kernel<2, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && sig == (SIG_R0OUT | SIG_PROJECT)) {
        vec_kernel<2, 1, SIG_R0OUT | SIG_PROJECT><<<grid, VBLOCK, vec_smem<SIG_R0OUT | SIG_PROJECT>(), st>>>(g, P, A, B, L, ptype);
        wide_fix_kernel<2, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && sig == (SIG_ERR)) {
        vec_kernel<2, 1, SIG_ERR><<<grid, VBLOCK, vec_smem<SIG_ERR>(), st>>>(g, P, A, B, L, ptype);
        wide_fix_kernel<2, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && sig == (SIG_P0 | SIG_PROJECT)) {
        vec_kernel<2, 1, SIG_P0 | SIG_PROJECT><<<grid, VBLOCK, vec_smem<SIG_P0 | SIG_PROJECT>(), st>>>(g, P, A, B, L, ptype);
        wide_fix_kernel<2, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && sig == (SIG_ERR | SIG_R0OUT)) {
        vec_kernel<2, 1, SIG_ERR | SIG_R0OUT><<<grid, VBLOCK, vec_smem<SIG_ERR | SIG_R0OUT>(), st>>>(g, P, A, B, L, ptype);
        wide_fix_kernel<2, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && sig == (SIG_PROJECT)) {
        vec_kernel<3, 1, SIG_PROJECT><<<grid, VBLOCK, vec_smem<SIG_PROJECT>(), st>>>(g, P, A, B, L, ptype);
        wide_fix_kernel<3, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && sig == (SIG_P2 | SIG_PROJECT)) {
        vec_kernel<3, 1, SIG_P2 | SIG_PROJECT><<<grid, VBLOCK, vec_smem<SIG_P2 | SIG_PROJECT>(), st>>>(g, P, A, B, L, ptype);
        wide_fix_kernel<3, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
        vec_kernel<3, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT><<<grid, VBLOCK, vec_smem<SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>(), st>>>(g, P, A, B, L, ptype);
        wide_fix_kernel<3, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && sig == (SIG_R0OUT | SIG_PROJECT)) {
        vec_kernel<3, 1, SIG_R0OUT | SIG_PROJECT><<<grid, VBLOCK, vec_smem<SIG_R0OUT | SIG_PROJECT>(), st>>>(g, P, A, B, L, ptype);
        wide_fix_kernel<3, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && sig == (SIG_ERR)) {
        vec_kernel<3, 1, SIG_ERR><<<grid, VBLOCK, vec_smem<SIG_ERR>(), st>>>(g, P, A, B, L, ptype);
        wide_fix_kernel<3, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && sig == (SIG_P0 | SIG_PROJECT)) {
        vec_kernel<3, 1, SIG_P0 | SIG_PROJECT><<<grid, VBLOCK, vec_smem<SIG_P0 | SIG_PROJECT>(), st>>>(g, P, A, B, L, ptype);
        wide_fix_kernel<3, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && sig == (SIG_ERR | SIG_R0OUT)) {
        vec_kernel<3, 1, SIG_ERR | SIG_R0OUT><<<grid, VBLOCK, vec_smem<SIG_ERR | SIG_R0OUT>(), st>>>(g, P, A, B, L, ptype);
        wide_fix_kernel<3, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    *done = false;
    return 0;
}

int launchd_v32k1(const Geom &g, unsigned sig, const Pass<float> *dP, cudaStream_t st, const float *A,
             const float *B, const float *L, const signed char *ptype, bool *done)
{
    const dim3 grid((g.nx + 2 * VTX - 1) / (2 * VTX), (g.ny + VTY - 1) / VTY, g.nz);
    *done = true;
    if (g.dim == 2 && sig == (SIG_R0OUT | SIG_PROJECT)) {
        vec_kernel_d<2, 1, SIG_R0OUT | SIG_PROJECT><<<grid, VBLOCK, vec_smem<SIG_R0OUT | SIG_PROJECT>(), st>>>(g, dP, A, B, L, ptype);
        wide_fix_kernel_d<2, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, dP, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
        vec_kernel_d<2, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT><<<grid, VBLOCK, vec_smem<SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>(), st>>>(g, dP, A, B, L, ptype);
        wide_fix_kernel_d<2, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, dP, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && sig == (SIG_P2 | SIG_PROJECT)) {
        vec_kernel_d<2, 1, SIG_P2 | SIG_PROJECT><<<grid, VBLOCK, vec_smem<SIG_P2 | SIG_PROJECT>(), st>>>(g, dP, A, B, L, ptype);
        wide_fix_kernel_d<2, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, dP, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && sig == (SIG_ERR)) {
        vec_kernel_d<2, 1, SIG_ERR><<<grid, VBLOCK, vec_smem<SIG_ERR>(), st>>>(g, dP, A, B, L, ptype);
        wide_fix_kernel_d<2, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, dP, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && sig == (SIG_R0OUT | SIG_PROJECT)) {
        vec_kernel_d<3, 1, SIG_R0OUT | SIG_PROJECT><<<grid, VBLOCK, vec_smem<SIG_R0OUT | SIG_PROJECT>(), st>>>(g, dP, A, B, L, ptype);
        wide_fix_kernel_d<3, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, dP, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
        vec_kernel_d<3, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT><<<grid, VBLOCK, vec_smem<SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>(), st>>>(g, dP, A, B, L, ptype);
        wide_fix_kernel_d<3, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, dP, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && sig == (SIG_P2 | SIG_PROJECT)) {
        vec_kernel_d<3, 1, SIG_P2 | SIG_PROJECT><<<grid, VBLOCK, vec_smem<SIG_P2 | SIG_PROJECT>(), st>>>(g, dP, A, B, L, ptype);
        wide_fix_kernel_d<3, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, dP, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && sig == (SIG_ERR)) {
        vec_kernel_d<3, 1, SIG_ERR><<<grid, VBLOCK, vec_smem<SIG_ERR>(), st>>>(g, dP, A, B, L, ptype);
        wide_fix_kernel_d<3, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(g, dP, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    *done = false;
    return 0;
}

int launchp_v32k1(int dim, unsigned sig, const VecInst *tab, const int *bstart, int n, int blocks, int *done,
             cudaStream_t st, bool *ok)
{
    *ok = true;
    if (dim == 2 && sig == (SIG_PROJECT)) {
        packed_kernel<2, 1, SIG_PROJECT><<<blocks, VBLOCK, vec_smem<SIG_PROJECT>(), st>>>(tab, bstart, n);
        packed_wide_fix_kernel<2, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(tab, n, done);
        return (int)cudaGetLastError();
    }
    if (dim == 2 && sig == (SIG_P2 | SIG_PROJECT)) {
        packed_kernel<2, 1, SIG_P2 | SIG_PROJECT><<<blocks, VBLOCK, vec_smem<SIG_P2 | SIG_PROJECT>(), st>>>(tab, bstart, n);
        packed_wide_fix_kernel<2, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(tab, n, done);
        return (int)cudaGetLastError();
    }
    if (dim == 2 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
        packed_kernel<2, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT><<<blocks, VBLOCK, vec_smem<SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>(), st>>>(tab, bstart, n);
        packed_wide_fix_kernel<2, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(tab, n, done);
        return (int)cudaGetLastError();
    }
    if (dim == 2 && sig == (SIG_R0OUT | SIG_PROJECT)) {
        packed_kernel<2, 1, SIG_R0OUT | SIG_PROJECT><<<blocks, VBLOCK, vec_smem<SIG_R0OUT | SIG_PROJECT>(), st>>>(tab, bstart, n);
        packed_wide_fix_kernel<2, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(tab, n, done);
        return (int)cudaGetLastError();
    }
    if (dim == 2 && sig == (SIG_ERR)) {
        packed_kernel<2, 1, SIG_ERR><<<blocks, VBLOCK, vec_smem<SIG_ERR>(), st>>>(tab, bstart, n);
        packed_wide_fix_kernel<2, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(tab, n, done);
        return (int)cudaGetLastError();
    }
    if (dim == 2 && sig == (SIG_P0 | SIG_PROJECT)) {
        packed_kernel<2, 1, SIG_P0 | SIG_PROJECT><<<blocks, VBLOCK, vec_smem<SIG_P0 | SIG_PROJECT>(), st>>>(tab, bstart, n);
        packed_wide_fix_kernel<2, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(tab, n, done);
        return (int)cudaGetLastError();
    }
    if (dim == 2 && sig == (SIG_ERR | SIG_R0OUT)) {
        packed_kernel<2, 1, SIG_ERR | SIG_R0OUT><<<blocks, VBLOCK, vec_smem<SIG_ERR | SIG_R0OUT>(), st>>>(tab, bstart, n);
        packed_wide_fix_kernel<2, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(tab, n, done);
        return (int)cudaGetLastError();
    }
    if (dim == 3 && sig == (SIG_PROJECT)) {
        packed_kernel<3, 1, SIG_PROJECT><<<blocks, VBLOCK, vec_smem<SIG_PROJECT>(), st>>>(tab, bstart, n);
        packed_wide_fix_kernel<3, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(tab, n, done);
        return (int)cudaGetLastError();
    }
    if (dim == 3 && sig == (SIG_P2 | SIG_PROJECT)) {
        packed_kernel<3, 1, SIG_P2 | SIG_PROJECT><<<blocks, VBLOCK, vec_smem<SIG_P2 | SIG_PROJECT>(), st>>>(tab, bstart, n);
        packed_wide_fix_kernel<3, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(tab, n, done);
        return (int)cudaGetLastError();
    }
    if (dim == 3 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
        packed_kernel<3, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT><<<blocks, VBLOCK, vec_smem<SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>(), st>>>(tab, bstart, n);
        packed_wide_fix_kernel<3, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(tab, n, done);
        return (int)cudaGetLastError();
    }
    if (dim == 3 && sig == (SIG_R0OUT | SIG_PROJECT)) {
        packed_kernel<3, 1, SIG_R0OUT | SIG_PROJECT><<<blocks, VBLOCK, vec_smem<SIG_R0OUT | SIG_PROJECT>(), st>>>(tab, bstart, n);
        packed_wide_fix_kernel<3, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(tab, n, done);
        return (int)cudaGetLastError();
    }
    if (dim == 3 && sig == (SIG_ERR)) {
        packed_kernel<3, 1, SIG_ERR><<<blocks, VBLOCK, vec_smem<SIG_ERR>(), st>>>(tab, bstart, n);
        packed_wide_fix_kernel<3, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(tab, n, done);
        return (int)cudaGetLastError();
    }
    if (dim == 3 && sig == (SIG_P0 | SIG_PROJECT)) {
        packed_kernel<3, 1, SIG_P0 | SIG_PROJECT><<<blocks, VBLOCK, vec_smem<SIG_P0 | SIG_PROJECT>(), st>>>(tab, bstart, n);
        packed_wide_fix_kernel<3, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(tab, n, done);
        return (int)cudaGetLastError();
    }
    if (dim == 3 && sig == (SIG_ERR | SIG_R0OUT)) {
        packed_kernel<3, 1, SIG_ERR | SIG_R0OUT><<<blocks, VBLOCK, vec_smem<SIG_ERR | SIG_R0OUT>(), st>>>(tab, bstart, n);
        packed_wide_fix_kernel<3, 1><<<WIDE_FIX_BLOCKS, VCELLS, 0, st>>>(tab, n, done);
        return (int)cudaGetLastError();
    }
    *ok = false;
    return 0;
}

int prepare_v32k1()
{
    if (cudaFuncSetAttribute(vec_kernel<2, 1, SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel<2, 1, SIG_P2 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_P2 | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel<2, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel<2, 1, SIG_R0OUT | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_R0OUT | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel<2, 1, SIG_ERR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_ERR>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel<2, 1, SIG_P0 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_P0 | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel<2, 1, SIG_ERR | SIG_R0OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_ERR | SIG_R0OUT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel<3, 1, SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel<3, 1, SIG_P2 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_P2 | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel<3, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel<3, 1, SIG_R0OUT | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_R0OUT | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel<3, 1, SIG_ERR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_ERR>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel<3, 1, SIG_P0 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_P0 | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel<3, 1, SIG_ERR | SIG_R0OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_ERR | SIG_R0OUT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel_d<2, 1, SIG_R0OUT | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_R0OUT | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel_d<2, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel_d<2, 1, SIG_P2 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_P2 | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel_d<2, 1, SIG_ERR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_ERR>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel_d<3, 1, SIG_R0OUT | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_R0OUT | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel_d<3, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel_d<3, 1, SIG_P2 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_P2 | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(vec_kernel_d<3, 1, SIG_ERR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_ERR>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(packed_kernel<2, 1, SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(packed_kernel<2, 1, SIG_P2 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_P2 | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(packed_kernel<2, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(packed_kernel<2, 1, SIG_R0OUT | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_R0OUT | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(packed_kernel<2, 1, SIG_ERR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_ERR>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(packed_kernel<2, 1, SIG_P0 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_P0 | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(packed_kernel<2, 1, SIG_ERR | SIG_R0OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_ERR | SIG_R0OUT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(packed_kernel<3, 1, SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(packed_kernel<3, 1, SIG_P2 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_P2 | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(packed_kernel<3, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(packed_kernel<3, 1, SIG_R0OUT | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_R0OUT | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(packed_kernel<3, 1, SIG_ERR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_ERR>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(packed_kernel<3, 1, SIG_P0 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_P0 | SIG_PROJECT>()) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(packed_kernel<3, 1, SIG_ERR | SIG_R0OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem<SIG_ERR | SIG_R0OUT>()) != cudaSuccess) return -1;
    return 1;
}

}  // namespace pfk
