// pf_stage_f64.cu -- double instantiations of the fused stage pass.
#include "pf_internal.h"

namespace pfk {

int launch_f64(const Geom &g, const Pass<double> &P, unsigned sig, cudaStream_t st, const double *A, const double *B,
             const double *L, const signed char *ptype, const TmaMaps *tma, bool *done)
{
    const dim3 grid(g.tiles_x, g.tiles_y, g.nz);
    *done = true;
    const size_t sm = sizeof(Smem<double>);
    if (g.dim == 2 && g.K == 0 && sig == SIG_GENERIC) {
        cell_kernel<double, 2, 0, SIG_GENERIC><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && g.K == 1 && sig == SIG_GENERIC) {
        cell_kernel<double, 2, 1, SIG_GENERIC><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && g.K == 0 && sig == SIG_GENERIC) {
        cell_kernel<double, 3, 0, SIG_GENERIC><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && g.K == 1 && sig == SIG_GENERIC) {
        cell_kernel<double, 3, 1, SIG_GENERIC><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    (void)tma;
    *done = false;
    return 0;
}

int launchd_f64(const Geom &g, unsigned sig, const Pass<double> *dP, cudaStream_t st, const double *A, const double *B,
             const double *L, const signed char *ptype)
{
    const dim3 grid(g.tiles_x, g.tiles_y, g.nz);
    const size_t sm = sizeof(Smem<double>);
    if (g.dim == 2 && g.K == 0) {
        cell_kernel_d<double, 2, 0, SIG_GENERIC><<<grid, BLOCK, sm, st>>>(g, dP, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && g.K == 1) {
        cell_kernel_d<double, 2, 1, SIG_GENERIC><<<grid, BLOCK, sm, st>>>(g, dP, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && g.K == 0) {
        cell_kernel_d<double, 3, 0, SIG_GENERIC><<<grid, BLOCK, sm, st>>>(g, dP, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && g.K == 1) {
        cell_kernel_d<double, 3, 1, SIG_GENERIC><<<grid, BLOCK, sm, st>>>(g, dP, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    (void)sig;
    return (int)cudaErrorInvalidValue;
}

int prepare_f64()
{
    if (cudaFuncSetAttribute(cell_kernel<double, 2, 0, SIG_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<double>)) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<double, 2, 1, SIG_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<double>)) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<double, 3, 0, SIG_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<double>)) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<double, 3, 1, SIG_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<double>)) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel_d<double, 2, 0, SIG_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<double>)) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel_d<double, 2, 1, SIG_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<double>)) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel_d<double, 3, 0, SIG_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<double>)) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel_d<double, 3, 1, SIG_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<double>)) != cudaSuccess) return -1;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cell_kernel<double, 3, 0, SIG_GENERIC>, BLOCK, sizeof(Smem<double>)) != cudaSuccess) return -1;
    return nb;
}

}  // namespace pfk
