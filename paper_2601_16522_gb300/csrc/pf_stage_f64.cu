// pf_stage_f64.cu -- double instantiations of the fused stage pass (generated list).
#include "pf_internal.h"

namespace pfk {

int launch_f64(const Geom &g, const Pass<double> &P, unsigned sig, cudaStream_t st, const double *A, const double *B,
             const double *L, const signed char *ptype, bool *done)
{
    const dim3 grid(g.tiles_x, g.tiles_y, g.nz);
    const size_t sm = sizeof(Smem<double>);
    *done = true;
    if (g.dim == 2 && g.K == 0 && sig == (SIG_GENERIC)) {
        cell_kernel<double, 2, 0, SIG_GENERIC><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && g.K == 1 && sig == (SIG_GENERIC)) {
        cell_kernel<double, 2, 1, SIG_GENERIC><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && g.K == 0 && sig == (SIG_GENERIC)) {
        cell_kernel<double, 3, 0, SIG_GENERIC><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && g.K == 1 && sig == (SIG_GENERIC)) {
        cell_kernel<double, 3, 1, SIG_GENERIC><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    *done = false;
    return 0;
}

int prepare_f64()
{
    const int sm = (int)sizeof(Smem<double>);
    if (cudaFuncSetAttribute(cell_kernel<double, 2, 0, SIG_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<double, 2, 1, SIG_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<double, 3, 0, SIG_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<double, 3, 1, SIG_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return -1;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cell_kernel<double, 3, 0, SIG_GENERIC>, BLOCK, sm) != cudaSuccess) return -1;
    return nb;
}

}  // namespace pfk
