// pf_stage_f32k0.cu -- float instantiations of the fused stage pass (generated list).
#include "pf_internal.h"

namespace pfk {

int launch_f32k0(const Geom &g, const Pass<float> &P, unsigned sig, cudaStream_t st, const float *A, const float *B,
             const float *L, const signed char *ptype, bool *done)
{
    const dim3 grid(g.tiles_x, g.tiles_y, g.nz);
    const size_t sm = sizeof(Smem<float>);
    *done = true;
    const size_t smf = sizeof(ListSmem<float>);
    if (g.N <= 32 && g.Vs * (long long)(g.N + g.K) < 0x7fffffffLL) {
        if (g.N <= 4) {
            if (g.dim == 2 && sig == (SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P2 | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_P2 | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_R0OUT | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_R0OUT | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_ERR)) {
                fast_kernel<2, 0, SIG_ERR, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_P0 | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P2 | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_P2 | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_R0OUT | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_R0OUT | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_ERR)) {
                fast_kernel<3, 0, SIG_ERR, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_P0 | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
        }
        if (g.N > 4) {
            if (g.dim == 2 && sig == (SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P2 | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_P2 | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_R0OUT | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_R0OUT | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_ERR)) {
                fast_kernel<2, 0, SIG_ERR, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_PROJECT)) {
                fast_kernel<2, 0, SIG_P0 | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P2 | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_P2 | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_R0OUT | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_R0OUT | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_ERR)) {
                fast_kernel<3, 0, SIG_ERR, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_PROJECT)) {
                fast_kernel<3, 0, SIG_P0 | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
        }
    }
    if (g.dim == 2 && g.K == 0 && sig == (SIG_PROJECT)) {
        cell_kernel<float, 2, 0, SIG_PROJECT><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && g.K == 0 && sig == (SIG_P2 | SIG_PROJECT)) {
        cell_kernel<float, 2, 0, SIG_P2 | SIG_PROJECT><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && g.K == 0 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
        cell_kernel<float, 2, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && g.K == 0 && sig == (SIG_R0OUT | SIG_PROJECT)) {
        cell_kernel<float, 2, 0, SIG_R0OUT | SIG_PROJECT><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && g.K == 0 && sig == (SIG_ERR)) {
        cell_kernel<float, 2, 0, SIG_ERR><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && g.K == 0 && sig == (SIG_P0 | SIG_PROJECT)) {
        cell_kernel<float, 2, 0, SIG_P0 | SIG_PROJECT><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 2 && g.K == 0 && sig == (SIG_GENERIC)) {
        cell_kernel<float, 2, 0, SIG_GENERIC><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && g.K == 0 && sig == (SIG_PROJECT)) {
        cell_kernel<float, 3, 0, SIG_PROJECT><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && g.K == 0 && sig == (SIG_P2 | SIG_PROJECT)) {
        cell_kernel<float, 3, 0, SIG_P2 | SIG_PROJECT><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && g.K == 0 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
        cell_kernel<float, 3, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && g.K == 0 && sig == (SIG_R0OUT | SIG_PROJECT)) {
        cell_kernel<float, 3, 0, SIG_R0OUT | SIG_PROJECT><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && g.K == 0 && sig == (SIG_ERR)) {
        cell_kernel<float, 3, 0, SIG_ERR><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && g.K == 0 && sig == (SIG_P0 | SIG_PROJECT)) {
        cell_kernel<float, 3, 0, SIG_P0 | SIG_PROJECT><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && g.K == 0 && sig == (SIG_GENERIC)) {
        cell_kernel<float, 3, 0, SIG_GENERIC><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    *done = false;
    return 0;
}

int prepare_f32k0()
{
    const int sm = (int)sizeof(Smem<float>);
    if (cudaFuncSetAttribute(cell_kernel<float, 2, 0, SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<float, 2, 0, SIG_P2 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<float, 2, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<float, 2, 0, SIG_R0OUT | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<float, 2, 0, SIG_ERR>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<float, 2, 0, SIG_P0 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<float, 2, 0, SIG_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<float, 3, 0, SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<float, 3, 0, SIG_P2 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<float, 3, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<float, 3, 0, SIG_R0OUT | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<float, 3, 0, SIG_ERR>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<float, 3, 0, SIG_P0 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<float, 3, 0, SIG_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return -1;
    const int smf = (int)sizeof(ListSmem<float>);
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_P2 | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_R0OUT | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_ERR, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_P0 | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_P2 | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_R0OUT | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_ERR, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_P0 | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_P2 | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_R0OUT | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_ERR, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 0, SIG_P0 | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_P2 | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_R0OUT | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_ERR, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 0, SIG_P0 | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cell_kernel<float, 3, 0, SIG_GENERIC>, BLOCK, sm) != cudaSuccess) return -1;
    return nb;
}

}  // namespace pfk
