// pf_stage_f32k1.cu -- float instantiations of the fused stage pass.
#include "pf_internal.h"

namespace pfk {

int launch_f32k1(const Geom &g, const Pass<float> &P, unsigned sig, cudaStream_t st, const float *A, const float *B,
             const float *L, const signed char *ptype, const TmaMaps *tma, bool *done)
{
    const dim3 grid(g.tiles_x, g.tiles_y, g.nz);
    *done = true;
    const size_t smf = sizeof(ListSmem<float>);
    const size_t smt = 1024 + sizeof(TmaSmem) + sizeof(ListSmem<float>);
    if (g.N > 32 && g.N <= 128 && g.Vs < 0x7fffffffLL) {
        if (g.dim == 2 && sig == (SIG_O2 | SIG_PROJECT)) {
            fast_kernel<2, 1, SIG_O2 | SIG_PROJECT, 128><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
        if (g.dim == 2 && sig == (SIG_Z | SIG_PROJECT)) {
            fast_kernel<2, 1, SIG_Z | SIG_PROJECT, 128><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
        if (g.dim == 2 && sig == (SIG_Z | SIG_O2 | SIG_PROJECT)) {
            fast_kernel<2, 1, SIG_Z | SIG_O2 | SIG_PROJECT, 128><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
        if (g.dim == 2 && sig == (SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT)) {
            fast_kernel<2, 1, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 128><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
        if (g.dim == 3 && sig == (SIG_O2 | SIG_PROJECT)) {
            fast_kernel<3, 1, SIG_O2 | SIG_PROJECT, 128><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
        if (g.dim == 3 && sig == (SIG_Z | SIG_PROJECT)) {
            fast_kernel<3, 1, SIG_Z | SIG_PROJECT, 128><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
        if (g.dim == 3 && sig == (SIG_Z | SIG_O2 | SIG_PROJECT)) {
            fast_kernel<3, 1, SIG_Z | SIG_O2 | SIG_PROJECT, 128><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
        if (g.dim == 3 && sig == (SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT)) {
            fast_kernel<3, 1, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 128><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
    }
    if (g.N > 32 && g.N <= 250 && g.Vs < 0x7fffffffLL) {
        if (g.dim == 2 && sig == (SIG_PROJECT)) {
            big_kernel<2, 1, SIG_PROJECT><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
        if (g.dim == 2 && sig == (SIG_P2 | SIG_PROJECT)) {
            big_kernel<2, 1, SIG_P2 | SIG_PROJECT><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
        if (g.dim == 2 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
            big_kernel<2, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
        if (g.dim == 2 && sig == (SIG_R0OUT | SIG_PROJECT)) {
            big_kernel<2, 1, SIG_R0OUT | SIG_PROJECT><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
        if (g.dim == 2 && sig == (SIG_ERR)) {
            big_kernel<2, 1, SIG_ERR><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
        if (g.dim == 2 && sig == (SIG_P0 | SIG_PROJECT)) {
            big_kernel<2, 1, SIG_P0 | SIG_PROJECT><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
        if (g.dim == 3 && sig == (SIG_PROJECT)) {
            big_kernel<3, 1, SIG_PROJECT><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
        if (g.dim == 3 && sig == (SIG_P2 | SIG_PROJECT)) {
            big_kernel<3, 1, SIG_P2 | SIG_PROJECT><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
        if (g.dim == 3 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
            big_kernel<3, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
        if (g.dim == 3 && sig == (SIG_R0OUT | SIG_PROJECT)) {
            big_kernel<3, 1, SIG_R0OUT | SIG_PROJECT><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
        if (g.dim == 3 && sig == (SIG_ERR)) {
            big_kernel<3, 1, SIG_ERR><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
        if (g.dim == 3 && sig == (SIG_P0 | SIG_PROJECT)) {
            big_kernel<3, 1, SIG_P0 | SIG_PROJECT><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
            return (int)cudaGetLastError();
        }
    }
    if (g.N <= 32 && g.Vs < 0x7fffffffLL) {
        if (tma && g.dim == 3 && g.N > 4) {
            if (sig == (SIG_PROJECT)) {
                tma_kernel<1, SIG_PROJECT><<<grid, TMA_BLOCK, smt, st>>>(g, P, *tma, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (sig == (SIG_P2 | SIG_PROJECT)) {
                tma_kernel<1, SIG_P2 | SIG_PROJECT><<<grid, TMA_BLOCK, smt, st>>>(g, P, *tma, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
                tma_kernel<1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT><<<grid, TMA_BLOCK, smt, st>>>(g, P, *tma, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (sig == (SIG_R0OUT | SIG_PROJECT)) {
                tma_kernel<1, SIG_R0OUT | SIG_PROJECT><<<grid, TMA_BLOCK, smt, st>>>(g, P, *tma, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (sig == (SIG_ERR)) {
                tma_kernel<1, SIG_ERR><<<grid, TMA_BLOCK, smt, st>>>(g, P, *tma, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (sig == (SIG_P0 | SIG_PROJECT)) {
                tma_kernel<1, SIG_P0 | SIG_PROJECT><<<grid, TMA_BLOCK, smt, st>>>(g, P, *tma, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
        }
        if (g.N <= 4) {
            if (g.dim == 2 && sig == (SIG_PROJECT)) {
                fast_kernel<2, 1, SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P2 | SIG_PROJECT)) {
                fast_kernel<2, 1, SIG_P2 | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
                fast_kernel<2, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_R0OUT | SIG_PROJECT)) {
                fast_kernel<2, 1, SIG_R0OUT | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_ERR)) {
                fast_kernel<2, 1, SIG_ERR, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_PROJECT)) {
                fast_kernel<2, 1, SIG_P0 | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_ERR | SIG_R0OUT)) {
                fast_kernel<2, 1, SIG_ERR | SIG_R0OUT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_O2 | SIG_PROJECT)) {
                fast_kernel<2, 1, SIG_O2 | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_Z | SIG_PROJECT)) {
                fast_kernel<2, 1, SIG_Z | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_Z | SIG_O2 | SIG_PROJECT)) {
                fast_kernel<2, 1, SIG_Z | SIG_O2 | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT)) {
                fast_kernel<2, 1, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_PROJECT)) {
                fast_kernel<3, 1, SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P2 | SIG_PROJECT)) {
                fast_kernel<3, 1, SIG_P2 | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
                fast_kernel<3, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_R0OUT | SIG_PROJECT)) {
                fast_kernel<3, 1, SIG_R0OUT | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_ERR)) {
                fast_kernel<3, 1, SIG_ERR, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_PROJECT)) {
                fast_kernel<3, 1, SIG_P0 | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_ERR | SIG_R0OUT)) {
                fast_kernel<3, 1, SIG_ERR | SIG_R0OUT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_O2 | SIG_PROJECT)) {
                fast_kernel<3, 1, SIG_O2 | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_Z | SIG_PROJECT)) {
                fast_kernel<3, 1, SIG_Z | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_Z | SIG_O2 | SIG_PROJECT)) {
                fast_kernel<3, 1, SIG_Z | SIG_O2 | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT)) {
                fast_kernel<3, 1, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
        }
        if (g.N > 4) {
            if (g.dim == 2 && sig == (SIG_PROJECT)) {
                fast_kernel<2, 1, SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P2 | SIG_PROJECT)) {
                fast_kernel<2, 1, SIG_P2 | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
                fast_kernel<2, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_R0OUT | SIG_PROJECT)) {
                fast_kernel<2, 1, SIG_R0OUT | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_ERR)) {
                fast_kernel<2, 1, SIG_ERR, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_PROJECT)) {
                fast_kernel<2, 1, SIG_P0 | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_ERR | SIG_R0OUT)) {
                fast_kernel<2, 1, SIG_ERR | SIG_R0OUT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_O2 | SIG_PROJECT)) {
                fast_kernel<2, 1, SIG_O2 | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_Z | SIG_PROJECT)) {
                fast_kernel<2, 1, SIG_Z | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_Z | SIG_O2 | SIG_PROJECT)) {
                fast_kernel<2, 1, SIG_Z | SIG_O2 | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT)) {
                fast_kernel<2, 1, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_PROJECT)) {
                fast_kernel<3, 1, SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P2 | SIG_PROJECT)) {
                fast_kernel<3, 1, SIG_P2 | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
                fast_kernel<3, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_R0OUT | SIG_PROJECT)) {
                fast_kernel<3, 1, SIG_R0OUT | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_ERR)) {
                fast_kernel<3, 1, SIG_ERR, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_PROJECT)) {
                fast_kernel<3, 1, SIG_P0 | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_ERR | SIG_R0OUT)) {
                fast_kernel<3, 1, SIG_ERR | SIG_R0OUT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_O2 | SIG_PROJECT)) {
                fast_kernel<3, 1, SIG_O2 | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_Z | SIG_PROJECT)) {
                fast_kernel<3, 1, SIG_Z | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_Z | SIG_O2 | SIG_PROJECT)) {
                fast_kernel<3, 1, SIG_Z | SIG_O2 | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT)) {
                fast_kernel<3, 1, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, P, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
        }
    }
    const size_t sm = sizeof(Smem<float>);
    if (g.dim == 2 && g.K == 1 && sig == SIG_GENERIC) {
        cell_kernel<float, 2, 1, SIG_GENERIC><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    if (g.dim == 3 && g.K == 1 && sig == SIG_GENERIC) {
        cell_kernel<float, 3, 1, SIG_GENERIC><<<grid, BLOCK, sm, st>>>(g, P, A, B, L, ptype);
        return (int)cudaGetLastError();
    }
    (void)tma;
    *done = false;
    return 0;
}

int launchd_f32k1(const Geom &g, unsigned sig, const Pass<float> *dP, cudaStream_t st, const float *A, const float *B,
             const float *L, const signed char *ptype)
{
    const dim3 grid(g.tiles_x, g.tiles_y, g.nz);
    const size_t smf = sizeof(ListSmem<float>);
    if (g.N <= 32 && g.Vs < 0x7fffffffLL) {
        if (g.N <= 4) {
            if (g.dim == 2 && sig == (SIG_R0OUT | SIG_PROJECT)) {
                fast_kernel_d<2, 1, SIG_R0OUT | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, dP, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
                fast_kernel_d<2, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, dP, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P2 | SIG_PROJECT)) {
                fast_kernel_d<2, 1, SIG_P2 | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, dP, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_ERR)) {
                fast_kernel_d<2, 1, SIG_ERR, 4><<<grid, BLOCK, smf, st>>>(g, dP, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_R0OUT | SIG_PROJECT)) {
                fast_kernel_d<3, 1, SIG_R0OUT | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, dP, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
                fast_kernel_d<3, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, dP, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P2 | SIG_PROJECT)) {
                fast_kernel_d<3, 1, SIG_P2 | SIG_PROJECT, 4><<<grid, BLOCK, smf, st>>>(g, dP, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_ERR)) {
                fast_kernel_d<3, 1, SIG_ERR, 4><<<grid, BLOCK, smf, st>>>(g, dP, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
        }
        if (g.N > 4) {
            if (g.dim == 2 && sig == (SIG_R0OUT | SIG_PROJECT)) {
                fast_kernel_d<2, 1, SIG_R0OUT | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, dP, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
                fast_kernel_d<2, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, dP, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_P2 | SIG_PROJECT)) {
                fast_kernel_d<2, 1, SIG_P2 | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, dP, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 2 && sig == (SIG_ERR)) {
                fast_kernel_d<2, 1, SIG_ERR, 32><<<grid, BLOCK, smf, st>>>(g, dP, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_R0OUT | SIG_PROJECT)) {
                fast_kernel_d<3, 1, SIG_R0OUT | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, dP, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT)) {
                fast_kernel_d<3, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, dP, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_P2 | SIG_PROJECT)) {
                fast_kernel_d<3, 1, SIG_P2 | SIG_PROJECT, 32><<<grid, BLOCK, smf, st>>>(g, dP, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
            if (g.dim == 3 && sig == (SIG_ERR)) {
                fast_kernel_d<3, 1, SIG_ERR, 32><<<grid, BLOCK, smf, st>>>(g, dP, A, B, L, ptype);
                return (int)cudaGetLastError();
            }
        }
    }
    (void)sig;
    return (int)cudaErrorInvalidValue;
}

int prepare_f32k1()
{
    const int smf = (int)sizeof(ListSmem<float>);
    const int smt = (int)(1024 + sizeof(TmaSmem) + sizeof(ListSmem<float>));
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_O2 | SIG_PROJECT, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_Z | SIG_PROJECT, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_Z | SIG_O2 | SIG_PROJECT, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_O2 | SIG_PROJECT, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_Z | SIG_PROJECT, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_Z | SIG_O2 | SIG_PROJECT, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(big_kernel<2, 1, SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(big_kernel<2, 1, SIG_P2 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(big_kernel<2, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(big_kernel<2, 1, SIG_R0OUT | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(big_kernel<2, 1, SIG_ERR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(big_kernel<2, 1, SIG_P0 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(big_kernel<3, 1, SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(big_kernel<3, 1, SIG_P2 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(big_kernel<3, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(big_kernel<3, 1, SIG_R0OUT | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(big_kernel<3, 1, SIG_ERR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(big_kernel<3, 1, SIG_P0 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(tma_kernel<1, SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smt) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(tma_kernel<1, SIG_P2 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smt) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(tma_kernel<1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smt) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(tma_kernel<1, SIG_R0OUT | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smt) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(tma_kernel<1, SIG_ERR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smt) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(tma_kernel<1, SIG_P0 | SIG_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smt) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_P2 | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_R0OUT | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_ERR, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_P0 | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_ERR | SIG_R0OUT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_O2 | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_Z | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_Z | SIG_O2 | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_P2 | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_R0OUT | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_ERR, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_P0 | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_ERR | SIG_R0OUT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_O2 | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_Z | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_Z | SIG_O2 | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_P2 | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_R0OUT | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_ERR, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_P0 | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_ERR | SIG_R0OUT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_O2 | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_Z | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_Z | SIG_O2 | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<2, 1, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_P2 | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_R0OUT | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_ERR, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_P0 | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_ERR | SIG_R0OUT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_O2 | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_Z | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_Z | SIG_O2 | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel<3, 1, SIG_P0 | SIG_Z | SIG_EMB | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<float, 2, 1, SIG_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<float>)) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(cell_kernel<float, 3, 1, SIG_GENERIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<float>)) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel_d<2, 1, SIG_R0OUT | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel_d<2, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel_d<2, 1, SIG_P2 | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel_d<2, 1, SIG_ERR, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel_d<3, 1, SIG_R0OUT | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel_d<3, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel_d<3, 1, SIG_P2 | SIG_PROJECT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel_d<3, 1, SIG_ERR, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel_d<2, 1, SIG_R0OUT | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel_d<2, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel_d<2, 1, SIG_P2 | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel_d<2, 1, SIG_ERR, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel_d<3, 1, SIG_R0OUT | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel_d<3, 1, SIG_P0 | SIG_P2 | SIG_R0IN | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel_d<3, 1, SIG_P2 | SIG_PROJECT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    if (cudaFuncSetAttribute(fast_kernel_d<3, 1, SIG_ERR, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smf) != cudaSuccess) return -1;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cell_kernel<float, 3, 1, SIG_GENERIC>, BLOCK, sizeof(Smem<float>)) != cudaSuccess) return -1;
    return nb;
}

}  // namespace pfk
