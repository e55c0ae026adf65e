// pf_internal.h -- declarations shared by the engine's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include "pf_kernels.cuh"

namespace pfk {

// Launch one fused pass: the instantiation is chosen from the pass signature
// (specialised FP32 hot passes) or the generic kernel.  Returns a cudaError_t.
// tma: tensor maps of the pass's buffers for the TMA-staged FP32 kernels
// (nullptr: plain loads).
template <typename T>
int launch_stage(const Geom &g, const Pass<T> &P, cudaStream_t st, const T *A, const T *B, const T *L,
                 const signed char *ptype, const TmaMaps *tma);

// Opt every instantiation into its shared memory on the current device;
// returns the resident blocks per SM of the generic 3D kernel (<= 0: error).
template <typename T>
int prepare_stage();

}  // namespace pfk
