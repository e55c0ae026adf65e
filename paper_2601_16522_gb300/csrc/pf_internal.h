// pf_internal.h -- declarations shared by the engine's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include "pf_kernels.cuh"
#include "pf_vec.cuh"
#include "pf_slots.cuh"

namespace pfk {

// Launch one fused pass: the instantiation is chosen from the pass signature
// (specialised FP32 hot passes) or the generic kernel.  Returns a cudaError_t.
// tma: tensor maps of the pass's buffers for the TMA-staged FP32 kernels
// (nullptr: plain loads).
// *nk (may be null) receives the number of kernels the pass launched.
template <typename T>
int launch_stage(const Geom &g, const Pass<T> &P, cudaStream_t st, const T *A, const T *B, const T *L,
                 const signed char *ptype, const TmaMaps *tma, int *nk = nullptr);

// Kernels one pass of the device-driven loop launches (two-cell passes add
// the wide pass of their crowded cells).
template <typename T>
int kernels_per_pass_d(const Geom &g);

// Launch one pass whose description (buffers, coefficients) sits in device
// memory at dP, written there by a planning kernel before the launch runs
// (device-driven adaptive steps).  sig: the pass signature the description
// will have (stage 1, RKL body or error sweep).  Returns a cudaError_t.
template <typename T>
int launch_stage_d(const Geom &g, unsigned sig, const Pass<T> *dP, cudaStream_t st, const T *A, const T *B,
                   const T *L, const signed char *ptype);

// Packed launch of one pass kind (dimension dim, K, signature sig) over the n
// problems of a device table (two-cell FP32 passes; see VecInst): blocks is
// the sum of their block counts, bstart their prefix sums, done a zeroed
// device counter of the caller.  Returns a cudaError_t; *ok false when the
// pass kind has no packed form.
int launch_packed(int dim, int K, unsigned sig, const VecInst *tab, const int *bstart, int n, int blocks, int *done,
                  cudaStream_t st, bool *ok);

// Opt every instantiation into its shared memory on the current device;
// returns the resident blocks per SM of the generic 3D kernel (<= 0: error).
template <typename T>
int prepare_stage();

}  // namespace pfk
