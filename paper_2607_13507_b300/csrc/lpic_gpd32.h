// lpic_gpd32.h -- host-side launchers of the FP32 tile kernels.
//
// Each (dimension, shape order) instance of the fused kernel, its persistent
// ensemble form and its escape kernel is compiled in a translation unit of its
// own (lpic_gpd32_<dim><order>.cu), so the heavy instances build in parallel;
// the rest of the library calls them through these declarations.
#pragma once
#include <cuda_runtime.h>

#include "lpic_fp32.cuh"

namespace lpic {

template <int DIM, int ORDER>
struct Gpd32 {
    // raises the dynamic shared-memory limit of the tile and queue kernels
    static cudaError_t set_smem(size_t bytes);
    // one block per work item
    static void tile(const GpdArgs& A, unsigned blocks, size_t smem, cudaStream_t st);
    // the particles the tile kernel queued beyond its drift margin
    static void escape(const GpdArgs& A, unsigned blocks, cudaStream_t st);
    // persistent blocks over the device queue of a batch of grids
    static void queue(const GpdArgs* slots, const int* order, const int* prefix, int nslots, int* head,
                      unsigned blocks, size_t smem, cudaStream_t st);
    static const void* queue_fn();
};

// The unfused stages (kGpdGather, kGpdFieldsIn), compiled in translation
// units of their own (lpic_gpd32s_<dim><order>.cu).
template <int DIM, int ORDER>
struct Gpd32Stages {
    static cudaError_t set_smem(size_t bytes);
    static void gather(const GpdArgs& A, unsigned blocks, size_t smem, cudaStream_t st);
    static void push(const GpdArgs& A, unsigned blocks, size_t smem, cudaStream_t st);
};

// The fused kernel with nonlinear Compton emission inside the push
// (kGpdQed), compiled in translation units of its own
// (lpic_gpd32q_<dim><order>.cu); its escapes go to Gpd32::escape.
template <int DIM, int ORDER>
struct Gpd32Qed {
    static cudaError_t set_smem(size_t bytes);
    static void tile(const GpdArgs& A, unsigned blocks, size_t smem, cudaStream_t st);
};

}  // namespace lpic
