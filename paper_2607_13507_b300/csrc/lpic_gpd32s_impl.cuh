// lpic_gpd32s_impl.cuh -- definitions of the unfused-stage launchers; included
// only by the per-instance translation units lpic_gpd32s_<dim><order>.cu.
#pragma once
#include "lpic_gpd32.h"

namespace lpic {

template <int DIM, int ORDER>
cudaError_t Gpd32Stages<DIM, ORDER>::set_smem(size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_gpd32<DIM, ORDER, kGpdGather>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_gpd32<DIM, ORDER, kGpdFieldsIn>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes);
}

template <int DIM, int ORDER>
void Gpd32Stages<DIM, ORDER>::gather(const GpdArgs& A, unsigned blocks, size_t smem, cudaStream_t st) {
    k_gpd32<DIM, ORDER, kGpdGather><<<blocks, kGpdThreads, smem, st>>>(A);
}

template <int DIM, int ORDER>
void Gpd32Stages<DIM, ORDER>::push(const GpdArgs& A, unsigned blocks, size_t smem, cudaStream_t st) {
    k_gpd32<DIM, ORDER, kGpdFieldsIn><<<blocks, kGpdThreads, smem, st>>>(A);
}

}  // namespace lpic
