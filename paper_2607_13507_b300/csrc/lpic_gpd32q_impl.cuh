// lpic_gpd32q_impl.cuh -- definitions of the launchers of the tile kernel
// with emission inside the push; included only by the per-instance
// translation units lpic_gpd32q_<dim><order>.cu.
#pragma once
#include "lpic_gpd32.h"

namespace lpic {

template <int DIM, int ORDER>
cudaError_t Gpd32Qed<DIM, ORDER>::set_smem(size_t bytes) {
    return cudaFuncSetAttribute(k_gpd32<DIM, ORDER, kGpdQed>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes);
}

template <int DIM, int ORDER>
void Gpd32Qed<DIM, ORDER>::tile(const GpdArgs& A, unsigned blocks, size_t smem, cudaStream_t st) {
    k_gpd32<DIM, ORDER, kGpdQed><<<blocks, kGpdThreads, smem, st>>>(A);
}

}  // namespace lpic
