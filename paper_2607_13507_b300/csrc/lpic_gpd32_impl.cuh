// lpic_gpd32_impl.cuh -- definitions of the Gpd32 launchers; included only by
// the per-instance translation units.
#pragma once
#include "lpic_gpd32.h"

namespace lpic {

template <int DIM, int ORDER>
cudaError_t Gpd32<DIM, ORDER>::set_smem(size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_gpd32<DIM, ORDER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_gpd32_queue<DIM, ORDER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int DIM, int ORDER>
void Gpd32<DIM, ORDER>::tile(const GpdArgs& A, unsigned blocks, size_t smem, cudaStream_t st) {
    k_gpd32<DIM, ORDER><<<blocks, kGpdThreads, smem, st>>>(A);
}

template <int DIM, int ORDER>
void Gpd32<DIM, ORDER>::escape(const GpdArgs& A, unsigned blocks, cudaStream_t st) {
    k_gpd32_escape<DIM, ORDER><<<blocks, 256, 0, st>>>(A);
}

template <int DIM, int ORDER>
void Gpd32<DIM, ORDER>::queue(const GpdArgs* slots, const int* order, const int* prefix, int nslots, int* head,
                              unsigned blocks, size_t smem, cudaStream_t st) {
    k_gpd32_queue<DIM, ORDER><<<blocks, kGpdThreads, smem, st>>>(slots, order, prefix, nslots, head);
}

template <int DIM, int ORDER>
const void* Gpd32<DIM, ORDER>::queue_fn() {
    return reinterpret_cast<const void*>(k_gpd32_queue<DIM, ORDER>);
}

}  // namespace lpic
