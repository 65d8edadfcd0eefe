// The FP32 tile kernels for dimension 2, shape order 2.
#include "lpic_gpd32_impl.cuh"

template struct lpic::Gpd32<2, 2>;
