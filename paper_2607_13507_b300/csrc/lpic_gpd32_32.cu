// The FP32 tile kernels for dimension 3, shape order 2.
#include "lpic_gpd32_impl.cuh"

template struct lpic::Gpd32<3, 2>;
