// The unfused-stage tile kernels for dimension 2, shape order 2.
#include "lpic_gpd32s_impl.cuh"

template struct lpic::Gpd32Stages<2, 2>;
