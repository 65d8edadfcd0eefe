// The unfused-stage tile kernels for dimension 3, shape order 1.
#include "lpic_gpd32s_impl.cuh"

template struct lpic::Gpd32Stages<3, 1>;
