// The tile kernel with emission inside the push, dimension 3, shape order 2.
#include "lpic_gpd32q_impl.cuh"

template struct lpic::Gpd32Qed<3, 2>;
