// Render kernels for material kind K_F32x8.
#include "stf_launch.cuh"
STF_INSTANTIATE_KIND(stf::K_F32x8, launch_view_F32x8)
