// Render kernels for material kind K_U8x4_F16x2.
#include "stf_launch.cuh"
STF_INSTANTIATE_KIND(stf::K_U8x4_F16x2, launch_view_U8x4_F16x2)
