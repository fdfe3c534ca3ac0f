// Render kernels for material kind K_F16x4.
#include "stf_launch.cuh"
STF_INSTANTIATE_KIND(stf::K_F16x4, launch_view_F16x4)
