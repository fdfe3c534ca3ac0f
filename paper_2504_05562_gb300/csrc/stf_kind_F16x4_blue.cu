// Render kernels for material kind K_F16x4 with blue-noise selection uniforms.
#include "stf_launch.cuh"
STF_INSTANTIATE_KIND_BLUE(stf::K_F16x4, launch_view_F16x4)
