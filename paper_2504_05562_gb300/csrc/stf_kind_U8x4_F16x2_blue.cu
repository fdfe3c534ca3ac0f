// Render kernels for material kind K_U8x4_F16x2 with blue-noise selection uniforms.
#include "stf_launch.cuh"
STF_INSTANTIATE_KIND_BLUE(stf::K_U8x4_F16x2, launch_view_U8x4_F16x2)
