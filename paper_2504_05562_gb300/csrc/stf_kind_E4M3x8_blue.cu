// Render kernels for material kind K_E4M3x8 with blue-noise selection uniforms.
#include "stf_launch.cuh"
STF_INSTANTIATE_KIND_BLUE(stf::K_E4M3x8, launch_view_E4M3x8)
