// Render kernels for material kind K_BF16x8 with blue-noise selection uniforms.
#include "stf_launch.cuh"
STF_INSTANTIATE_KIND_BLUE(stf::K_BF16x8, launch_view_BF16x8)
