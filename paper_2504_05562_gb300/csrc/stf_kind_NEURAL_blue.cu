// Render kernels for material kind K_NEURAL with blue-noise selection uniforms.
#include "stf_launch.cuh"
STF_INSTANTIATE_KIND_BLUE(stf::K_NEURAL, launch_view_NEURAL)
