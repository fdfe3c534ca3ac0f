// Render kernels for the neural material kind (texels decoded on the tensor cores).
#include "stf_launch.cuh"
STF_INSTANTIATE_KIND(stf::K_NEURAL, launch_view_NEURAL)
