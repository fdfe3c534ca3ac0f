// Render kernels for material kind K_BF16x8.
#include "stf_launch.cuh"
STF_INSTANTIATE_KIND(stf::K_BF16x8, launch_view_BF16x8)
