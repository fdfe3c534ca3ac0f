// Render kernels for material kind K_E4M3x8.
#include "stf_launch.cuh"
STF_INSTANTIATE_KIND(stf::K_E4M3x8, launch_view_E4M3x8)
