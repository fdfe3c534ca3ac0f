// Neural texel decode used by the K_NEURAL render kernels (declared here, defined with the
// decoder in stf_neural.cuh when that kind is compiled).
#pragma once

#include "stf_device.cuh"

namespace stf {

template <int C>
__device__ __forceinline__ void neural_decode_warp(const DevView& v, int x, int y, float (&t)[C]);

}  // namespace stf
