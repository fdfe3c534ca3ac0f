// Neural texture decoder.
#include "stf_internal.h"

stf_status stf_create_neural_texture(const stf_texture_desc*, stf_texture**)
{
    return stf_fail(STF_ERR_UNSUPPORTED, "neural textures are not built yet");
}

cudaError_t stf_launch_neural_view(const stf::DevView&, int, cudaStream_t) { return cudaErrorNotSupported; }
