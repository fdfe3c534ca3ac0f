// Multi-view rendering.
#include "stf_internal.h"

using namespace stf;

stf_status stf_render_batch(const stf_view* views, int n, int filter, int mode, unsigned long long seed)
{
    const float* lut = nullptr;
    stf_status s = stf_device_state(nullptr, &lut);
    if (s != STF_OK) return s;
    for (int i = 0; i < n; ++i) {
        DevView d;
        stf_fill_devview(views[i], filter, mode, seed, lut, d);
        cudaError_t e = stf_launch_single(d, views[i].tex->kind, mode, stf_stream());
        if (e != cudaSuccess) return stf_cuda_fail(e, "render launch");
    }
    return STF_OK;
}
