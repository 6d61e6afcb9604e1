// The fused potential kernel with the per-species networks on the tensor cores
// (BF16 and split-BF16 forms): its launch, instantiated in a translation unit
// of its own.
#include "potential_launch.cuh"

namespace aenet {

cudaError_t launch_fused_tc(Context &c, const Grid &g, int n) {
    if (!c.md_prezeroed) {  // (inside an MD step the kick + drift kernel has cleared both)
        cudaError_t e = cudaMemsetAsync(c.d_stats, 0, sizeof(unsigned long long) * 4, c.stream);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(c.d_F4, 0, sizeof(float4) * (size_t)(n > 0 ? n : 1), c.stream);
        if (e != cudaSuccess) return e;
    }
    return c.precision == AENET_BF16X3 ? dispatch<kFusedTCx3>(c, g) : dispatch<kFusedTC>(c, g);
}

}  // namespace aenet
