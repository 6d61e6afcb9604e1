// Device helpers of the potential kernel (potential.cu): warp reductions and
// the flags of the staged neighbour tile.
#pragma once

#include "aenet_internal.cuh"

namespace aenet {
namespace detail {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kShiftBit = 0x80000000;  // staged index flag: image shift != 0

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__device__ inline int floor_div(int a, int b) {
    int q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

// 64 per-lane partial sums -> lane l holds the warp totals of slots 2l, 2l+1.
__device__ inline void transpose_reduce64(float (&v)[64], int lane) {
#define AENET_STAGE(O, N)                                                   \
    {                                                                       \
        const bool up = (lane & (O)) != 0;                                  \
        _Pragma("unroll") for (int k = 0; k < (N); ++k) {                   \
            float send = up ? v[k] : v[k + (N)];                            \
            float keep = up ? v[k + (N)] : v[k];                            \
            v[k] = keep + __shfl_xor_sync(kFull, send, (O));                \
        }                                                                   \
    }
    AENET_STAGE(16, 32)
    AENET_STAGE(8, 16)
    AENET_STAGE(4, 8)
    AENET_STAGE(2, 4)
    AENET_STAGE(1, 2)
#undef AENET_STAGE
}

// 16 per-lane partial sums -> lanes 2q and 2q+1 each hold the total of slot q
// over the 16 lanes that share their bit 0 (one more xor-1 shuffle completes it).
__device__ inline float transpose_reduce16(float (&v)[16], int lane) {
#define AENET_STAGE(O, N)                                                   \
    {                                                                       \
        const bool up = (lane & (O)) != 0;                                  \
        _Pragma("unroll") for (int k = 0; k < (N); ++k) {                   \
            float send = up ? v[k] : v[k + (N)];                            \
            float keep = up ? v[k + (N)] : v[k];                            \
            v[k] = keep + __shfl_xor_sync(kFull, send, (O));                \
        }                                                                   \
    }
    AENET_STAGE(16, 8)
    AENET_STAGE(8, 4)
    AENET_STAGE(4, 2)
    AENET_STAGE(2, 1)
#undef AENET_STAGE
    return v[0];
}

// 32 per-lane partial sums -> lane l holds the warp total of slot l.
__device__ inline float transpose_reduce32(float (&v)[32], int lane) {
#define AENET_STAGE(O, N)                                                   \
    {                                                                       \
        const bool up = (lane & (O)) != 0;                                  \
        _Pragma("unroll") for (int k = 0; k < (N); ++k) {                   \
            float send = up ? v[k] : v[k + (N)];                            \
            float keep = up ? v[k + (N)] : v[k];                            \
            v[k] = keep + __shfl_xor_sync(kFull, send, (O));                \
        }                                                                   \
    }
    AENET_STAGE(16, 16)
    AENET_STAGE(8, 8)
    AENET_STAGE(4, 4)
    AENET_STAGE(2, 2)
    AENET_STAGE(1, 1)
#undef AENET_STAGE
    return v[0];
}

// Next (j, k) of the flattened unordered pair enumeration, k = j + 1 + rem.
__device__ inline void pair_advance(int n, int step, int &j, int &rem) {
    rem += step;
    while (j < n - 1 && rem >= n - 1 - j) {
        rem -= n - 1 - j;
        ++j;
    }
}

__device__ inline float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

}  // namespace detail
}  // namespace aenet
