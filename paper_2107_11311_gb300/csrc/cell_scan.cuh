// Exclusive scan of the cell counts of a cell list into the cell starts, by
// the threads of one CTA (shared by the scan kernel and the MD kick + drift
// kernel, whose last CTA runs it).
#pragma once

#include "aenet_internal.cuh"

namespace aenet {

// start[c] = sum of count[0 .. c-1] for c = 0 .. ncell. Each thread takes four
// consecutive cells per pass (one 128-bit load and store), so a pass of 1,024
// threads covers 4,096 cells. The counts are read through L2 (they may come
// from other CTAs' atomics in the same kernel) and set back to zero as they
// are read, so the next binning needs no memset. blockDim.x: a multiple of 32.
__device__ inline void scan_cells_block(int ncell, int *__restrict__ count, int *__restrict__ start) {
    __shared__ int warp_sums[32];
    __shared__ int carry;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < ncell; base += 4 * blockDim.x) {
        const int i0 = base + 4 * tid;  // a multiple of 4: 16-byte aligned in both arrays
        int v[4];
        if (i0 + 3 < ncell) {
            const int4 q = __ldcg(reinterpret_cast<const int4 *>(count + i0));
            *reinterpret_cast<int4 *>(count + i0) = make_int4(0, 0, 0, 0);
            v[0] = q.x;
            v[1] = q.y;
            v[2] = q.z;
            v[3] = q.w;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                v[k] = i0 + k < ncell ? __ldcg(count + i0 + k) : 0;
                if (i0 + k < ncell) count[i0 + k] = 0;
            }
        }
        const int tot = (v[0] + v[1]) + (v[2] + v[3]);
        int x = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[wid] = x;
        __syncthreads();
        if (wid == 0) {
            const int nw = blockDim.x >> 5;
            int s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            if (lane < nw) warp_sums[lane] = s;
        }
        __syncthreads();
        const int excl = carry + (wid ? warp_sums[wid - 1] : 0) + x - tot;
        const int e1 = excl + v[0], e2 = e1 + v[1], e3 = e2 + v[2];
        if (i0 + 3 < ncell) {
            *reinterpret_cast<int4 *>(start + i0) = make_int4(excl, e1, e2, e3);
        } else {
            const int e[4] = {excl, e1, e2, e3};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (i0 + k < ncell) start[i0 + k] = e[k];
        }
        __syncthreads();  // every thread has read carry
        if (tid == blockDim.x - 1) carry = e3 + v[3];
        __syncthreads();
    }
    if (tid == 0) start[ncell] = carry;
}

}  // namespace aenet
