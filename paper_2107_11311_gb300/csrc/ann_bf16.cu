// Weights of the BF16 forms' networks (Sec. II.A, Eq. ANN-layer) in the
// operand layouts of the tensor-core kernels, packed on the device from the
// FP32 parameters (at set-up and on every parameter update, with no host round
// trip): the warp-MMA fragments of the fused kernel's 16-row tiles (below) and,
// through pack_tcgen05_weights, the shared-memory operands of the three-kernel
// path's tcgen05 network kernel. Also the grouping of atoms by species that
// the network kernel and the weight gradient use.
#include <cuda_bf16.h>

#include "aenet_internal.cuh"
#include "bf16_mma.cuh"

namespace aenet {

namespace {

// The network parameters (FP32 [species][n_params]: W1 b1 W2 b2 w3 b3, W row
// major) packed for the tensor cores, on the device: for every GEMM a block of
// [k-steps][n-tiles][32 lanes][2 words] in mma B-fragment order (lane g = l/4,
// t = l%4 holds (k 2t + 8r, 2t + 8r + 1; column g) in word r), hi and lo BF16
// parts per species; then FP32 biases b1 [H1p], b2 [H2p], w3 [H2p], b3.
//   w1f = W1^T (K = 64, N = H1p)    w2f = W2^T (K = H1p, N = H2p)
//   w2b = W2   (K = H2p, N = H1p)   w1b = W1   (K = H1p, N = 64)
// One thread per word pair (hi, lo) of one species, or per bias entry.
__global__ void k_pack_bf16(int ns, int n_params, int D, int H1, int H2, PackedNet pk, const float *__restrict__ P,
                            uint32_t *__restrict__ wpk, float *__restrict__ bias) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int per_sp = pk.words, nbias = pk.H1p + 2 * pk.H2p + 1;
    if (tid < ns * per_sp) {
        const int t = tid / per_sp, w = tid - t * per_sp;
        const float *p = P + (size_t)t * n_params;
        const float *W1 = p, *W2 = p + H1 * D + H1;
        int blk, off, N;
        if (w < pk.off_w2f) { blk = 0; off = pk.off_w1f; N = pk.H1p; }
        else if (w < pk.off_w2b) { blk = 1; off = pk.off_w2f; N = pk.H2p; }
        else if (w < pk.off_w1b) { blk = 2; off = pk.off_w2b; N = pk.H1p; }
        else { blk = 3; off = pk.off_w1b; N = kKD; }
        const int idx = w - off, r = idx & 1, lane = (idx >> 1) & 31, tile = idx >> 6;
        const int NTb = N / 8, ks = tile / NTb, nt = tile - ks * NTb;
        const int n = nt * 8 + (lane >> 2), k0 = ks * 16 + 2 * (lane & 3) + 8 * r;
        float v[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int k = k0 + e;
            float x = 0.f;
            if (blk == 0) x = (k < D && n < H1) ? W1[n * D + k] : 0.f;
            else if (blk == 1) x = (k < H1 && n < H2) ? W2[n * H1 + k] : 0.f;
            else if (blk == 2) x = (k < H2 && n < H1) ? W2[k * H1 + n] : 0.f;
            else x = (k < H1 && n < D) ? W1[k * D + n] : 0.f;
            v[e] = x;
        }
        uint32_t hi, lo;
        split_bf2(v[0], v[1], hi, lo);
        uint32_t *base = wpk + (size_t)t * 2 * per_sp;
        base[w] = hi;
        base[per_sp + w] = lo;
        return;
    }
    const int b = tid - ns * per_sp;
    if (b >= ns * nbias) return;
    const int t = b / nbias, i = b - t * nbias;
    const float *p = P + (size_t)t * n_params;
    const float *b1 = p + H1 * D, *b2 = b1 + H1 + H2 * H1, *w3 = b2 + H2, *b3 = w3 + H2;
    float x = 0.f;
    if (i < pk.H1p) x = i < H1 ? b1[i] : 0.f;
    else if (i < pk.H1p + pk.H2p) x = i - pk.H1p < H2 ? b2[i - pk.H1p] : 0.f;
    else if (i < pk.H1p + 2 * pk.H2p) x = i - pk.H1p - pk.H2p < H2 ? w3[i - pk.H1p - pk.H2p] : 0.f;
    else x = b3[0];
    bias[b] = x;
}

// ---- species grouping: count, offsets, scatter
__global__ void k_species_count(int n, const float4 *__restrict__ pos4, int *__restrict__ cnt, int *__restrict__ rank) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    rank[s] = atomicAdd(&cnt[__float_as_int(pos4[s].w)], 1);
}

// Species offsets: thread 0 scans the (<= 8) species counts, then the counts
// are reset for the next evaluation.
__global__ void k_species_offsets(int n_species, int *__restrict__ cnt, int *__restrict__ off) {
    if (threadIdx.x == 0) {
        int o = 0;
        for (int t = 0; t < n_species; ++t) {
            off[t] = o;
            o += cnt[t];
        }
    }
    __syncthreads();
    if (threadIdx.x < n_species) cnt[threadIdx.x] = 0;
}

__global__ void k_species_scatter(int n, const float4 *__restrict__ pos4, const int *__restrict__ off,
                                  const int *__restrict__ rank, int *__restrict__ list) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    list[off[__float_as_int(pos4[s].w)] + rank[s]] = s;
}

}  // namespace

bool bf16_supported(const Net &net) {
    return net.n_layers == 3 && net.widths[1] <= 32 && net.widths[2] <= 32 && net.widths[0] <= kKD;
}

cudaError_t prepare_bf16_weights(Context &c) {
    if (!bf16_supported(c.net)) return cudaErrorInvalidValue;
    const int H1 = c.net.widths[1], H2 = c.net.widths[2];
    const PackedNet pk = make_packed(H1, H2);
    const int ns = c.net.n_species;
    const size_t words = (size_t)ns * 2 * pk.words;
    const size_t nb = (size_t)ns * (pk.H1p + 2 * pk.H2p + 1);
    cudaError_t e;
    if (!c.d_wbf) {  // allocated once at set-up, reused by every parameter update
        if ((e = cudaMalloc(&c.d_wbf, sizeof(uint32_t) * words + sizeof(float) * nb)) != cudaSuccess) return e;
    }
    c.wbf_elems = words;
    uint32_t *wpk = reinterpret_cast<uint32_t *>(c.d_wbf);
    float *bias = reinterpret_cast<float *>(wpk + words);
    const int total = (int)(words / 2 + nb);
    k_pack_bf16<<<(total + 255) / 256, 256, 0, c.stream>>>(ns, c.net.n_params, c.net.widths[0], H1, H2, pk,
                                                           c.d_params, wpk, bias);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return pack_tcgen05_weights(c);  // the three-kernel path's network kernel
}

cudaError_t launch_species_group(Context &c, int n) {
    if (n <= 0) return cudaSuccess;
    k_species_count<<<(n + 255) / 256, 256, 0, c.stream>>>(n, c.d_pos4, c.d_sp_cnt, c.d_sp_rank);
    k_species_offsets<<<1, 32, 0, c.stream>>>(c.basis.n_species, c.d_sp_cnt, c.d_sp_off);
    k_species_scatter<<<(n + 255) / 256, 256, 0, c.stream>>>(n, c.d_pos4, c.d_sp_off, c.d_sp_rank, c.d_sp_list);
    return cudaGetLastError();
}

}  // namespace aenet
