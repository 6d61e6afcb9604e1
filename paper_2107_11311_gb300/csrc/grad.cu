// The energy gradient with respect to the network
// parameters (back-propagation, Sec. II.C), summed over the atoms of each
// species:
//   dE/dW^l[o][k] = sum_i delta^l_i[o] x^{l-1}_i[k],   dE/db^l[o] = sum_i delta^l_i[o]
// with x^0 = g (the standardised descriptor) and delta^L = 1 for the linear
// output. The network kernels leave one activation record per atom
// (g, x_l, delta_l); this kernel turns them into per-species sums.
//
// Every parameter is one product of two record entries (or of an entry and 1);
// a table built at set-up gives the two indices. CTAs take contiguous chunks of
// one species' atoms, stage their records in shared memory and accumulate their
// share of the parameters in FP32 registers; chunk partials are summed in FP64
// in a fixed order, so the result is deterministic.
#include <algorithm>
#include <vector>

#include "aenet_internal.cuh"

namespace aenet {

namespace {

constexpr int kGThreads = 256;
constexpr int kGChunk = 512;   // atoms per CTA
constexpr int kGTile = 32;     // atoms staged at a time
constexpr int kGMaxJ = 16;     // parameters per thread: n_params <= 16 * 256

__global__ void __launch_bounds__(kGThreads)
    k_dEdW_partial(int n, int n_species, int n_params, int rec_len, const int *__restrict__ list,
                   const int *__restrict__ sp_off, const float *__restrict__ act, const int2 *__restrict__ pairs,
                   float *__restrict__ partial, int n_chunks) {
    extern __shared__ float tile[];  // [kGTile][rec_len]
    const int chunk = blockIdx.x, t = blockIdx.y, tid = threadIdx.x;
    const int off = sp_off[t];
    const int cnt = (t + 1 < n_species ? sp_off[t + 1] : n) - off;
    const int a0 = chunk * kGChunk, a1 = min(cnt, a0 + kGChunk);
    float acc[kGMaxJ];
    int2 pr[kGMaxJ];
#pragma unroll
    for (int j = 0; j < kGMaxJ; ++j) {
        acc[j] = 0.f;
        const int w = tid + j * kGThreads;
        pr[j] = w < n_params ? pairs[w] : make_int2(-2, -2);
    }
    for (int b = a0; b < a1; b += kGTile) {
        const int rows = min(kGTile, a1 - b);
        __syncthreads();
        for (int k = tid; k < rows * rec_len; k += kGThreads) {
            const int r = k / rec_len, col = k % rec_len;
            tile[k] = act[(size_t)list[off + b + r] * rec_len + col];
        }
        __syncthreads();
        for (int r = 0; r < rows; ++r) {
            const float *rec = tile + r * rec_len;
#pragma unroll
            for (int j = 0; j < kGMaxJ; ++j) {
                if (pr[j].x == -2) continue;
                const float fa = pr[j].x >= 0 ? rec[pr[j].x] : 1.0f;
                const float fb = pr[j].y >= 0 ? rec[pr[j].y] : 1.0f;
                acc[j] = fmaf(fa, fb, acc[j]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kGMaxJ; ++j) {
        const int w = tid + j * kGThreads;
        if (w < n_params) partial[((size_t)t * n_chunks + chunk) * n_params + w] = acc[j];
    }
}

// out[t][w] = sum over chunks of partial[t][chunk][w], FP64, fixed order.
__global__ void k_dEdW_reduce(int n_species, int n_params, int n_chunks, const float *__restrict__ partial,
                              double *__restrict__ out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_species * n_params) return;
    const int t = idx / n_params, w = idx % n_params;
    double s0 = 0.0, s1 = 0.0;
    int c = 0;
    for (; c + 1 < n_chunks; c += 2) {
        s0 += (double)partial[((size_t)t * n_chunks + c) * n_params + w];
        s1 += (double)partial[((size_t)t * n_chunks + c + 1) * n_params + w];
    }
    if (c < n_chunks) s0 += (double)partial[((size_t)t * n_chunks + c) * n_params + w];
    out[idx] = s0 + s1;
}

}  // namespace

int grad_max_params() { return kGMaxJ * kGThreads; }

// Record indices of the two factors of every parameter, in the canonical
// per-species order W^1 b^1 W^2 b^2 ... (-1 = the constant 1).
std::vector<int2> grad_pairs(const Net &net) {
    std::vector<int> rx(net.n_layers + 1, 0), rd(net.n_layers + 1, -1);
    int r = net.widths[0];
    for (int l = 1; l < net.n_layers; ++l) {
        rx[l] = r;
        rd[l] = r + net.widths[l];
        r += 2 * net.widths[l];
    }
    std::vector<int2> p;
    for (int l = 1; l <= net.n_layers; ++l) {
        const int no = net.widths[l], ni = net.widths[l - 1];
        for (int o = 0; o < no; ++o)
            for (int k = 0; k < ni; ++k) p.push_back(make_int2(rd[l] >= 0 ? rd[l] + o : -1, l == 1 ? k : rx[l - 1] + k));
        for (int o = 0; o < no; ++o) p.push_back(make_int2(rd[l] >= 0 ? rd[l] + o : -1, -1));
    }
    return p;
}

cudaError_t launch_grad_weights(Context &c, int n) {
    const int ns = c.basis.n_species, np = c.net.n_params, rec = activation_record_len(c.net);
    const int n_chunks = std::max(1, (n + kGChunk - 1) / kGChunk);
    const size_t need = (size_t)ns * n_chunks * np;
    cudaError_t e;
    if (need > c.cap_wpart || !c.d_wpart) {
        if (c.d_wpart) cudaFree(c.d_wpart);
        c.d_wpart = nullptr;
        c.cap_wpart = 0;
        if ((e = cudaMalloc(&c.d_wpart, sizeof(float) * need)) != cudaSuccess) return e;
        c.cap_wpart = need;
    }
    if ((e = launch_species_group(c, n)) != cudaSuccess) return e;
    const size_t smem = sizeof(float) * kGTile * rec;
    if ((e = allow_max_smem(k_dEdW_partial)) != cudaSuccess) return e;
    k_dEdW_partial<<<dim3(n_chunks, ns), kGThreads, smem, c.stream>>>(
        n, ns, np, rec, c.d_sp_list, c.d_sp_off, c.d_act, c.d_wpairs, c.d_wpart, n_chunks);
    k_dEdW_reduce<<<(ns * np + 255) / 256, 256, 0, c.stream>>>(ns, np, n_chunks, c.d_wpart, c.d_dEdW);
    return cudaGetLastError();
}

}  // namespace aenet
