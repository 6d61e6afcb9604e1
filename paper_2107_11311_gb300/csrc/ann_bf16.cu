// The precision form of the per-species networks (Sec. II.A,
// Eq. ANN-layer; two tanh hidden layers, linear output) and their
// back-propagation to dE/dG as dense BF16 tensor-core products over atoms
// grouped by species, accumulated in FP32.
//
// Atoms are grouped by species into 16-row tiles (one warp per tile). Each
// layer is one small GEMM on mma.m16n8k16 (BF16 x BF16 -> FP32):
//   forward   Z1 = g W1^T (K = D padded to 64), Z2 = X1 W2^T, E = X2 w3 + b3
//   backward  dX1 = (delta2) W2, dE/dg = (delta1) W1
// The accumulator fragment of two adjacent n8 tiles is the A fragment of the
// next k16 step, so activations never leave registers. The standardisation
// g = (G - shift) * scale and tanh' stay in FP32. AENET_BF16X3 splits every
// operand into hi + lo BF16 parts and sums hi*hi + hi*lo + lo*hi.
// Weights are packed once at set-up into fragment order (one 64-bit load per
// lane per fragment).
#include <cuda_bf16.h>

#include "aenet_internal.cuh"
#include "bf16_mma.cuh"

namespace aenet {

namespace {

constexpr int kTileRows = 16;
constexpr int kAnnWarps = 4;  // tiles per CTA

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

struct AnnBf16Args {
    int n, D, n_species;
    PackedNet pk;
    int H1, H2;
    const float *G;          // [n, D] sorted order
    const int *list;         // atoms grouped by species
    const int4 *tiles;       // (list offset, rows, species, 0)
    const int *n_tiles;
    const uint32_t *wpk;     // packed weights [species][2 parts][words]
    const float *bias;       // [species][H1p + H2p + H2p + 1]: b1, b2, w3, b3 (FP32, zero padded)
    const float *shift, *scale;  // [species][D]
    float *dEdG, *eatom;
    double *e_part;          // [max tiles]
    float *act;              // optional activation records [n, rec_len]: g, x1, d1, x2, d2
    int rec_len;
};

// Write an accumulator tile set (rows = the tile's atoms, cols = neurons < H) at
// record offset `off` of each atom's activation record.
template <int NT>
__device__ inline void store_rows(const AnnBf16Args &a, const float (&C)[NT][4], int off, int H, int s0, int s1,
                                  int tq) {
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int col = nt * 8 + 2 * tq + (e & 1);
            const int s = e < 2 ? s0 : s1;
            if (col < H && s >= 0) a.act[(size_t)s * a.rec_len + off + col] = C[nt][e];
        }
}

template <int H1T, int H2T, bool X3>
__global__ void __launch_bounds__(32 * kAnnWarps) k_ann_bf16(AnnBf16Args a) {
    constexpr int NT1 = H1T / 8, NT2 = H2T / 8, KS1 = kKD / 16, KSH1 = H1T / 16, KSH2 = H2T / 16;
    const int lane = threadIdx.x & 31;
    const int tile = blockIdx.x * kAnnWarps + (threadIdx.x >> 5);
    const int g = lane >> 2, tq = lane & 3;
    if (tile >= *a.n_tiles) {
        if (lane == 0) a.e_part[tile] = 0.0;
        return;
    }
    const int4 td = a.tiles[tile];
    const int sp = td.z;
    const int r0 = g, r1 = g + 8;
    const bool v0 = r0 < td.y, v1 = r1 < td.y;
    const int s0 = v0 ? a.list[td.x + r0] : -1, s1 = v1 ? a.list[td.x + r1] : -1;
    const int D = a.D;
    const float *sh = a.shift + sp * D, *sc = a.scale + sp * D;
    const uint32_t *wbase = a.wpk + (size_t)sp * 2 * a.pk.words;
    const uint2 *Wh = reinterpret_cast<const uint2 *>(wbase), *Wl = reinterpret_cast<const uint2 *>(wbase + a.pk.words);
    const float *bias = a.bias + sp * (a.pk.H1p + 2 * a.pk.H2p + 1);

    // ---- layer 1 input: standardised descriptor rows as A fragments (K = 64)
    uint32_t A0h[KS1][4], A0l[KS1][4];
#pragma unroll
    for (int ks = 0; ks < KS1; ++ks) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {      // column half: +0 / +8
            const int col = ks * 16 + 2 * tq + 8 * h;
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {  // row g / g + 8
                const int s = rr ? s1 : s0;
                float x0 = 0.f, x1 = 0.f;
                if (s >= 0) {
                    if (col < D) x0 = (a.G[(size_t)s * D + col] - sh[col]) * sc[col];
                    if (col + 1 < D) x1 = (a.G[(size_t)s * D + col + 1] - sh[col + 1]) * sc[col + 1];
                }
                if (a.act && s >= 0) {
                    float *rec = a.act + (size_t)s * a.rec_len;
                    if (col < D) rec[col] = x0;
                    if (col + 1 < D) rec[col + 1] = x1;
                }
                uint32_t hi, lo = 0;
                if (X3) split_bf2(x0, x1, hi, lo); else hi = pack_bf2(x0, x1);
                A0h[ks][2 * h + rr] = hi;
                A0l[ks][2 * h + rr] = lo;
            }
        }
    }
    // ---- forward
    float C1[NT1][4];
#pragma unroll
    for (int nt = 0; nt < NT1; ++nt) {
        const float b0 = bias[nt * 8 + 2 * tq], b1 = bias[nt * 8 + 2 * tq + 1];
        C1[nt][0] = b0; C1[nt][1] = b1; C1[nt][2] = b0; C1[nt][3] = b1;
    }
    gemm<KS1, NT1, X3>(C1, A0h, A0l, Wh + a.pk.off_w1f / 2, Wl + a.pk.off_w1f / 2, lane);
#pragma unroll
    for (int nt = 0; nt < NT1; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) C1[nt][e] = (nt * 8 + 2 * tq + (e & 1) < a.H1) ? tanhf(C1[nt][e]) : 0.f;
    if (a.act) store_rows<NT1>(a, C1, D, a.H1, s0, s1, tq);  // x1
    uint32_t A1h[KSH1][4], A1l[KSH1][4];
    to_a<NT1, X3>(C1, A1h, A1l);
    float C2[NT2][4];
    const float *b2 = bias + a.pk.H1p;
#pragma unroll
    for (int nt = 0; nt < NT2; ++nt) {
        const float b0 = b2[nt * 8 + 2 * tq], b1 = b2[nt * 8 + 2 * tq + 1];
        C2[nt][0] = b0; C2[nt][1] = b1; C2[nt][2] = b0; C2[nt][3] = b1;
    }
    gemm<KSH1, NT2, X3>(C2, A1h, A1l, Wh + a.pk.off_w2f / 2, Wl + a.pk.off_w2f / 2, lane);
    // output layer in FP32 on the accumulator fragments: E_row = sum_n w3_n x2_n + b3
    const float *w3 = bias + a.pk.H1p + a.pk.H2p;
    const float b3 = bias[a.pk.H1p + 2 * a.pk.H2p];
    float e0 = 0.f, e1 = 0.f;
    float D2[NT2][4];  // delta2 = (1 - x2^2) w3
#pragma unroll
    for (int nt = 0; nt < NT2; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int col = nt * 8 + 2 * tq + (e & 1);
            const float x = col < a.H2 ? tanhf(C2[nt][e]) : 0.f;
            const float w = w3[col];
            if (e < 2) e0 = fmaf(w, x, e0); else e1 = fmaf(w, x, e1);
            D2[nt][e] = (1.0f - x * x) * w;
        }
    e0 += __shfl_xor_sync(0xffffffffu, e0, 1);
    e0 += __shfl_xor_sync(0xffffffffu, e0, 2);
    e1 += __shfl_xor_sync(0xffffffffu, e1, 1);
    e1 += __shfl_xor_sync(0xffffffffu, e1, 2);
    e0 += b3;
    e1 += b3;
    if (a.act) {
        float X2[NT2][4];
#pragma unroll
        for (int nt = 0; nt < NT2; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int col = nt * 8 + 2 * tq + (e & 1);
                X2[nt][e] = col < a.H2 ? tanhf(C2[nt][e]) : 0.f;
            }
        store_rows<NT2>(a, X2, D + 2 * a.H1, a.H2, s0, s1, tq);           // x2
        store_rows<NT2>(a, D2, D + 2 * a.H1 + a.H2, a.H2, s0, s1, tq);    // delta2
    }
    // ---- backward: dX1 = delta2 W2, delta1 = (1 - x1^2) dX1, dE/dg = delta1 W1
    uint32_t A2h[KSH2][4], A2l[KSH2][4];
    to_a<NT2, X3>(D2, A2h, A2l);
    float C3[NT1][4];
#pragma unroll
    for (int nt = 0; nt < NT1; ++nt) C3[nt][0] = C3[nt][1] = C3[nt][2] = C3[nt][3] = 0.f;
    gemm<KSH2, NT1, X3>(C3, A2h, A2l, Wh + a.pk.off_w2b / 2, Wl + a.pk.off_w2b / 2, lane);
#pragma unroll
    for (int nt = 0; nt < NT1; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) C3[nt][e] *= (1.0f - C1[nt][e] * C1[nt][e]);
    if (a.act) store_rows<NT1>(a, C3, D + a.H1, a.H1, s0, s1, tq);  // delta1
    uint32_t A3h[KSH1][4], A3l[KSH1][4];
    to_a<NT1, X3>(C3, A3h, A3l);
    float C4[kKD / 8][4];
#pragma unroll
    for (int nt = 0; nt < kKD / 8; ++nt) C4[nt][0] = C4[nt][1] = C4[nt][2] = C4[nt][3] = 0.f;
    gemm<KSH1, kKD / 8, X3>(C4, A3h, A3l, Wh + a.pk.off_w1b / 2, Wl + a.pk.off_w1b / 2, lane);
    // ---- outputs: dE/dG = dE/dg * scale (FP32), E_i, tile energy partial
#pragma unroll
    for (int nt = 0; nt < kKD / 8; ++nt) {
        const int col = nt * 8 + 2 * tq;
        if (col < D) {
            if (s0 >= 0) {
                a.dEdG[(size_t)s0 * D + col] = C4[nt][0] * sc[col];
                if (col + 1 < D) a.dEdG[(size_t)s0 * D + col + 1] = C4[nt][1] * sc[col + 1];
            }
            if (s1 >= 0) {
                a.dEdG[(size_t)s1 * D + col] = C4[nt][2] * sc[col];
                if (col + 1 < D) a.dEdG[(size_t)s1 * D + col + 1] = C4[nt][3] * sc[col + 1];
            }
        }
    }
    double et = 0.0;
    if (tq == 0) {
        if (s0 >= 0) {
            a.eatom[s0] = e0;
            et += e0;
        }
        if (s1 >= 0) {
            a.eatom[s1] = e1;
            et += e1;
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) et += __shfl_xor_sync(0xffffffffu, et, o);
    if (lane == 0) a.e_part[tile] = et;
}

// ---- species grouping: count, scan into 16-row tiles, scatter
__global__ void k_species_count(int n, const float4 *__restrict__ pos4, int *__restrict__ cnt, int *__restrict__ rank) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    rank[s] = atomicAdd(&cnt[__float_as_int(pos4[s].w)], 1);
}

// Species offsets and 16-row tiles: thread 0 scans the (<= 8) species counts,
// then all threads write the tile table in parallel; counts are reset for the
// next evaluation.
__global__ void k_species_tiles(int n_species, int *__restrict__ cnt, int *__restrict__ off, int4 *__restrict__ tiles,
                                int *__restrict__ n_tiles) {
    __shared__ int s_cnt[kMaxSpecies], s_off[kMaxSpecies], s_t0[kMaxSpecies + 1];
    if (threadIdx.x == 0) {
        int o = 0, nt = 0;
        for (int t = 0; t < n_species; ++t) {
            s_cnt[t] = cnt[t];
            s_off[t] = o;
            s_t0[t] = nt;
            off[t] = o;
            o += s_cnt[t];
            nt += (s_cnt[t] + kTileRows - 1) / kTileRows;
        }
        s_t0[n_species] = nt;
        *n_tiles = nt;
    }
    __syncthreads();
    const int total = s_t0[n_species];
    for (int k = threadIdx.x; k < total; k += blockDim.x) {
        int t = 0;
        while (t + 1 < n_species && s_t0[t + 1] <= k) ++t;
        const int r = (k - s_t0[t]) * kTileRows;
        tiles[k] = make_int4(s_off[t] + r, min(kTileRows, s_cnt[t] - r), t, 0);
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

template <int H1T, int H2T>
cudaError_t launch_bf16_variant(const AnnBf16Args &a, int max_tiles, bool x3, cudaStream_t st) {
    const int blocks = (max_tiles + kAnnWarps - 1) / kAnnWarps;
    if (x3) k_ann_bf16<H1T, H2T, true><<<blocks, 32 * kAnnWarps, 0, st>>>(a);
    else k_ann_bf16<H1T, H2T, false><<<blocks, 32 * kAnnWarps, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

int bf16_max_tiles(const Context &c, int n) {
    return (n + kTileRows - 1) / kTileRows + c.basis.n_species;
}

int bf16_eparts(const Context &c, int n) {
    return (bf16_max_tiles(c, n) + kAnnWarps - 1) / kAnnWarps * kAnnWarps;
}

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
    k_species_tiles<<<1, 256, 0, c.stream>>>(c.basis.n_species, c.d_sp_cnt, c.d_sp_off, c.d_tiles, c.d_n_tiles);
    k_species_scatter<<<(n + 255) / 256, 256, 0, c.stream>>>(n, c.d_pos4, c.d_sp_off, c.d_sp_rank, c.d_sp_list);
    return cudaGetLastError();
}

cudaError_t launch_ann_bf16(Context &c, int n) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e;
    if ((e = launch_species_group(c, n)) != cudaSuccess) return e;
    AnnBf16Args a{};
    a.n = n;
    a.D = c.basis.D;
    a.n_species = c.basis.n_species;
    a.H1 = c.net.widths[1];
    a.H2 = c.net.widths[2];
    a.pk = make_packed(a.H1, a.H2);
    a.G = c.d_G;
    a.list = c.d_sp_list;
    a.tiles = c.d_tiles;
    a.n_tiles = c.d_n_tiles;
    a.wpk = reinterpret_cast<const uint32_t *>(c.d_wbf);
    a.bias = reinterpret_cast<const float *>(reinterpret_cast<const uint32_t *>(c.d_wbf) + c.wbf_elems);
    a.shift = c.d_shift;
    a.scale = c.d_scale;
    a.dEdG = c.d_dEdG;
    a.eatom = c.d_eatom;
    a.e_part = c.d_e_part;
    a.act = c.keep_act ? c.d_act : nullptr;
    a.rec_len = activation_record_len(c.net);
    const bool x3 = c.precision == AENET_BF16X3;
    const int mt = bf16_max_tiles(c, n);
    if (a.pk.H1p == 16 && a.pk.H2p == 16) return launch_bf16_variant<16, 16>(a, mt, x3, c.stream);
    if (a.pk.H1p == 32 && a.pk.H2p == 32) return launch_bf16_variant<32, 32>(a, mt, x3, c.stream);
    if (a.pk.H1p == 16 && a.pk.H2p == 32) return launch_bf16_variant<16, 32>(a, mt, x3, c.stream);
    return launch_bf16_variant<32, 16>(a, mt, x3, c.stream);
}

}  // namespace aenet
