// The per-species networks of the three-kernel path (Sec. II.A, Eq. ANN-layer:
// two tanh hidden layers, linear output) and their back-propagation to dE/dG,
// as dense GEMMs on the fifth-generation tensor cores over atoms grouped by
// species: tcgen05.mma (BF16 x BF16, FP32 accumulation) issued by one thread
// per CTA, operands in shared memory, accumulators in tensor memory (TMEM),
// read back with tcgen05.ld for the epilogues.
//
// Persistent CTAs of 128 threads take tiles of up to 128 atoms of one species; thread r
// owns row r (atom) in every epilogue, which is exactly the TMEM lane it may
// read (warp w reads lanes 32w .. 32w + 31). Per tile, M = 128 atoms:
//   Z1 = g W1^T          K = 64 (D padded),   N = 32 (hidden padded)
//   Z2 = X1 W2^T         K = 32,              N = 32
//   dX1 = delta2 W2      K = 32,              N = 32
//   dE/dg = delta1 W1    K = 32,              N = 64
// with X1 = tanh(Z1 + b1), X2 = tanh(Z2 + b2), E = X2 w3 + b3 (FP32),
// delta2 = (1 - X2^2) w3, delta1 = (1 - X1^2) dX1. With split operands
// (AENET_BF16X3) every product is hi*hi + hi*lo + lo*hi.
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// core matrices of 8 rows x 16 bytes (8 BF16 along K), the core matrices of
// one 8-row group consecutive along K (leading byte offset 128 B), 8-row
// groups (K / 8) * 128 B apart (stride byte offset). One MMA takes K = 16,
// i.e. two core matrices along K; the next K-step starts 256 B further on.
#include <cuda_bf16.h>

#include <algorithm>

#include "aenet_internal.cuh"
#include "bf16_mma.cuh"

namespace aenet {
namespace {

constexpr int kURows = 128;  // atoms per tile: the MMA's M
constexpr int kUHid = 32;    // hidden widths padded to 32
constexpr int kUThreads = 128;
constexpr int kUCols = 128;  // TMEM columns of one CTA (three CTAs per SM: 384 of 512)

// Byte offsets of the operands in dynamic shared memory, hi part then lo part.
// The later layers' A operands reuse the g rows' space: layer 1 has read them
// by the time the first of them is written.
constexpr int kA0 = 0;                          // g rows: 128 x 64 BF16 = 16 KB per part
constexpr int kA1 = kA0;                        // x1 / delta2 / delta1 rows: 128 x 32 = 8 KB per part
constexpr int kB1 = kA0 + 2 * kURows * 64 * 2;  // W1: 32 x 64 = 4 KB per part
constexpr int kB2 = kB1 + 2 * 32 * 64 * 2;      // W2: 32 x 32 = 2 KB per part
constexpr int kB3 = kB2 + 2 * 32 * 32 * 2;      // W2^T: 32 x 32
constexpr int kB4 = kB3 + 2 * 32 * 32 * 2;      // W1^T: 64 x 32 = 4 KB per part
constexpr int kBias = kB4 + 2 * 64 * 32 * 2;    // b1 [32], b2 [32], w3 [32], b3, padding: 512 B
constexpr int kUSmem = kBias + 512;             // 56.5 KB: three CTAs per SM (four would need <= 56 KB)
// One species' weights as the kernel holds them (B operands hi and lo, then the
// biases): packed once per parameter set, brought in by one bulk copy.
constexpr int kWtcBytes = kUSmem - kB1;

// Byte offset of element (row, k) in an operand of K columns.
__device__ __forceinline__ int uoff(int row, int k, int K) {
    return (((row >> 3) * (K >> 3) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// D[128 x N] (+)= A[128 x K] B[N x K]^T over K / 16 steps; split products when X3.
template <bool X3>
__device__ __forceinline__ void umma_gemm(uint32_t d_tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                          uint32_t b_lo, int K, int N) {
    const uint32_t idesc = umma_idesc(kURows, N);
    const uint32_t a_sbo = (K >> 3) << 7, b_sbo = a_sbo;
    for (int ks = 0; ks < K / 16; ++ks) {
        const uint32_t step = ks * 256;
        umma_bf16(d_tmem, umma_desc(a_hi + step, 128, a_sbo), umma_desc(b_hi + step, 128, b_sbo), idesc, ks > 0);
        if (X3) {
            umma_bf16(d_tmem, umma_desc(a_hi + step, 128, a_sbo), umma_desc(b_lo + step, 128, b_sbo), idesc, 1);
            umma_bf16(d_tmem, umma_desc(a_lo + step, 128, a_sbo), umma_desc(b_hi + step, 128, b_sbo), idesc, 1);
        }
    }
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// Wait for phase `parity` of the mbarrier, bounded: false if it never came.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// tanh x = 1 - 2 / (exp(2x) + 1): absolute error a few 1e-7, below the BF16
// operands' rounding; exactly +-1 in the limits.
__device__ __forceinline__ float tanh_exp(float x) { return 1.0f - __fdividef(2.0f, __expf(2.0f * x) + 1.0f); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Row `row` (K = 32 values) of an A operand, split into hi and lo parts.
template <bool X3>
__device__ __forceinline__ void store_row32(unsigned char *smem, int a_off, int row, const float (&x)[32]) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint4 hi, lo;
        uint32_t *h = &hi.x, *l = &lo.x;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            if (X3) split_bf2(x[8 * c + 2 * p], x[8 * c + 2 * p + 1], h[p], l[p]);
            else h[p] = pack_bf2(x[8 * c + 2 * p], x[8 * c + 2 * p + 1]);
        }
        *reinterpret_cast<uint4 *>(smem + a_off + uoff(row, 8 * c, 32)) = hi;
        if (X3) *reinterpret_cast<uint4 *>(smem + a_off + kURows * 32 * 2 + uoff(row, 8 * c, 32)) = lo;
    }
}

struct AnnTcArgs {
    int n, D, n_species, H1, H2, rec_len, n_tiles;
    const float *G;              // [n, D] sorted order
    const unsigned char *wtc;    // [species][kWtcBytes] packed weights (k_pack_tcgen05)
    const float *shift, *scale;
    const int *list;             // atoms grouped by species
    const int *sp_off;           // [species] first list entry of each species
    float *dEdG, *eatom;
    float *act;                  // optional activation records [n, rec_len]: g, x1, d1, x2, d2
    double *e_part;              // [grid]
    unsigned *err;
};

// The weights of every species into the B-operand layout of k_ann_tcgen05 (hi
// and lo BF16 parts) and its bias block: one thread per pair of K-adjacent
// elements of one operand row, or per bias entry.
__global__ void k_pack_tcgen05(int ns, int n_params, int D, int H1, int H2, const float *__restrict__ P,
                               unsigned char *__restrict__ out) {
    constexpr int n1 = 32 * 32, n2 = 32 * 16, n4 = 64 * 16, nb = 128;
    const int per = n1 + 2 * n2 + n4 + nb;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ns * per) return;
    const int t = idx / per;
    int w = idx - t * per;
    const float *p = P + (size_t)t * n_params;
    const float *W1 = p, *b1 = W1 + H1 * D, *W2 = b1 + H1, *b2 = W2 + H2 * H1, *w3 = b2 + H2, *b3 = w3 + H2;
    unsigned char *o = out + (size_t)t * kWtcBytes - kB1;  // so that o + kBx addresses operand x
    float v0 = 0.f, v1 = 0.f;
    int off, part;
    if (w < n1) {  // W1 [n][k]: n < 32, k < 64
        const int nn = w >> 5, k = (w & 31) * 2;
        v0 = (nn < H1 && k < D) ? W1[nn * D + k] : 0.f;
        v1 = (nn < H1 && k + 1 < D) ? W1[nn * D + k + 1] : 0.f;
        off = kB1 + uoff(nn, k, 64);
        part = 32 * 64 * 2;
    } else if ((w -= n1) < n2) {  // W2 [n][k]: n < 32, k < 32
        const int nn = w >> 4, k = (w & 15) * 2;
        v0 = (nn < H2 && k < H1) ? W2[nn * H1 + k] : 0.f;
        v1 = (nn < H2 && k + 1 < H1) ? W2[nn * H1 + k + 1] : 0.f;
        off = kB2 + uoff(nn, k, 32);
        part = 32 * 32 * 2;
    } else if ((w -= n2) < n2) {  // W2^T [n][k] = W2[k][n]
        const int nn = w >> 4, k = (w & 15) * 2;
        v0 = (nn < H1 && k < H2) ? W2[k * H1 + nn] : 0.f;
        v1 = (nn < H1 && k + 1 < H2) ? W2[(k + 1) * H1 + nn] : 0.f;
        off = kB3 + uoff(nn, k, 32);
        part = 32 * 32 * 2;
    } else if ((w -= n2) < n4) {  // W1^T [c][j] = W1[j][c]: c < 64, j < 32
        const int c = w >> 4, j = (w & 15) * 2;
        v0 = (c < D && j < H1) ? W1[j * D + c] : 0.f;
        v1 = (c < D && j + 1 < H1) ? W1[(j + 1) * D + c] : 0.f;
        off = kB4 + uoff(c, j, 32);
        part = 64 * 32 * 2;
    } else {  // bias block
        w -= n4;
        float x = 0.f;
        if (w < 32) x = w < H1 ? b1[w] : 0.f;
        else if (w < 64) x = w - 32 < H2 ? b2[w - 32] : 0.f;
        else if (w < 96) x = w - 64 < H2 ? w3[w - 64] : 0.f;
        else if (w == 96) x = b3[0];
        reinterpret_cast<float *>(o + kBias)[w] = x;
        return;
    }
    uint32_t hi, lo;
    split_bf2(v0, v1, hi, lo);
    *reinterpret_cast<uint32_t *>(o + off) = hi;
    *reinterpret_cast<uint32_t *>(o + off + part) = lo;
}

// Persistent CTAs take tiles (tile k of the species groups in order) with a
// stride of the grid; a species' weights stay in shared memory until the CTA
// reaches a tile of another species.
template <bool X3>
__global__ void __launch_bounds__(kUThreads, 3) k_ann_tcgen05(AnnTcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t s_mbar[2];  // MMA completion, weight copy
    __shared__ uint32_t s_tmem;
    __shared__ double s_e[kUThreads / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float *s_bias = reinterpret_cast<const float *>(smem + kBias);  // b1, b2, w3, b3

    // ---- TMEM (warp 0 allocates) and the barriers
    const uint32_t mbar = smem_u32(&s_mbar[0]), mbar_w = smem_u32(&s_mbar[1]);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kUCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_w) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * warp) << 16);
    const uint32_t base = smem_u32(smem);
    const int D = a.D, H1 = a.H1, H2 = a.H2;
    bool ok = true;
    uint32_t phase = 0, phase_w = 0;
    int cur_t = -1;
    double e_cta = 0.0;

    auto run = [&](uint32_t d_col, int a_off, int a_K, int b_off, int b_rows, int K, int N) {
        if (tid == 0) {
            tc_fence_after();
            umma_gemm<X3>(tmem + d_col, base + a_off, base + a_off + kURows * a_K * 2, base + b_off,
                          base + b_off + b_rows * K * 2, K, N);
            umma_commit(mbar);
        }
        ok = mbar_wait(mbar, phase) && ok;
        phase ^= 1u;
        tc_fence_after();
    };

    for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
        // ---- species t and rows r0 .. r0 + rows - 1 of its group
        int t = 0, r0 = 0, cnt_t = 0;
        {
            int k = tile;
            for (t = 0; t < a.n_species; ++t) {
                cnt_t = (t + 1 < a.n_species ? a.sp_off[t + 1] : a.n) - a.sp_off[t];
                const int tiles = (cnt_t + kURows - 1) / kURows;
                if (k < tiles) break;
                k -= tiles;
            }
            if (t >= a.n_species) break;
            r0 = k * kURows;
        }
        const int rows = min(kURows, cnt_t - r0);
        // ---- this species' weights (one bulk copy) when the CTA changes species;
        // the previous tile's MMAs and bias reads are over (barrier below)
        const bool new_w = t != cur_t;
        if (new_w) {
            if (tid == 0) {
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar_w), "r"(kWtcBytes)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        base + kB1),
                    "l"(a.wtc + (size_t)t * kWtcBytes), "r"(kWtcBytes), "r"(mbar_w)
                    : "memory");
            }
            cur_t = t;
        }
        // ---- row tid: the standardised descriptor g of its atom (A0, K = 64)
        const bool valid = tid < rows;
        const int s = valid ? a.list[a.sp_off[t] + r0 + tid] : -1;
        float *rec = (a.act && valid) ? a.act + (size_t)s * a.rec_len : nullptr;
        const float *sh = a.shift + t * D, *sc = a.scale + t * D;
        const float *grow = valid ? a.G + (size_t)s * D : nullptr;
        float g[64];  // the row, all loads issued before any conversion
#pragma unroll
        for (int k = 0; k < 64; ++k) g[k] = 0.f;
        if (valid) {
            if ((D & 3) == 0) {  // rows start on 16-byte boundaries
#pragma unroll
                for (int k = 0; k < 64; k += 4)
                    if (k < D) {
                        const float4 v = *reinterpret_cast<const float4 *>(grow + k);
                        g[k] = v.x;
                        g[k + 1] = v.y;
                        g[k + 2] = v.z;
                        g[k + 3] = v.w;
                    }
            } else {
#pragma unroll
                for (int k = 0; k < 64; ++k)
                    if (k < D) g[k] = grow[k];
            }
#pragma unroll
            for (int k = 0; k < 64; ++k) {
                g[k] = k < D ? (g[k] - sh[k]) * sc[k] : 0.f;
                if (rec && k < D) rec[k] = g[k];
            }
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            uint4 hi, lo;
            uint32_t *h = &hi.x, *l = &lo.x;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                if (X3) split_bf2(g[8 * c + 2 * p], g[8 * c + 2 * p + 1], h[p], l[p]);
                else h[p] = pack_bf2(g[8 * c + 2 * p], g[8 * c + 2 * p + 1]);
            }
            *reinterpret_cast<uint4 *>(smem + kA0 + uoff(tid, 8 * c, 64)) = hi;
            if (X3) *reinterpret_cast<uint4 *>(smem + kA0 + kURows * 64 * 2 + uoff(tid, 8 * c, 64)) = lo;
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (new_w) {  // the species' weights have landed
            ok = mbar_wait(mbar_w, phase_w) && ok;
            phase_w ^= 1u;
        }
        float x1[kUHid];
        float v[32];
        // ---- layer 1: Z1 = g W1^T (TMEM columns 0..31)
        run(0, kA0, 64, kB1, 32, 64, 32);
        tmem_ld32(lane_addr + 0, v);
#pragma unroll
        for (int j = 0; j < kUHid; ++j) x1[j] = j < H1 ? tanh_exp(v[j] + s_bias[j]) : 0.f;
        store_row32<X3>(smem, kA1, tid, x1);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();

        // ---- layer 2: Z2 = X1 W2^T (columns 32..63); output layer and delta2 in FP32
        run(32, kA1, 32, kB2, 32, 32, 32);
        tmem_ld32(lane_addr + 32, v);
        float e = s_bias[3 * kUHid];
#pragma unroll
        for (int j = 0; j < kUHid; ++j) {
            const float x2 = j < H2 ? tanh_exp(v[j] + s_bias[kUHid + j]) : 0.f;
            const float w = s_bias[2 * kUHid + j];
            e = fmaf(w, x2, e);
            v[j] = (1.0f - x2 * x2) * w;  // delta2
            if (rec && j < H2) {
                rec[D + 2 * H1 + j] = x2;
                rec[D + 2 * H1 + H2 + j] = v[j];
            }
        }
        store_row32<X3>(smem, kA1, tid, v);  // the layer-2 MMAs are complete: A1 is free
        fence_async_smem();
        tc_fence_before();
        __syncthreads();

        // ---- backward: dX1 = delta2 W2 (columns 64..95), delta1 = (1 - x1^2) dX1
        run(64, kA1, 32, kB3, 32, 32, 32);
        tmem_ld32(lane_addr + 64, v);
#pragma unroll
        for (int j = 0; j < kUHid; ++j) {
            v[j] *= (1.0f - x1[j] * x1[j]);
            if (rec && j < H1) {
                rec[D + j] = x1[j];
                rec[D + H1 + j] = v[j];
            }
        }
        store_row32<X3>(smem, kA1, tid, v);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();

        // ---- dE/dg = delta1 W1 (columns 0..63), dE/dG = dE/dg * scale
        run(0, kA1, 32, kB4, 64, 32, 64);
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            tmem_ld32(lane_addr + 32 * half, v);
            if (valid) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int k = 32 * half + j;
                    if (k < D) a.dEdG[(size_t)s * D + k] = v[j] * sc[k];
                }
            }
        }
        if (valid) {
            a.eatom[s] = e;
            e_cta += (double)e;
        }
        tc_fence_before();
        __syncthreads();  // TMEM reads and A-operand reads of this tile are over
    }
    // energy partial of the CTA (FP64, fixed order)
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) e_cta += __shfl_xor_sync(0xffffffffu, e_cta, o);
    if (lane == 0) s_e[warp] = e_cta;
    if (!ok && tid == 0) atomicOr(a.err, kErrTimeout);
    tc_fence_before();
    __syncthreads();
    if (tid == 0) a.e_part[blockIdx.x] = s_e[0] + s_e[1] + s_e[2] + s_e[3];
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kUCols) : "memory");
    }
}

}  // namespace

int tcgen05_tiles(const Context &c, int n) { return (n + kURows - 1) / kURows + c.basis.n_species; }

// Persistent CTAs of the network kernel: three fit an SM (56.5 KB of shared
// memory and 128 TMEM columns each).
static int tcgen05_ctas(const Context &c, int n) { return std::min(tcgen05_tiles(c, n), 3 * std::max(1, c.n_sm)); }

int tcgen05_eparts(const Context &c, int n) { return tcgen05_ctas(c, n); }

cudaError_t pack_tcgen05_weights(Context &c) {
    const int ns = c.net.n_species;
    cudaError_t e;
    if (!c.d_wtc && (e = cudaMalloc(&c.d_wtc, (size_t)ns * kWtcBytes)) != cudaSuccess) return e;
    const int per = 32 * 32 + 2 * 32 * 16 + 64 * 16 + 128;
    k_pack_tcgen05<<<(ns * per + 255) / 256, 256, 0, c.stream>>>(ns, c.net.n_params, c.net.widths[0],
                                                                   c.net.widths[1], c.net.widths[2], c.d_params,
                                                                   c.d_wtc);
    return cudaGetLastError();
}

cudaError_t launch_ann_tcgen05(Context &c, int n) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e;
    if ((e = launch_species_group(c, n)) != cudaSuccess) return e;
    AnnTcArgs a{};
    a.n = n;
    a.D = c.basis.D;
    a.n_species = c.basis.n_species;
    a.H1 = c.net.widths[1];
    a.H2 = c.net.widths[2];
    a.rec_len = activation_record_len(c.net);
    a.n_tiles = tcgen05_tiles(c, n);
    a.G = c.d_G;
    a.wtc = c.d_wtc;
    a.shift = c.d_shift;
    a.scale = c.d_scale;
    a.list = c.d_sp_list;
    a.sp_off = c.d_sp_off;
    a.dEdG = c.d_dEdG;
    a.eatom = c.d_eatom;
    a.act = c.keep_act ? c.d_act : nullptr;
    a.e_part = c.d_e_part;
    a.err = c.d_err;
    const bool x3 = c.precision == AENET_BF16X3;
    auto kern = x3 ? k_ann_tcgen05<true> : k_ann_tcgen05<false>;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kUSmem)) != cudaSuccess) return e;
    kern<<<tcgen05_ctas(c, n), kUThreads, kUSmem, c.stream>>>(a);
    return cudaGetLastError();
}

}  // namespace aenet
