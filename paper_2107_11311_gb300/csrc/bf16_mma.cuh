// Warp-level BF16 tensor-core helpers shared by the network kernel
// (ann_bf16.cu) and the fused potential's tensor-core form: operand packing
// and splitting, the m16n8k16 product with FP32 accumulation, a small GEMM over
// fragment-ordered B operands, and the accumulator-to-A-fragment hand-off that
// keeps activations in registers between layers.
//
// Fragment layout of mma.m16n8k16 (row-major A 16x16, column-major B 16x8, FP32
// C 16x8), with g = lane / 4 and t = lane % 4:
//   A regs 0..3: (row g, k 2t..2t+1), (row g+8, k 2t..2t+1), (row g, k 2t+8..+9),
//                (row g+8, k 2t+8..+9);
//   B regs 0..1: (k 2t..2t+1, col g), (k 2t+8..+9, col g);
//   C regs 0..3: (row g, col 2t), (row g, col 2t+1), (row g+8, col 2t), (row g+8, col 2t+1).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace aenet {
namespace {

constexpr int kKD = 64;       // padded descriptor length

// Packed-weight layout (uint32 words, each = 2 BF16), per species, per part
// (hi, lo): for each GEMM a block of [k-steps][n-tiles][32 lanes][2 words].
struct PackedNet {
    int H1p, H2p;              // hidden widths padded to a multiple of 16 (H1p = H2p)
    int off_w1f, off_w2f, off_w2b, off_w1b;  // word offsets inside a species/part block
    int words;                 // words per species/part block
};

__host__ __device__ inline int pad16(int x) { return (x + 15) & ~15; }

// Both hidden layers are padded to the larger width (16 or 32), so that one
// tile shape serves every layer.
inline PackedNet make_packed(int H1, int H2) {
    PackedNet p{};
    p.H1p = pad16(H1 > H2 ? H1 : H2);
    p.H2p = p.H1p;
    int w = 0;
    p.off_w1f = w;  // K = 64, N = H1p
    w += (kKD / 16) * (p.H1p / 8) * 64;
    p.off_w2f = w;  // K = H1p, N = H2p
    w += (p.H1p / 16) * (p.H2p / 8) * 64;
    p.off_w2b = w;  // K = H2p, N = H1p
    w += (p.H2p / 16) * (p.H1p / 8) * 64;
    p.off_w1b = w;  // K = H1p, N = 64
    w += (p.H1p / 16) * (kKD / 8) * 64;
    p.words = w;
    return p;
}

__device__ inline uint32_t pack_bf2(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}

// Split (a, b) into BF16 hi and lo parts.
__device__ inline void split_bf2(float a, float b, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = pack_bf2(a - hf.x, b - hf.y);
}

__device__ inline void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// C[16 x NT*8] += A[16 x KS*16] * B, A given as hi/lo fragments per k-step.
template <int KS, int NT, bool X3>
__device__ inline void gemm(float (&C)[NT][4], const uint32_t (&Ah)[KS][4], const uint32_t (&Al)[KS][4],
                            const uint2 *__restrict__ Bh, const uint2 *__restrict__ Bl, int lane) {
#pragma unroll
    for (int ks = 0; ks < KS; ++ks)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const uint2 bh = Bh[(ks * NT + nt) * 32 + lane];
            mma_bf16(C[nt], Ah[ks], bh.x, bh.y);
            if (X3) {
                const uint2 bl = Bl[(ks * NT + nt) * 32 + lane];
                mma_bf16(C[nt], Ah[ks], bl.x, bl.y);
                mma_bf16(C[nt], Al[ks], bh.x, bh.y);
            }
        }
}

// Accumulator tiles (FP32, 16 x NT*8) -> A fragments of the next GEMM (K = NT*8).
template <int NT, bool X3>
__device__ inline void to_a(const float (&C)[NT][4], uint32_t (&Ah)[NT / 2][4], uint32_t (&Al)[NT / 2][4]) {
#pragma unroll
    for (int ks = 0; ks < NT / 2; ++ks) {
        const float *c0 = C[2 * ks], *c1 = C[2 * ks + 1];
        if (X3) {
            split_bf2(c0[0], c0[1], Ah[ks][0], Al[ks][0]);
            split_bf2(c0[2], c0[3], Ah[ks][1], Al[ks][1]);
            split_bf2(c1[0], c1[1], Ah[ks][2], Al[ks][2]);
            split_bf2(c1[2], c1[3], Ah[ks][3], Al[ks][3]);
        } else {
            Ah[ks][0] = pack_bf2(c0[0], c0[1]);
            Ah[ks][1] = pack_bf2(c0[2], c0[3]);
            Ah[ks][2] = pack_bf2(c1[0], c1[1]);
            Ah[ks][3] = pack_bf2(c1[2], c1[3]);
        }
    }
}

}  // namespace
}  // namespace aenet
