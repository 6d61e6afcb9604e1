// Device code of the potential: the fused kernel k_potential (and its
// descriptor-only, forces-only and list-building forms) and the Verlet-list
// kernel k_potential_list, with their shared-memory layouts. Included by
// potential.cu (cell-list evaluation) and potential_md.cu (MD with a Verlet
// list), which are compiled in parallel; each instantiates the forms it launches.
//
// Fused potential kernel: neighbours, descriptor (Sec. II.B), network
// (Sec. II.A) and chain rule to forces and virial in one pass per atom.
//
// One CTA per cell, one warp per atom (atoms handed out dynamically inside the
// CTA). For each atom the warp
//   1. builds the neighbour list once, from the CTA's shared-memory tile of the
//      (2m+1)^3 neighbour cells (image shifts applied when staging), storing per
//      entry the displacement, r, 1/r, the radial cutoff f_c and f_c' and the
//      species weight; angular entries additionally keep the unit vector and
//      the angular f_c, f_c';
//   2. evaluates the descriptor (Sec. II.B: Eq. radial, Eq. angular over
//      unordered pairs doubled to the paper's ordered sum, the species-weighted
//      copy) in registers and reduces it across the warp;
//   3. runs its species' network (Sec. II.A, Eq. ANN-layer; tanh hidden layers,
//      linear output) warp-cooperatively in FP32 -- one lane per neuron, weights
//      in shared memory -- and back-propagates to dE/dG;
//   4. applies the chain rule through every radial term and angular pair to
//      forces (one FP32 vector atomic per neighbour entry) and the virial.
// G and dE/dG never leave the SM, the list is never rebuilt and the pair loops
// need no division or transcendental call. Energy and virial leave as FP64
// per-CTA partials, reduced in a fixed order by the reduction kernel.
//
// The same kernel in two other modes serves the split path (the BF16 network
// forms, networks wider than 32, the descriptor-only API): kDescriptor writes
// the G rows, kForces reads dE/dG rows and applies steps 1 and 4 only.
#pragma once

#include <stdio.h>

#include <algorithm>

#include "aenet_internal.cuh"
#include "bf16_mma.cuh"
#include "fp_common.cuh"
#include "sh_angular.cuh"

namespace aenet {

namespace {

using namespace detail;

constexpr int kPWarps = 8;
constexpr int kPThreads = kPWarps * 32;
constexpr int kSlots = 64;

// What one launch of k_potential computes.
enum Mode : int {
    kFused = 0,       // descriptor -> FP32 network -> forces, energy and virial
    kDescriptor = 1,  // descriptor only: G rows (sorted order)
    kForces = 2,      // forces and virial from given dE/dG rows (sorted order)
    kBuildList = 3,   // Verlet list: every image-atom within rc_max + skin (no potential)
    kFusedTC = 4,     // descriptor -> BF16 tensor-core network -> forces (one geometry pass)
    kFusedTCx3 = 5    // the same with split-BF16 operands (hi*hi + hi*lo + lo*hi)
};

__host__ __device__ constexpr bool is_tc_mode(int mode) { return mode == kFusedTC || mode == kFusedTCx3; }

// Atoms of one sub-item of the tensor-core form: a work item's atoms are taken
// in sub-items of at most this many, each in two halves of at most 16 (one
// 16-row tensor-core tile per species and half).
constexpr int kTcMaxAtoms = 32;
// Parameter block of one species in the tensor-core form: the standardisation
// shift [64] and scale [64] in slot order (the network itself is read from L2).
constexpr int kTcParStride = 2 * kSlots;
// Bounded wait of a warp for its half's network (then kErrTimeout is raised).
constexpr int kTcSpin = 1 << 22;

// Network of the tensor-core form: BF16 weights packed in mma B-fragment order
// (hi and lo parts per species, hidden widths padded to pk.H1p = pk.H2p), FP32
// biases b1 [H1p], b2 [H2p], output weights w3 [H2p] and b3 per species.
struct TcNet {
    const uint32_t *wpk = nullptr;  // [species][2][pk.words]
    const float *bias = nullptr;    // [species][H1p + 2 H2p + 1]
    PackedNet pk{};
    int H1 = 0, H2 = 0;
    int rec_len = 0;                // activation record length when records are kept
};

// Per-species parameter block in shared memory (floats), every hidden layer
// zero-padded to the compile-time width bound hb (16 or 32) so the network
// loops run a fixed trip count with no masks; padded neurons see zero weights
// and biases, so they stay at tanh(0) = 0 and contribute nothing:
//   W1  [hb][kW1Stride]    layer-1 weights, row o = neuron o over the 64 slots
//   b1  [hb]
//   for hidden l = 2..L-1: W_l [hb][hb + 4] (row o = neuron o), b_l [hb]
//   wL  [hb], bL [1]
//   shift [64 slots], scale [64 slots] (scale 0 on unused slots)
// Row strides of 4 mod 32 floats (68 = 17 x 16 B, 36 = 9 x 16 B, 20 = 5 x 16 B)
// keep the 128-bit loads of eight lanes reading eight rows free of bank
// conflicts, and a row read by all lanes at consecutive columns is too.
constexpr int kW1Stride = kSlots + 4;
struct FusedNet {
    int L;                          // weight layers
    int hb;                         // hidden-width bound of the layout (16 or 32)
    int H[kMaxLayers + 1];          // widths
    int offW[kMaxLayers + 1];       // offset of W_l in the block
    int offB[kMaxLayers + 1];       // offset of b_l
    int offShift, offScale, stride; // stride = floats per species (rounded to 4)
    int srcOff[kMaxLayers + 1];     // offset of W_l in the canonical FP32 parameters
    int n_params;                   // canonical floats per species
    int Hlast, offWL, offBL, srcOffL;  // last hidden width and output-layer offsets (scalars:
                                       // kernels never index the arrays above with runtime values)
    // per-atom activation record (for dE/dW): g [D], then x_l [H_l], delta_l [H_l]
    // for every hidden layer l
    int rec_len, rec_x[kMaxLayers], rec_d[kMaxLayers], rec_dlast;
};

inline int hidden_bound(const Net &net) {
    int h = 0;
    for (int l = 1; l < net.n_layers; ++l) h = h > net.widths[l] ? h : net.widths[l];
    return h <= 16 ? 16 : 32;
}

inline FusedNet make_fused_net(const Net &net) {
    FusedNet f{};
    f.L = net.n_layers;
    f.hb = hidden_bound(net);
    const int hb = f.hb;
    for (int l = 0; l <= net.n_layers; ++l) f.H[l] = net.widths[l];
    int p = 0;
    f.offW[1] = p;
    p += hb * kW1Stride;
    f.offB[1] = p;
    p += hb;
    for (int l = 2; l < f.L; ++l) {
        f.offW[l] = p;
        p += hb * (hb + 4);
        f.offB[l] = p;
        p += hb;
    }
    f.offW[f.L] = p;
    p += hb;
    f.offB[f.L] = p;
    p += 1;
    f.offShift = p;
    p += kSlots;
    f.offScale = p;
    p += kSlots;
    f.stride = (p + 3) & ~3;
    int q = 0;
    for (int l = 1; l <= f.L; ++l) {
        f.srcOff[l] = q;
        q += f.H[l] * f.H[l - 1] + f.H[l];
    }
    f.n_params = q;
    int r = f.H[0];
    for (int l = 1; l < f.L; ++l) {
        f.rec_x[l] = r;
        f.rec_d[l] = r + f.H[l];
        r += 2 * f.H[l];
    }
    f.rec_len = r;
    f.rec_dlast = f.rec_d[f.L - 1];
    f.Hlast = f.H[f.L - 1];
    f.offWL = f.offW[f.L];
    f.offBL = f.offB[f.L];
    f.srcOffL = f.srcOff[f.L];
    return f;
}

struct PLayout {
    size_t off_start, off_count, off_prefix, off_shift, s_pos, s_idx, params, warp_base, warp_bytes, total;
    size_t e_d, e_j, e_fx, e_fy, e_fz, a_u, a_x, a_s, coef;  // inside a warp region
    size_t tc_g, tc_cl, tc_nnb;                         // tensor-core form: rows, compact lists, counts
};

__host__ __device__ inline PLayout make_playout(int n_off, int tile, int cap, int acap, int n_species, int stride,
                                                int nw = kPWarps, bool tc = false) {
    PLayout L{};
    size_t p = 0;
    L.off_start = p;
    p = align16(p + sizeof(int) * n_off);
    L.off_count = p;
    p = align16(p + sizeof(int) * n_off);
    L.off_prefix = p;
    p = align16(p + sizeof(int) * (n_off + 1));
    L.off_shift = p;
    p = align16(p + sizeof(float4) * n_off);
    L.s_pos = p;
    p = align16(p + sizeof(float4) * tile);
    L.s_idx = p;
    p = align16(p + sizeof(int) * tile);
    L.params = p;
    p = align16(p + sizeof(float) * (size_t)n_species * stride);
    L.tc_g = L.tc_cl = L.tc_nnb = p;
    if (tc) {
        L.tc_g = p;  // [kTcMaxAtoms][64] float: standardised g, then dE/dG, in slot order
        p = align16(p + sizeof(float) * kTcMaxAtoms * kSlots);
        L.tc_cl = p;  // [kTcMaxAtoms][cap] int: staging index of every list entry
        p = align16(p + sizeof(int) * (size_t)kTcMaxAtoms * cap);
        L.tc_nnb = p;  // [kTcMaxAtoms] int: list lengths
        p = align16(p + sizeof(int) * kTcMaxAtoms);
    }
    L.warp_base = p;
    size_t q = 0;
    L.e_d = q;
    q = align16(q + sizeof(float4) * cap);
    L.e_j = q;
    q = align16(q + sizeof(int) * cap);
    L.e_fx = q;
    q = align16(q + sizeof(float) * cap);
    L.e_fy = q;
    q = align16(q + sizeof(float) * cap);
    L.e_fz = q;
    q = align16(q + sizeof(float) * cap);
    L.a_u = q;
    q = align16(q + sizeof(float4) * acap);
    L.a_x = q;
    q = align16(q + sizeof(float4) * acap);
    L.a_s = q;  // also the scratch of the spherical-harmonic angular form (kShScratch floats)
    q = align16(q + sizeof(float) * (acap > kShScratch ? acap : kShScratch));
    L.coef = q;
    q = align16(q + sizeof(float) * kSlots);
    L.warp_bytes = q;
    L.total = p + q * nw;
    return L;
}

// Descriptor slot -> G column (-1 if unused); slots are [rad | ang | rad_w | ang_w]
// of compile-time widths KRT, KAT.
template <int KRT, int KAT>
__device__ inline int slot_col(int slot, int Kr, int Ka) {
    if (slot < KRT) return slot < Kr ? slot : -1;
    if (slot < KRT + KAT) return slot - KRT < Ka ? Kr + slot - KRT : -1;
    if (slot < 2 * KRT + KAT) return slot - KRT - KAT < Kr ? Kr + Ka + slot - KRT - KAT : -1;
    if (slot < 2 * KRT + 2 * KAT) return slot - 2 * KRT - KAT < Ka ? 2 * Kr + Ka + slot - 2 * KRT - KAT : -1;
    return -1;
}

template <int KRT, int KAT>
__device__ inline bool slot_is_angular(int slot) {
    return (slot >= KRT && slot < KRT + KAT) || (slot >= 2 * KRT + KAT && slot < 2 * KRT + 2 * KAT);
}

struct WarpLists {
    float4 *e_d, *a_u, *a_x;  // e_d: (dx, dy, dz, r)
    float *a_s;               // species weight of each angular entry (also a_x.z), unit-stride for the descriptor;
                              // in the spherical-harmonic form the warp's scratch (kShScratch floats)
    int *e_j;                 // sorted neighbour index | species << 28
    float *e_fx, *e_fy, *e_fz, *coef;
};

// Phase 1 of the list build: append the image-atoms of the staged tile that
// lie within the largest cutoff of atom i, as (d, r^2) and index | species << 28.
// Only a ballot compaction runs per 32 candidates; everything per neighbour is
// deferred to the dense phase 2 (complete_list), so that the ~85% of lanes
// whose candidate is out of range do not idle through it. With CL the staging
// index of every kept entry (qbase + its index in the staged chunk) is also
// written to cl[], so that the list can be rebuilt later without a new scan.
template <bool CL = false>
__device__ __forceinline__ void scan_tile(const float4 *s_pos, const int *s_idx, int len, float4 ui, int i_s,
                                          const Basis &B, const Caps &caps, const WarpLists &W, int lane,
                                          int &nnb, int *cl = nullptr, int qbase = 0) {
    const float rc2max = B.rc_max * B.rc_max;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int base = 0; base < len; base += 32) {
        const int q = base + lane;
        bool in = false;
        float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
        int jid = 0, typ = 0;
        if (q < len) {
            const float4 p = s_pos[q];
            jid = s_idx[q];
            dx = p.x - ui.x;
            dy = p.y - ui.y;
            dz = p.z - ui.z;
            r2 = dx * dx + dy * dy + dz * dz;
            typ = __float_as_int(p.w);
            in = (r2 <= rc2max) && (jid != i_s);
        }
        const unsigned m = __ballot_sync(kFull, in);
        if (in) {
            const int slot = nnb + __popc(m & lt_mask);
            if (slot < caps.nb) {
                W.e_d[slot] = make_float4(dx, dy, dz, r2);
                W.e_j[slot] = (jid & ~kShiftBit) | (typ << 28);
                if constexpr (CL) cl[slot] = qbase + q;
            }
        }
        nnb += __popc(m);
    }
}

// Cosine cutoff of the radial term and its derivative (Eq. cos-cutoff), for
// r <= R_c: f_c = (cos(pi r / R_c) + 1) / 2, f_c' = -(pi / 2R_c) sin(pi r / R_c).
// Recomputed where needed rather than stored per entry: the per-warp lists then
// fit two CTAs per SM for networks up to 32 wide.
// The argument pi r / R_c lies in [0, pi], where the hardware sine and cosine
// (__sincosf) are accurate to ~2^-21 absolute, below the FP32 rounding of the
// sums they enter.
__device__ __forceinline__ void radial_cutoff(float r, float inv_rc, float &fc, float &dfc) {
    float sn, cs;
    __sincosf(3.14159265358979f * (r * inv_rc), &sn, &cs);
    fc = 0.5f * (cs + 1.0f);
    dfc = -0.5f * 3.14159265358979f * inv_rc * sn;
}

// Phase 2 of the list build, dense over the nnb entries: r, and the angular
// sub-list (unit vector, 1/r, angular f_c, f_c', species weight, index of the
// main entry).
__device__ __forceinline__ void complete_list(const Basis &B, const float *s_tw, const Caps &caps,
                                              const WarpLists &W, int lane, int nnb, int &nang, unsigned *err) {
    const float inv_rca = 1.0f / B.rc_ang;
    const unsigned lt_mask = (1u << lane) - 1u;
    nang = 0;
    for (int base = 0; base < nnb; base += 32) {
        const int k = base + lane;
        bool ina = false;
        float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
        float r = 0.f, inv = 0.f;
        if (k < nnb) {
            e = W.e_d[k];
            // r and 1/r from one reciprocal square root (a few ulp, far below the
            // cutoff-function and descriptor error budget)
            if (e.w < 1e-12f) {  // r < 1e-6 A
                atomicOr(err, kErrOverlap);
                r = 1e-6f;
                inv = 1e6f;
            } else {
                inv = rsqrtf(e.w);
                r = e.w * inv;
            }
            W.e_d[k].w = r;
            ina = r <= B.rc_ang;
        }
        const unsigned ma = __ballot_sync(kFull, ina);
        if (ina) {
            const int aslot = nang + __popc(ma & lt_mask);
            if (aslot < caps.ang) {
                float sn, cs;
                __sincosf(3.14159265358979f * (r * inv_rca), &sn, &cs);  // argument in [0, pi]
                W.a_u[aslot] = make_float4(e.x * inv, e.y * inv, e.z * inv, 0.5f * (cs + 1.0f));
                const float sw = s_tw[W.e_j[k] >> 28];
                W.a_x[aslot] = make_float4(inv, -0.5f * 3.14159265358979f * inv_rca * sn, sw,
                                           __int_as_float(k));
                W.a_s[aslot] = sw;
            }
        }
        nang += __popc(ma);
    }
}

// Verlet-list build: append the staged image-atoms within rc_list of atom i
// (their staged entries, index | image-offset code) to the atom's row of the
// global list; entries past the capacity are counted but not stored.
__device__ __forceinline__ void scan_tile_build(const float4 *s_pos, const int *s_idx, int len, float4 ui, int self,
                                                float rc2, int *__restrict__ row, int cap, int lane, int &nnb) {
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int base = 0; base < len; base += 32) {
        const int q = base + lane;
        bool in = false;
        int e = 0;
        if (q < len) {
            const float4 p = s_pos[q];
            e = s_idx[q];
            const float dx = p.x - ui.x, dy = p.y - ui.y, dz = p.z - ui.z;
            in = (dx * dx + dy * dy + dz * dz <= rc2) && (e != self);
        }
        const unsigned m = __ballot_sync(kFull, in);
        if (in) {
            const int slot = nnb + __popc(m & lt_mask);
            if (slot < cap) row[slot] = e;
        }
        nnb += __popc(m);
    }
}

// scan_tile_build for two atoms at once (u0 and u1; the second only if two):
// each staged image-atom is loaded once and tested against both.
__device__ __forceinline__ void scan_tile_build2(const float4 *s_pos, const int *s_idx, int len, float4 u0, float4 u1,
                                                 int self0, int self1, bool two, float rc2, int *__restrict__ row0,
                                                 int *__restrict__ row1, int cap, int lane, int &n0, int &n1) {
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int base = 0; base < len; base += 32) {
        const int q = base + lane;
        bool in0 = false, in1 = false;
        int e = 0;
        if (q < len) {
            const float4 p = s_pos[q];
            e = s_idx[q];
            const float dx0 = p.x - u0.x, dy0 = p.y - u0.y, dz0 = p.z - u0.z;
            const float dx1 = p.x - u1.x, dy1 = p.y - u1.y, dz1 = p.z - u1.z;
            in0 = (dx0 * dx0 + dy0 * dy0 + dz0 * dz0 <= rc2) && (e != self0);
            in1 = two && (dx1 * dx1 + dy1 * dy1 + dz1 * dz1 <= rc2) && (e != self1);
        }
        const unsigned m0 = __ballot_sync(kFull, in0), m1 = __ballot_sync(kFull, in1);
        if (in0) {
            const int slot = n0 + __popc(m0 & lt_mask);
            if (slot < cap) row0[slot] = e;
        }
        if (in1) {
            const int slot = n1 + __popc(m1 & lt_mask);
            if (slot < cap) row1[slot] = e;
        }
        n0 += __popc(m0);
        n1 += __popc(m1);
    }
}

__device__ __forceinline__ void store_list_count(int *vl_count, int i_s, int nnb, int cap, int lane, unsigned *err) {
    if (lane == 0) {
        vl_count[i_s] = nnb < cap ? nnb : cap;
        if (nnb > cap) atomicOr(err, kErrNbCap);
    }
}

// Phase 1 of the list build from the Verlet list: the entries of atom i that
// now lie within the largest cutoff, with the displacement computed exactly as
// from the staged tile, (u_j + offset) - u_i. The entries of kListRounds rounds
// of 32 are loaded together, then their positions together, so that a list of
// up to 32 kListRounds entries costs two dependent L2 round trips, not two per
// round; the kept entries stay in list order.
constexpr int kListRounds = 4;

__device__ __forceinline__ void scan_list(const int *__restrict__ row, int cnt, const float4 *__restrict__ pos4,
                                          const float4 *off_shift, float4 ui, int jbits, const Basis &B,
                                          const Caps &caps, const WarpLists &W, int lane, int &nnb) {
    const float rc2max = B.rc_max * B.rc_max;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int jmask = (1 << jbits) - 1;
    for (int base = 0; base < cnt; base += kListRounds * 32) {
        int e[kListRounds];
        float4 p[kListRounds];
#pragma unroll
        for (int r = 0; r < kListRounds; ++r) {
            const int k = base + 32 * r + lane;
            e[r] = k < cnt ? __ldg(row + k) : -1;  // entries are non-negative
        }
#pragma unroll
        for (int r = 0; r < kListRounds; ++r)
            p[r] = e[r] >= 0 ? pos4[e[r] & jmask] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int r = 0; r < kListRounds; ++r) {
            bool in = false;
            float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
            int j = 0, typ = 0;
            if (e[r] >= 0) {
                j = e[r] & jmask;
                const float4 sh = off_shift[e[r] >> jbits];
                dx = (p[r].x + sh.x) - ui.x;
                dy = (p[r].y + sh.y) - ui.y;
                dz = (p[r].z + sh.z) - ui.z;
                r2 = dx * dx + dy * dy + dz * dz;
                typ = __float_as_int(p[r].w);
                in = r2 <= rc2max;
            }
            const unsigned m = __ballot_sync(kFull, in);
            if (in) {
                const int slot = nnb + __popc(m & lt_mask);
                if (slot < caps.nb) {
                    W.e_d[slot] = make_float4(dx, dy, dz, r2);
                    W.e_j[slot] = j | (typ << 28);
                }
            }
            nnb += __popc(m);
        }
    }
}

// Work counters of the persistent forms: work[0] hands out items, work[1]
// counts CTAs that have left the item loop; the last one puts both back to 0,
// so the next launch finds them cleared without a memset in between.
__device__ __forceinline__ void release_work_counter(unsigned *work) {
    __threadfence();
    if (atomicAdd(&work[1], 1u) == gridDim.x - 1) {
        atomicExch(&work[0], 0u);
        atomicExch(&work[1], 0u);
    }
}

// Step it of the rotation schedule over one block pair of angular entries:
// lane l pairs its entry with column cc of block B. Inside a diagonal block
// (A = B, n_A entries) step it uses the shift t = it + 1 and pairs l with
// (l + t) mod n_A, for t = 1 .. n_A/2, the last shift only from the lower half
// of the lanes when n_A is even, so each unordered pair is visited once; across
// blocks step it pairs l with (l + it) mod 32. v: a real pair (step inside the
// range, both entries present).
__device__ __forceinline__ void rotation_step(bool diag, int it, int nt, int nA, int nB, int lane, bool vj, int &cc,
                                              bool &v) {
    if (diag) {
        const int t = it + 1;
        cc = lane + t >= nA ? lane + t - nA : lane + t;
        v = vj && it < nt && !(2 * t == nA && lane >= t);
    } else {
        cc = (lane + it) & 31;
        v = vj && it < nt && cc < nB;
    }
}

// The lane whose partner in step it is this lane's entry (inverse rotation).
__device__ __forceinline__ int rotation_source(bool diag, int it, int nA, int lane) {
    if (diag) {
        const int t = it + 1;
        return lane - t < 0 ? lane - t + nA : lane - t;
    }
    return (lane - it) & 31;
}

// S(x) = sum_q a_q T_q(x) and S'(x) = sum_q a_q T_q'(x), a_q = a0[q] + w a1[q],
// by Clenshaw's recurrence b_q = a_q + 2x b_{q+1} - b_{q+2} (S = a_0 + x b_1 -
// b_2) and its derivative b'_q = 2 b_{q+1} + 2x b'_{q+1} - b'_{q+2} (S' = b_1 +
// x b'_1 - b'_2): five operations per order instead of the six or seven of the
// forward T and U recurrences.
template <int KT>
__device__ __forceinline__ void clenshaw_d(float x, float w, const float (&a0)[KT], const float (&a1)[KT], int K,
                                           float &S, float &dS) {
    float b1 = 0.f, b2 = 0.f, d1 = 0.f, d2 = 0.f;
    const float x2 = 2.0f * x;
#pragma unroll
    for (int q = KT - 1; q >= 1; --q) {
        if (q < K) {
            const float a = fmaf(w, a1[q], a0[q]);
            const float b = fmaf(x2, b1, a - b2);
            const float d = fmaf(x2, d1, fmaf(2.0f, b1, -d2));
            b2 = b1;
            b1 = b;
            d2 = d1;
            d1 = d;
        }
    }
    S = fmaf(x, b1, fmaf(w, a1[0], a0[0]) - b2);
    dS = fmaf(x, d1, b1 - d2);
}

// Packed FP32: one FFMA2 instruction applies the same fused multiply-add to
// both halves of a float2 (each half rounded exactly as fmaf), so two
// independent recurrences advance for one issue slot.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// clenshaw_d for two arguments at once (x.x with w.x, x.y with w.y; the
// coefficient pairs hold the same value in both halves). The derivative chain
// is carried halved, D_q = b'_q / 2, so that every step is packed FMAs with
// no negated operand: D_q = 2x D_{q+1} + (b_{q+1} - D_{q+2}). The results
// equal clenshaw_d's bit for bit (scaling by 2 is exact).
template <int KT>
__device__ __forceinline__ void clenshaw_d2(float2 x, float2 w, const float2 (&a0)[KT], const float2 (&a1)[KT], int K,
                                            float2 &S, float2 &dS) {
    const float2 m1 = dup2(-1.0f), x2 = __fadd2_rn(x, x);
    float2 b1 = dup2(0.f), b2 = b1, D1 = b1, D2 = b1;
#pragma unroll
    for (int q = KT - 1; q >= 1; --q) {
        if (q < K) {
            const float2 a = ffma2(w, a1[q], a0[q]);
            const float2 b = ffma2(x2, b1, ffma2(m1, b2, a));
            const float2 D = ffma2(x2, D1, ffma2(m1, D2, b1));
            b2 = b1;
            b1 = b;
            D2 = D1;
            D1 = D;
        }
    }
    S = ffma2(x, b1, ffma2(m1, b2, ffma2(w, a1[0], a0[0])));
    dS = ffma2(x2, D1, ffma2(dup2(-2.0f), D2, b1));
}

// Chain rule through one angular term T(cos th) f_c(r_j) f_c(r_k) weighted by
// b_q = ca_q + (s_j s_k) caw_q, given c = cos th, S = sum_q b_q T_q(c) and
// dS = sum_q b_q T_q'(c): adds dE/dd_j to (jx, jy, jz) and returns dE/dd_k in
// (gx, gy, gz); nothing when v is false (uk, xk then hold any valid entry).
//   d/dd_j [T(cos) f_j f_k] = T' f_j f_k (u_k - cos u_j) / r_j + T f_j' f_k u_j
__device__ __forceinline__ void pair_gradient(const float4 &uj, const float4 &xj, const float4 uk, const float4 xk,
                                              bool v, float c, float S, float dS, float &jx, float &jy, float &jz,
                                              float &gx, float &gy, float &gz) {
    const float fj = uj.w, fk = uk.w;
    const float Af = v ? dS * fj * fk : 0.f;
    const float Aj = Af * xj.x, Ak = Af * xk.x;
    const float Bj = v ? S * xj.y * fk : 0.f, Bk = v ? S * fj * xk.y : 0.f;
    jx += Aj * (uk.x - c * uj.x) + Bj * uj.x;
    jy += Aj * (uk.y - c * uj.y) + Bj * uj.y;
    jz += Aj * (uk.z - c * uj.z) + Bj * uj.z;
    gx = Ak * (uj.x - c * uk.x) + Bk * uk.x;
    gy = Ak * (uj.y - c * uk.y) + Bk * uk.y;
    gz = Ak * (uj.z - c * uk.z) + Bk * uk.z;
}

// Spherical-harmonic form (sh_angular.cuh): the component sums of atom i's
// angular entries, A_c = sum_j w_j v_c(u_j) (and sum_j w_j^2 at 49) into
// scratch [0, 64) and B_c with s_j w_j into [64, 128): four passes (two copies,
// two column groups), each lane accumulating its entries into 32 sums that
// are then reduced across the warp (lane l: sum l).
template <int M0, int M1, bool W2>
__device__ __forceinline__ void sh_component_group(int nang, const WarpLists &W, int lane, int copy) {
    float sh[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) sh[k] = 0.f;
    for (int k = lane; k < nang; k += 32) {
        const float4 ua = W.a_u[k];
        const float wt = copy ? ua.w * W.a_x[k].z : ua.w;
        sh_accumulate<M0, M1, W2>(ua.x, ua.y, ua.z, wt, sh);
    }
    const float v = transpose_reduce32(sh, lane);
    constexpr int c0 = sh_comp(M0, M0, 0), n = (W2 ? kShComps + 1 : sh_comp(M1 + 1, M1 + 1, 0)) - c0;
    __syncwarp();  // (the scratch may still be read by an earlier phase)
    if (lane < n) W.a_s[64 * copy + c0 + lane] = v;
}

__device__ __forceinline__ void sh_component_sums(int nang, const WarpLists &W, int lane) {
#pragma unroll 1
    for (int copy = 0; copy < 2; ++copy) {
        sh_component_group<0, 2, false>(nang, W, lane, copy);
        sh_component_group<3, kShL, true>(nang, W, lane, copy);
    }
    __syncwarp();
}

// Slots of the descriptor a lane returns: the plain slot l and its
// species-weighted copy l + P (P = KRT + KAT) for l < P, else the padding slots
// 2l and 2l + 1 (zero).
template <int KRT, int KAT>
__device__ __forceinline__ int desc_slot0(int lane) {
    return lane < KRT + KAT ? lane : 2 * lane;
}
template <int KRT, int KAT>
__device__ __forceinline__ int desc_slot1(int lane) {
    return lane < KRT + KAT ? lane + KRT + KAT : 2 * lane + 1;
}

// Descriptor of atom i (Sec. II.B: Eq. radial and Eq. angular with the cosine
// cutoff, and their species-weighted copy) from its neighbour lists, reduced
// across the warp: lane l returns the coefficients of slots desc_slot0(l) and
// desc_slot1(l). A plain slot s and its weighted copy s + P take the same
// Chebyshev value times two different weights, so they share one packed
// accumulator (acc[2s], acc[2s + 1]) and one FFMA2 per term; the Chebyshev
// recurrence runs duplicated in both halves. Angular slots carry the factor 2
// of the paper's ordered-pair sum.
template <int KRT, int KAT, bool EXACT>
__device__ __forceinline__ void atom_descriptor(int nnb, int nang, const Basis &B, const float *s_tw,
                                                const float *s_sh, const WarpLists &W, int lane, float &G0,
                                                float &G1) {
    constexpr bool kSh = sh_angular<KRT, KAT, EXACT>();
    const int Kr = EXACT ? KRT : B.Kr;
    const int Ka = EXACT ? KAT : B.Ka;
    const float inv_rcr = 1.0f / B.rc_rad;
    float acc[64];  // (slot s, slot s + P) at 2s, 2s + 1 for s < P; the rest stays zero
#pragma unroll
    for (int k = 0; k < 64; ++k) acc[k] = 0.f;
    auto acc_fma = [&](int s, float2 t, float2 f) {  // acc pair s += t * f
        const float2 r = ffma2(t, f, make_float2(acc[2 * s], acc[2 * s + 1]));
        acc[2 * s] = r.x;
        acc[2 * s + 1] = r.y;
    };
    auto acc_add = [&](int s, float2 f) {
        const float2 r = __fadd2_rn(make_float2(acc[2 * s], acc[2 * s + 1]), f);
        acc[2 * s] = r.x;
        acc[2 * s + 1] = r.y;
    };
    for (int k = lane; k < nnb; k += 32) {
        const float r = W.e_d[k].w;
        if (r <= B.rc_rad) {
            float fc, dfc;
            radial_cutoff(r, inv_rcr, fc, dfc);
            const float x = 2.0f * r * inv_rcr - 1.0f;
            const float2 f = make_float2(fc, s_tw[W.e_j[k] >> 28] * fc);  // (f_c, s_j f_c)
            const float2 x2 = dup2(2.0f * x);
            float2 tm1 = dup2(1.0f), t = dup2(x);
            acc_add(0, f);
#pragma unroll
            for (int q = 1; q < KRT; ++q) {
                if (q < Kr) {
                    acc_fma(q, t, f);
                    const float2 tn = ffma2(x2, t, make_float2(-tm1.x, -tm1.y));
                    tm1 = t;
                    t = tn;
                }
            }
        }
    }
    // angular (Eq. angular): every unordered pair once by the rotation schedule
    // (see for the backward pass below); doubled to the ordered sum at the end.
    // (The spherical-harmonic form computes it after the radial reduction.)
    if constexpr (!kSh) {
        const int nbk = (nang + 31) >> 5;
        for (int A = 0; A < nbk; ++A) {
            const int nA = min(32, nang - 32 * A);
            const bool vj = lane < nA;
            const int self = 32 * A + (vj ? lane : 0);  // a valid entry: stands in for masked partners
            const float4 uj = W.a_u[self];
            const float sj = W.a_s[self];
            for (int Bk = A; Bk < nbk; ++Bk) {
                const int nB = min(32, nang - 32 * Bk);
                const bool diag = Bk == A;
                const int nt = diag ? nA / 2 : 32;
                // two rotation steps per iteration: their Chebyshev recurrences
                // are independent, which hides the FMA latency of each chain;
                // every accumulator still takes step it before step it + 1
                for (int it = 0; it < nt; it += 2) {
                    int ccA, ccB;
                    bool vA, vB;
                    rotation_step(diag, it, nt, nA, nB, lane, vj, ccA, vA);
                    rotation_step(diag, it + 1, nt, nA, nB, lane, vj, ccB, vB);
                    const int kA = vA ? 32 * Bk + ccA : self, kB = vB ? 32 * Bk + ccB : self;
                    const float4 ukA = W.a_u[kA], ukB = W.a_u[kB];
                    const float skA = W.a_s[kA], skB = W.a_s[kB];
                    const float cA = uj.x * ukA.x + uj.y * ukA.y + uj.z * ukA.z;
                    const float cB = uj.x * ukB.x + uj.y * ukB.y + uj.z * ukB.z;
                    const float wA = vA ? uj.w * ukA.w : 0.f, wB = vB ? uj.w * ukB.w : 0.f;
                    const float2 fA = make_float2(wA, wA * sj * skA), fB = make_float2(wB, wB * sj * skB);
                    const float2 xA2 = dup2(2.0f * cA), xB2 = dup2(2.0f * cB);
                    float2 tA1 = dup2(1.0f), tA = dup2(cA), tB1 = tA1, tB = dup2(cB);
                    acc_add(KRT, fA);
                    acc_add(KRT, fB);
#pragma unroll
                    for (int q = 1; q < KAT; ++q) {
                        if (q < Ka) {
                            acc_fma(KRT + q, tA, fA);
                            acc_fma(KRT + q, tB, fB);
                            const float2 tnA = ffma2(xA2, tA, make_float2(-tA1.x, -tA1.y));
                            const float2 tnB = ffma2(xB2, tB, make_float2(-tB1.x, -tB1.y));
                            tA1 = tA;
                            tA = tnA;
                            tB1 = tB;
                            tB = tnB;
                        }
                    }
                }
            }
        }
    }
    transpose_reduce64(acc, lane);  // lane l: acc[0], acc[1] = indices 2l, 2l + 1
    const int s0 = desc_slot0<KRT, KAT>(lane), s1 = desc_slot1<KRT, KAT>(lane);
    G0 = slot_is_angular<KRT, KAT>(s0) ? 2.0f * acc[0] : acc[0];
    G1 = slot_is_angular<KRT, KAT>(s1) ? 2.0f * acc[1] : acc[1];
    if constexpr (kSh) {
        // the lane of angular order a = l - KRT holds slots KRT + a (plain) and
        // 2 KRT + KAT + a (weighted): S_a = sum_l b_al Q_l - sum_j w_j^2 (the
        // ordered-pair sum itself)
        sh_component_sums(nang, W, lane);
        if (lane >= KRT && lane < KRT + KAT) {
            G0 = sh_fingerprint(W.a_s, lane - KRT, s_sh);
            G1 = sh_fingerprint(W.a_s + 64, lane - KRT, s_sh);
        }
    }
}

// Chain rule of atom i's energy through every radial term and angular pair to
// forces (one FP32 vector atomic per neighbour entry) and the virial, given
// dE/dG of the atom in slot order (coef[64], shared memory; angular slots
// without the ordered-sum factor 2, which is applied here).
template <int KRT, int KAT, bool EXACT>
__device__ __forceinline__ void atom_chain_rule(int i_s, int nnb, int nang, const Basis &B, const float *s_tw,
                                                const float *s_sh, const WarpLists &W, const float *coef, int lane,
                                                float4 *__restrict__ F4, float (&vir)[9]) {
    constexpr bool kSh = sh_angular<KRT, KAT, EXACT>();
    constexpr int SLOT_ANG = KRT, SLOT_RADW = KRT + KAT, SLOT_ANGW = 2 * KRT + KAT;
    const int Kr = EXACT ? KRT : B.Kr;
    const int Ka = EXACT ? KAT : B.Ka;
    const float inv_rcr = 1.0f / B.rc_rad;
    float cr[KRT], crw[KRT];
    float2 ca[kSh ? 1 : KAT], caw[kSh ? 1 : KAT];  // the same coefficient in both halves (packed Clenshaw of two pairs)
#pragma unroll
    for (int q = 0; q < KRT; ++q) {
        cr[q] = coef[q];
        crw[q] = coef[SLOT_RADW + q];
    }
    if constexpr (!kSh) {
#pragma unroll
        for (int q = 0; q < KAT; ++q) {  // factor 2: ordered-pair sum
            ca[q] = dup2(2.0f * coef[SLOT_ANG + q]);
            caw[q] = dup2(2.0f * coef[SLOT_ANGW + q]);
        }
    }
    const float k2 = 2.0f * inv_rcr;
    for (int k = lane; k < nnb; k += 32) {
        const float4 e = W.e_d[k];
        float fx = 0.f, fy = 0.f, fz = 0.f;
        if (e.w <= B.rc_rad) {
            float fc, dfc;
            radial_cutoff(e.w, inv_rcr, fc, dfc);
            const float s = s_tw[W.e_j[k] >> 28];
            const float x = 2.0f * e.w * inv_rcr - 1.0f;
            // d/dr [T_q(x) f_c(r)] = T_q'(x) (2/Rc) f_c + T_q f_c', summed over q with
            // the coefficients cr_q + s crw_q
            float S, dS;
            clenshaw_d<KRT>(x, s, cr, crw, Kr, S, dS);
            const float dEdr = fmaf(dS, k2 * fc, S * dfc);
            const float gr = __fdividef(dEdr, e.w);  // dE_i/dd = gr * d; force on j = -dE_i/dd
            fx = -gr * e.x;
            fy = -gr * e.y;
            fz = -gr * e.z;
        }
        W.e_fx[k] = fx;
        W.e_fy[k] = fy;
        W.e_fz[k] = fz;
    }
    __syncwarp();
    if constexpr (kSh) {
        // Spherical-harmonic form: the component sums (scratch [0, 64) plain with
        // sum w^2 at 49, [64, 128) weighted) become the coefficient pairs
        // (D_c, D'_c) = 2 N_c^2 (A_c k_l, B_c k'_l), k_l = sum_a g_a b_al, at
        // scratch [2c], [2c + 1]; then each lane takes its entries on its own
        // (dE/dd_j needs no partner), so every entry is written by one lane.
        float gsum = 0.f, gwsum = 0.f;
#pragma unroll
        for (int a = 0; a < KAT; ++a) {
            gsum += coef[SLOT_ANG + a];
            gwsum += coef[SLOT_ANGW + a];
        }
        float dv[2], dwv[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = lane + 32 * h;
            dv[h] = dwv[h] = 0.f;
            if (c < kShComps) {
                const int l = (int)s_sh[kShTabL + c];
                float kl = 0.f, klw = 0.f;
#pragma unroll
                for (int a = 0; a < KAT; ++a) {
                    const float b = s_sh[kShTabB + a * (kShL + 1) + l];
                    kl = fmaf(coef[SLOT_ANG + a], b, kl);
                    klw = fmaf(coef[SLOT_ANGW + a], b, klw);
                }
                const float n2 = 2.0f * s_sh[kShTabN + c];
                dv[h] = n2 * W.a_s[c] * kl;
                dwv[h] = n2 * W.a_s[64 + c] * klw;
            }
        }
        __syncwarp();  // every lane has read its sums
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = lane + 32 * h;
            if (c < kShComps) *reinterpret_cast<float2 *>(W.a_s + 2 * c) = make_float2(dv[h], dwv[h]);
        }
        __syncwarp();
        // (warp-uniform trip count: sh_contract synchronises the warp; lanes past
        // the last entry work on entry 0 and write nothing)
        for (int base = 0; base < nang; base += 32) {
            const int k = base + lane < nang ? base + lane : 0;
            const float4 ua = W.a_u[k], xa = W.a_x[k];  // (u, f_c), (1/r, f_c', s, entry)
            float E, Fx, Fy, Fz;
            sh_contract(ua.x, ua.y, ua.z, xa.z, W.a_s, E, Fx, Fy, Fz);
            if (base + lane < nang) {
                const float rad = xa.y * (E - 2.0f * ua.w * fmaf(xa.z * xa.z, gwsum, gsum));
                const float fu = Fx * ua.x + Fy * ua.y + Fz * ua.z;
                const float t = ua.w * xa.x;
                const int sl = __float_as_int(xa.w);  // force on neighbour = -dE_i/dd
                W.e_fx[sl] -= fmaf(rad, ua.x, t * fmaf(-fu, ua.x, Fx));
                W.e_fy[sl] -= fmaf(rad, ua.y, t * fmaf(-fu, ua.y, Fy));
                W.e_fz[sl] -= fmaf(rad, ua.z, t * fmaf(-fu, ua.z, Fz));
            }
        }
    } else {
    // Angular chain rule by the rotation schedule: the angular entries form
    // blocks of 32 (lane l owns entries 32b + l). Inside a diagonal block, step t
    // pairs lane l with entry (l + t) mod n_A (t = 1..n_A/2; at t = n_A/2 only the
    // lower half of lanes, so each unordered pair is visited once); between
    // blocks A < B, step t pairs lane l with column (l + t) mod 32 of B. The lane
    // keeps dE/dd_j of its own entry in registers and hands dE/dd_k to the owner
    // of k with one rotation shuffle; every entry is written only by its owner,
    // so no atomics are needed. Coefficients carry the factor 2 of the ordered sum.
    {
        const int nbk = (nang + 31) >> 5;
        for (int A = 0; A < nbk; ++A) {
            const int nA = min(32, nang - 32 * A);
            const bool vj = lane < nA;
            const int self = 32 * A + (vj ? lane : 0);
            const float4 uj = W.a_u[self];
            const float4 xj = W.a_x[self];
            for (int Bk = A; Bk < nbk; ++Bk) {
                const int nB = min(32, nang - 32 * Bk);
                const bool diag = Bk == A;
                const int nt = diag ? nA / 2 : 32;
                float jx = 0.f, jy = 0.f, jz = 0.f, kx = 0.f, ky = 0.f, kz = 0.f;
                for (int it = 0; it < nt; it += 2) {  // two independent steps per iteration (ILP)
                    int ccA, ccB;
                    bool vA, vB;
                    rotation_step(diag, it, nt, nA, nB, lane, vj, ccA, vA);
                    rotation_step(diag, it + 1, nt, nA, nB, lane, vj, ccB, vB);
                    const int kA = vA ? 32 * Bk + ccA : self, kB = vB ? 32 * Bk + ccB : self;
                    const float4 ukA = W.a_u[kA], xkA = W.a_x[kA], ukB = W.a_u[kB], xkB = W.a_x[kB];
                    const float2 c = make_float2(uj.x * ukA.x + uj.y * ukA.y + uj.z * ukA.z,
                                                 uj.x * ukB.x + uj.y * ukB.y + uj.z * ukB.z);
                    float2 S, dS;  // both steps' Clenshaw sums in one packed recurrence
                    clenshaw_d2<KAT>(c, make_float2(xj.z * xkA.z, xj.z * xkB.z), ca, caw, Ka, S, dS);
                    float gAx, gAy, gAz, gBx, gBy, gBz;
                    pair_gradient(uj, xj, ukA, xkA, vA, c.x, S.x, dS.x, jx, jy, jz, gAx, gAy, gAz);
                    pair_gradient(uj, xj, ukB, xkB, vB, c.y, S.y, dS.y, jx, jy, jz, gBx, gBy, gBz);
                    // dE/dd_k goes to the lane that owns k: it sits t lanes to the left
                    const int srcA = rotation_source(diag, it, nA, lane);
                    const int srcB = rotation_source(diag, it + 1, nA, lane);
                    kx += __shfl_sync(kFull, gAx, srcA);
                    ky += __shfl_sync(kFull, gAy, srcA);
                    kz += __shfl_sync(kFull, gAz, srcA);
                    kx += __shfl_sync(kFull, gBx, srcB);
                    ky += __shfl_sync(kFull, gBy, srcB);
                    kz += __shfl_sync(kFull, gBz, srcB);
                }
                // force on neighbour = -dE_i/dd; each entry is touched by its owner lane only
                if (vj) {
                    const int sl = __float_as_int(xj.w);
                    W.e_fx[sl] -= jx;
                    W.e_fy[sl] -= jy;
                    W.e_fz[sl] -= jz;
                }
                if (lane < nB) {
                    const int sl = __float_as_int(W.a_x[32 * Bk + lane].w);
                    W.e_fx[sl] -= kx;
                    W.e_fy[sl] -= ky;
                    W.e_fz[sl] -= kz;
                }
            }
        }
    }
    }  // rotation form
    __syncwarp();
    float fix = 0.f, fiy = 0.f, fiz = 0.f;
    for (int k = lane; k < nnb; k += 32) {
        const float fx = W.e_fx[k], fy = W.e_fy[k], fz = W.e_fz[k];
        const float4 e = W.e_d[k];
        atomicAdd(&F4[W.e_j[k] & 0x0fffffff], make_float4(fx, fy, fz, 0.f));
        fix -= fx;
        fiy -= fy;
        fiz -= fz;
        vir[0] = fmaf(e.x, fx, vir[0]);
        vir[1] = fmaf(e.x, fy, vir[1]);
        vir[2] = fmaf(e.x, fz, vir[2]);
        vir[3] = fmaf(e.y, fx, vir[3]);
        vir[4] = fmaf(e.y, fy, vir[4]);
        vir[5] = fmaf(e.y, fz, vir[5]);
        vir[6] = fmaf(e.z, fx, vir[6]);
        vir[7] = fmaf(e.z, fy, vir[7]);
        vir[8] = fmaf(e.z, fz, vir[8]);
    }
    fix = warp_sum(fix);
    fiy = warp_sum(fiy);
    fiz = warp_sum(fiz);
    if (lane == 0) atomicAdd(&F4[i_s], make_float4(fix, fiy, fiz, 0.f));
    __syncwarp();
}

// tanh x = 1 - 2 / (exp(2x) + 1): the fast exponential and one division instead
// of the full-accuracy tanhf, for the FP32 network and the tensor-core forms'
// epilogues. Its absolute error (a few 1e-7) is below the FP32 rounding of the
// layer sums it follows and far below the 2^-16 relative rounding of the
// split-BF16 operands; the limits x -> +-inf give exactly +-1.
__device__ __forceinline__ float tanh_exp(float x) { return 1.0f - __fdividef(2.0f, __expf(2.0f * x) + 1.0f); }

template <int KRT, int KAT, bool EXACT, int MODE, int HB>
__device__ __forceinline__ void process_atom(int i_s, int nnb, int nang, const Basis &B, const FusedNet &net,
                                             const float *s_par, const float *s_tw, const float *s_sh,
                                             const WarpLists &W, int lane,
                                             const float4 *__restrict__ pos4, float4 *__restrict__ F4,
                                             float *__restrict__ eatom, float *__restrict__ G_out,
                                             const float *__restrict__ dEdG_in, double &e_acc, float (&vir)[9]) {
    const int Kr = EXACT ? KRT : B.Kr;
    const int Ka = EXACT ? KAT : B.Ka;
    const int s0 = 2 * lane, s1 = 2 * lane + 1;  // slots of the lane's dE/dG coefficients
    if constexpr (MODE != kForces) {
    float G0, G1;  // descriptor slots g0, g1
    atom_descriptor<KRT, KAT, EXACT>(nnb, nang, B, s_tw, s_sh, W, lane, G0, G1);
    const int g0 = desc_slot0<KRT, KAT>(lane), g1 = desc_slot1<KRT, KAT>(lane);
    if constexpr (MODE == kDescriptor) {
        const int D = 2 * (Kr + Ka);
        const int c0 = slot_col<KRT, KAT>(g0, Kr, Ka), c1 = slot_col<KRT, KAT>(g1, Kr, Ka);
        if (c0 >= 0) G_out[(size_t)i_s * D + c0] = G0;
        if (c1 >= 0) G_out[(size_t)i_s * D + c1] = G1;
        return;
    } else {
    // ---- network of the atom's species (FP32, one lane per neuron)
    const int t = __float_as_int(pos4[i_s].w);
    const float *Pt = s_par + t * net.stride;
    const float *sh = Pt + net.offShift, *sc = Pt + net.offScale;
    const float x00 = (G0 - sh[g0]) * sc[g0];
    const float x01 = (G1 - sh[g1]) * sc[g1];
    // optional activation record of this atom (G_out holds records in this mode)
    float *rec = G_out ? G_out + (size_t)i_s * net.rec_len : nullptr;
    if (rec) {
        const int c0 = slot_col<KRT, KAT>(g0, Kr, Ka), c1 = slot_col<KRT, KAT>(g1, Kr, Ka);
        if (c0 >= 0) rec[c0] = x00;
        if (c1 >= 0) rec[c1] = x01;
    }
    // Lanes own neurons: o = lane for hb = 32; for hb = 16 both half-warps hold
    // neurons 0..15 (o = lane & 15) and split every sum over its inputs in two
    // halves (half h takes the h-th half), joined by one shuffle. Inputs reach
    // every lane through the warp's scratch row (W.coef, 64 floats, later the
    // dE/dG coefficients) as broadcast 128-bit loads.
    const int o = lane & (HB - 1), h = HB == 16 ? lane >> 4 : 0;
    constexpr int HS = HB + 4;                                 // hidden-layer row stride
    constexpr int NS = ((2 * (KRT + KAT) + 7) / 8) * 8;       // slots the layer-1 sums run over
    constexpr int NK1 = HB == 16 ? NS / 2 : NS;               // ... per lane group
    constexpr int NKH = HB == 16 ? 8 : 32;                    // hidden inputs per lane group
    float *xs = W.coef;
    xs[g0] = x00;
    xs[g1] = x01;
    __syncwarp();
    const float *W1 = Pt + net.offW[1];
    float z;
    {
        const float *wr = W1 + o * kW1Stride + h * NK1, *gx = xs + h * NK1;
        // two partial sums (even and odd inputs) in the halves of one packed accumulator;
        // partial unrolling: all loads hoisted ahead of the FMAs would need ~100 registers
        float2 zab = dup2(0.f);
#pragma unroll 2
        for (int k = 0; k < NK1; k += 4) {
            const float4 gv = *reinterpret_cast<const float4 *>(gx + k);
            const float4 wv = *reinterpret_cast<const float4 *>(wr + k);
            zab = ffma2(make_float2(wv.x, wv.y), make_float2(gv.x, gv.y), zab);
            zab = ffma2(make_float2(wv.z, wv.w), make_float2(gv.z, gv.w), zab);
        }
        z = zab.x + zab.y;
        if constexpr (HB == 16) z += __shfl_xor_sync(kFull, z, 16);
    }
    float xl[kMaxLayers];  // this lane's neuron of every hidden layer
    xl[1] = tanh_exp(z + Pt[net.offB[1] + o]);
    if (rec && lane < net.H[1]) rec[net.rec_x[1] + lane] = xl[1];
#pragma unroll
    for (int l = 2; l < kMaxLayers; ++l) {
        if (l < net.L) {
            __syncwarp();  // the previous reads of the scratch row are done
            if (lane < HB) xs[lane] = xl[l - 1];
            __syncwarp();
            const float *wr = Pt + net.offW[l] + o * HS + h * NKH, *xv = xs + h * NKH;
            float2 zab = dup2(0.f);
#pragma unroll 2
            for (int k = 0; k < NKH; k += 4) {
                const float4 gv = *reinterpret_cast<const float4 *>(xv + k);
                const float4 wv = *reinterpret_cast<const float4 *>(wr + k);
                zab = ffma2(make_float2(wv.x, wv.y), make_float2(gv.x, gv.y), zab);
                zab = ffma2(make_float2(wv.z, wv.w), make_float2(gv.z, gv.w), zab);
            }
            float zz = zab.x + zab.y;
            if constexpr (HB == 16) zz += __shfl_xor_sync(kFull, zz, 16);
            xl[l] = tanh_exp(zz + Pt[net.offB[l] + o]);
            if (rec && lane < net.H[l]) rec[net.rec_x[l] + lane] = xl[l];
        }
    }
    float xlast = 0.f;
#pragma unroll
    for (int l = 1; l < kMaxLayers; ++l)
        if (l == net.L - 1) xlast = xl[l];
    const float wL = Pt[net.offWL + o];
    float E = wL * xlast;
#pragma unroll
    for (int m = HB / 2; m >= 1; m >>= 1) E += __shfl_xor_sync(kFull, E, m);
    E += Pt[net.offBL];
    // back-propagation: delta of the last hidden layer, then down to layer 1;
    // lane k collects dx_k = sum_q W_l[q][k] delta_q over the broadcast deltas
    float delta = (1.0f - xlast * xlast) * wL;
    if (rec && lane < net.Hlast) rec[net.rec_dlast + lane] = delta;
#pragma unroll
    for (int l = kMaxLayers - 1; l >= 2; --l) {
        if (l < net.L) {
            __syncwarp();
            if (lane < HB) xs[lane] = delta;
            __syncwarp();
            const float *wc = Pt + net.offW[l] + h * NKH * HS + o, *dv = xs + h * NKH;
            float2 dab = dup2(0.f);
#pragma unroll 2
            for (int q = 0; q < NKH; q += 4) {
                const float4 d4 = *reinterpret_cast<const float4 *>(dv + q);
                dab = ffma2(make_float2(wc[(q + 0) * HS], wc[(q + 1) * HS]), make_float2(d4.x, d4.y), dab);
                dab = ffma2(make_float2(wc[(q + 2) * HS], wc[(q + 3) * HS]), make_float2(d4.z, d4.w), dab);
            }
            float dx = dab.x + dab.y;
            if constexpr (HB == 16) dx += __shfl_xor_sync(kFull, dx, 16);
            delta = (1.0f - xl[l - 1] * xl[l - 1]) * dx;
            if (rec && lane < net.H[l - 1]) rec[net.rec_d[l - 1] + lane] = delta;
        }
    }
    // dE/dg of this lane's slots 2l, 2l + 1: sum_q W1[q][slot] delta1_q, both
    // slots in one packed accumulator (two, over even and odd q); the row holds
    // every delta twice, so that each 128-bit load gives two (delta, delta) pairs
    __syncwarp();
    if (lane < HB) *reinterpret_cast<float2 *>(xs + 2 * lane) = dup2(delta);
    __syncwarp();
    float2 dd = dup2(0.f), ee = dd;
#pragma unroll 2
    for (int q = 0; q < HB; q += 4) {
        const float4 d01 = *reinterpret_cast<const float4 *>(xs + 2 * q);
        const float4 d23 = *reinterpret_cast<const float4 *>(xs + 2 * q + 4);
        const float2 w0 = *reinterpret_cast<const float2 *>(W1 + (q + 0) * kW1Stride + 2 * lane);
        const float2 w1 = *reinterpret_cast<const float2 *>(W1 + (q + 1) * kW1Stride + 2 * lane);
        const float2 w2 = *reinterpret_cast<const float2 *>(W1 + (q + 2) * kW1Stride + 2 * lane);
        const float2 w3 = *reinterpret_cast<const float2 *>(W1 + (q + 3) * kW1Stride + 2 * lane);
        dd = ffma2(w0, make_float2(d01.x, d01.y), dd);
        ee = ffma2(w1, make_float2(d01.z, d01.w), ee);
        dd = ffma2(w2, make_float2(d23.x, d23.y), dd);
        ee = ffma2(w3, make_float2(d23.z, d23.w), ee);
    }
    const float d0 = dd.x + ee.x, d1 = dd.y + ee.y;
    __syncwarp();  // every lane has read the deltas: the row takes the coefficients
    W.coef[s0] = d0 * sc[s0];  // dE/dG = dE/dg * scale
    W.coef[s1] = d1 * sc[s1];
    if (lane == 0) {
        e_acc += (double)E;
        eatom[i_s] = E;
    }
    }  // MODE == kFused
    }  // MODE != kForces
    if constexpr (MODE == kForces) {  // dE/dG given: scatter the row into the slot layout
        const int D = 2 * (Kr + Ka);
        const int c0 = slot_col<KRT, KAT>(s0, Kr, Ka), c1 = slot_col<KRT, KAT>(s1, Kr, Ka);
        W.coef[s0] = c0 >= 0 ? dEdG_in[(size_t)i_s * D + c0] : 0.f;
        W.coef[s1] = c1 >= 0 ? dEdG_in[(size_t)i_s * D + c1] : 0.f;
        // the spherical-harmonic chain rule needs the atom's component sums,
        // which no descriptor pass has left in this launch
        if constexpr (sh_angular<KRT, KAT, EXACT>()) sh_component_sums(nang, W, lane);
    }
    __syncwarp();

    atom_chain_rule<KRT, KAT, EXACT>(i_s, nnb, nang, B, s_tw, s_sh, W, W.coef, lane, F4, vir);
}

// The network parameters of every species into the shared-memory layout of
// FusedNet (zero-padded to the width bound; slots mapped to G columns).
template <int KRT, int KAT, bool EXACT>
__device__ __forceinline__ void load_net_params(const Basis &B, const FusedNet &net, const float *__restrict__ params,
                                                const float *__restrict__ shift, const float *__restrict__ scale,
                                                float *s_par, int tid, int nthreads) {
    const int Kr = EXACT ? KRT : B.Kr, Ka = EXACT ? KAT : B.Ka, D = 2 * (Kr + Ka);
    for (int t = 0; t < B.n_species; ++t) {
        const float *src = params + (size_t)t * net.n_params;
        float *dst = s_par + t * net.stride;
        const int H1 = net.H[1], hb = net.hb;
        for (int idx = tid; idx < hb * kW1Stride; idx += nthreads) {  // W1: (neuron, slot)
            const int o = idx / kW1Stride, slot = idx - o * kW1Stride;
            const int col = slot < kSlots ? slot_col<KRT, KAT>(slot, Kr, Ka) : -1;
            dst[net.offW[1] + idx] = (o < H1 && col >= 0) ? src[net.srcOff[1] + o * D + col] : 0.f;
        }
        for (int o = tid; o < hb; o += nthreads) dst[net.offB[1] + o] = o < H1 ? src[net.srcOff[1] + H1 * D + o] : 0.f;
#pragma unroll
        for (int l = 2; l < kMaxLayers; ++l) {
            if (l >= net.L) break;
            const int Hi = net.H[l - 1], Ho = net.H[l];
            for (int idx = tid; idx < hb * (hb + 4); idx += nthreads) {
                const int o = idx / (hb + 4), k = idx % (hb + 4);
                dst[net.offW[l] + idx] = (o < Ho && k < Hi) ? src[net.srcOff[l] + o * Hi + k] : 0.f;
            }
            for (int o = tid; o < hb; o += nthreads)
                dst[net.offB[l] + o] = o < Ho ? src[net.srcOff[l] + Ho * Hi + o] : 0.f;
        }
        const int Hl = net.Hlast;
        for (int k = tid; k < hb; k += nthreads) dst[net.offWL + k] = k < Hl ? src[net.srcOffL + k] : 0.f;
        if (tid == 0) dst[net.offBL] = src[net.srcOffL + Hl];
        for (int slot = tid; slot < kSlots; slot += nthreads) {
            const int col = slot_col<KRT, KAT>(slot, Kr, Ka);
            dst[net.offShift + slot] = col >= 0 ? shift[t * D + col] : 0.f;
            dst[net.offScale + slot] = col >= 0 ? scale[t * D + col] : 0.f;
        }
    }
}

// Standardisation of every species in slot order for the tensor-core form:
// shift at [t][slot], scale at [t][64 + slot] (scale 0 on unused slots).
template <int KRT, int KAT, bool EXACT>
__device__ __forceinline__ void load_tc_params(const Basis &B, const float *__restrict__ shift,
                                               const float *__restrict__ scale, float *s_par, int tid, int nthreads) {
    const int Kr = EXACT ? KRT : B.Kr, Ka = EXACT ? KAT : B.Ka, D = 2 * (Kr + Ka);
    for (int idx = tid; idx < B.n_species * kSlots; idx += nthreads) {
        const int t = idx / kSlots, slot = idx - t * kSlots;
        const int col = slot_col<KRT, KAT>(slot, Kr, Ka);
        s_par[t * kTcParStride + slot] = col >= 0 ? shift[t * D + col] : 0.f;
        s_par[t * kTcParStride + kSlots + slot] = col >= 0 ? scale[t * D + col] : 0.f;
    }
}

// Position of the r-th set bit of mask (r from 0), or -1.
__device__ __forceinline__ int nth_bit(unsigned mask, int r) {
    for (int k = 0; k < r && mask; ++k) mask &= mask - 1u;
    return mask ? __ffs(mask) - 1 : -1;
}

// The network of one species (Sec. II.A, Eq. ANN-layer: two tanh hidden layers,
// linear output) and its back-propagation to dE/dG, on the tensor cores, for up
// to 16 atoms of that species: rows r = lane/4 and r + 8 of the mma tiles are
// the atoms a0 and a1 (sub-item indices, -1 for an empty row). Each layer is
// one small GEMM on mma.m16n8k16 (BF16 x BF16 -> FP32), operands split into
// hi + lo parts when X3 (hi*hi + hi*lo + lo*hi):
//   forward   Z1 = g W1^T + b1, X1 = tanh Z1; Z2 = X1 W2^T + b2, X2 = tanh Z2;
//             E = X2 w3 + b3 (FP32)
//   backward  delta2 = (1 - X2^2) w3; delta1 = (1 - X1^2) (delta2 W2); dE/dg = delta1 W1
// Input: the standardised rows g in s_g (slot order; slot = G column for the
// bases this form serves); output: dE/dG = dE/dg * scale written over the same
// rows, E_i to eatom and the warp's energy sum, and, when rec_base is given,
// the activation record (g, x1, delta1, x2, delta2) of every atom for dE/dW.
template <int HT, bool X3>
__device__ __forceinline__ void tc_tile_chain(int t, int a0, int a1, int lane, float *s_g, const float *sc,
                                              const TcNet &tn, int atom0, float *__restrict__ eatom,
                                              float *__restrict__ rec_base, int D, double &e_acc) {
    constexpr int NT = HT / 8, KS1 = kKD / 16, KSH = HT / 16, NTD = kKD / 8;
    const int tq = lane & 3;
    const uint32_t *wbase = tn.wpk + (size_t)t * 2 * tn.pk.words;
    const uint2 *Wh = reinterpret_cast<const uint2 *>(wbase);
    const uint2 *Wl = reinterpret_cast<const uint2 *>(wbase + tn.pk.words);
    const float *bias = tn.bias + t * (tn.pk.H1p + 2 * tn.pk.H2p + 1);
    float *rec0 = (rec_base && a0 >= 0) ? rec_base + (size_t)(atom0 + a0) * tn.rec_len : nullptr;
    float *rec1 = (rec_base && a1 >= 0) ? rec_base + (size_t)(atom0 + a1) * tn.rec_len : nullptr;
    const int H1 = tn.H1, H2 = tn.H2;

    // ---- layer 1: Z1 = b1 + g W1^T, the A fragments of g built per k-step from
    // the standardised rows (K = 64)
    float C1[NT][4];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const float b0 = bias[nt * 8 + 2 * tq], b1 = bias[nt * 8 + 2 * tq + 1];
        C1[nt][0] = b0; C1[nt][1] = b1; C1[nt][2] = b0; C1[nt][3] = b1;
    }
    {
        const uint2 *Bh = Wh + tn.pk.off_w1f / 2, *Bl = Wl + tn.pk.off_w1f / 2;
#pragma unroll
        for (int ks = 0; ks < KS1; ++ks) {
            uint32_t ah[4], al[4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int col = ks * 16 + 2 * tq + 8 * h;
#pragma unroll
                for (int rr = 0; rr < 2; ++rr) {
                    const int a = rr ? a1 : a0;
                    float *rec = rr ? rec1 : rec0;
                    float2 v = make_float2(0.f, 0.f);
                    if (a >= 0) v = *reinterpret_cast<const float2 *>(s_g + a * kSlots + col);
                    if (rec) {
                        if (col < D) rec[col] = v.x;
                        if (col + 1 < D) rec[col + 1] = v.y;
                    }
                    uint32_t hi, lo = 0u;
                    if (X3) split_bf2(v.x, v.y, hi, lo); else hi = pack_bf2(v.x, v.y);
                    ah[2 * h + rr] = hi;
                    al[2 * h + rr] = lo;
                }
            }
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const uint2 bh = Bh[(ks * NT + nt) * 32 + lane];
                mma_bf16(C1[nt], ah, bh.x, bh.y);
                if (X3) {
                    const uint2 bl = Bl[(ks * NT + nt) * 32 + lane];
                    mma_bf16(C1[nt], ah, bl.x, bl.y);
                    mma_bf16(C1[nt], al, bh.x, bh.y);
                }
            }
        }
    }
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) C1[nt][e] = (nt * 8 + 2 * tq + (e & 1) < H1) ? tanh_exp(C1[nt][e]) : 0.f;

    // ---- layer 2 and the linear output layer (FP32): delta2 = (1 - x2^2) w3
    float D2[NT][4];
    float e0 = 0.f, e1 = 0.f;
    {
        uint32_t A1h[KSH][4], A1l[KSH][4];
        to_a<NT, X3>(C1, A1h, A1l);
        float C2[NT][4];
        const float *b2 = bias + tn.pk.H1p;
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const float b0 = b2[nt * 8 + 2 * tq], b1 = b2[nt * 8 + 2 * tq + 1];
            C2[nt][0] = b0; C2[nt][1] = b1; C2[nt][2] = b0; C2[nt][3] = b1;
        }
        gemm<KSH, NT, X3>(C2, A1h, A1l, Wh + tn.pk.off_w2f / 2, Wl + tn.pk.off_w2f / 2, lane);
        const float *w3 = bias + tn.pk.H1p + tn.pk.H2p;
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int col = nt * 8 + 2 * tq + (e & 1);
                const float x = col < H2 ? tanh_exp(C2[nt][e]) : 0.f;
                const float w = w3[col];
                if (e < 2) e0 = fmaf(w, x, e0); else e1 = fmaf(w, x, e1);
                D2[nt][e] = (1.0f - x * x) * w;
                float *rec = e < 2 ? rec0 : rec1;
                if (rec && col < H2) {  // x2 and delta2 of the record
                    rec[D + 2 * H1 + col] = x;
                    rec[D + 2 * H1 + H2 + col] = D2[nt][e];
                }
            }
    }
    e0 += __shfl_xor_sync(kFull, e0, 1);
    e0 += __shfl_xor_sync(kFull, e0, 2);
    e1 += __shfl_xor_sync(kFull, e1, 1);
    e1 += __shfl_xor_sync(kFull, e1, 2);
    const float b3 = bias[tn.pk.H1p + 2 * tn.pk.H2p];
    e0 += b3;
    e1 += b3;

    // ---- backward: delta1 = (1 - x1^2) (delta2 W2)
    uint32_t A3h[KSH][4], A3l[KSH][4];
    {
        uint32_t A2h[KSH][4], A2l[KSH][4];
        to_a<NT, X3>(D2, A2h, A2l);
        float C3[NT][4];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) C3[nt][0] = C3[nt][1] = C3[nt][2] = C3[nt][3] = 0.f;
        gemm<KSH, NT, X3>(C3, A2h, A2l, Wh + tn.pk.off_w2b / 2, Wl + tn.pk.off_w2b / 2, lane);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                C3[nt][e] *= (1.0f - C1[nt][e] * C1[nt][e]);
                const int col = nt * 8 + 2 * tq + (e & 1);
                float *rec = e < 2 ? rec0 : rec1;
                if (rec && col < H1) {  // x1 and delta1 of the record
                    rec[D + col] = C1[nt][e];
                    rec[D + H1 + col] = C3[nt][e];
                }
            }
        to_a<NT, X3>(C3, A3h, A3l);
    }

    // ---- dE/dg = delta1 W1, in two halves of the 64 columns; dE/dG = dE/dg *
    // scale written over the rows g was read from (every (row, column) pair
    // belongs to one lane, which has already read its inputs)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        float C4[NTD / 2][4];
#pragma unroll
        for (int j = 0; j < NTD / 2; ++j) C4[j][0] = C4[j][1] = C4[j][2] = C4[j][3] = 0.f;
        const uint2 *Bh = Wh + tn.pk.off_w1b / 2, *Bl = Wl + tn.pk.off_w1b / 2;
#pragma unroll
        for (int ks = 0; ks < KSH; ++ks)
#pragma unroll
            for (int j = 0; j < NTD / 2; ++j) {
                const int nt = half * (NTD / 2) + j;
                const uint2 bh = Bh[(ks * NTD + nt) * 32 + lane];
                mma_bf16(C4[j], A3h[ks], bh.x, bh.y);
                if (X3) {
                    const uint2 bl = Bl[(ks * NTD + nt) * 32 + lane];
                    mma_bf16(C4[j], A3h[ks], bl.x, bl.y);
                    mma_bf16(C4[j], A3l[ks], bh.x, bh.y);
                }
            }
#pragma unroll
        for (int j = 0; j < NTD / 2; ++j) {
            const int col = (half * (NTD / 2) + j) * 8 + 2 * tq;
            const float2 s2 = *reinterpret_cast<const float2 *>(sc + col);
            if (a0 >= 0)
                *reinterpret_cast<float2 *>(s_g + a0 * kSlots + col) = make_float2(C4[j][0] * s2.x, C4[j][1] * s2.y);
            if (a1 >= 0)
                *reinterpret_cast<float2 *>(s_g + a1 * kSlots + col) = make_float2(C4[j][2] * s2.x, C4[j][3] * s2.y);
        }
    }
    // E_i of the tile's atoms; their FP64 sum joins the warp's energy (lane 0)
    double et = 0.0;
    if (tq == 0) {
        if (a0 >= 0) {
            eatom[atom0 + a0] = e0;
            et += (double)e0;
        }
        if (a1 >= 0) {
            eatom[atom0 + a1] = e1;
            et += (double)e1;
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) et += __shfl_xor_sync(kFull, et, o);
    if (lane == 0) e_acc += et;
}

// Networks of the cnt atoms of one species in a sub-item whose first atom is
// the sorted atom atom0: order[0 .. cnt) are their sub-item indices, taken in
// tiles of 16 rows.
template <int HT, bool X3>
__device__ __noinline__ void tc_species_network(int t, const int *order, int cnt, int atom0, int lane,
                                                   float *s_g, const float *s_par, const TcNet &tn,
                                                   float *__restrict__ eatom, float *__restrict__ rec_base, int D,
                                                   double &e_acc) {
    const int g = lane >> 2;
    for (int r0 = 0; r0 < cnt; r0 += 16) {
        const int a0 = r0 + g < cnt ? order[r0 + g] : -1;
        const int a1 = r0 + g + 8 < cnt ? order[r0 + g + 8] : -1;
        tc_tile_chain<HT, X3>(t, a0, a1, lane, s_g, s_par + t * kTcParStride + kSlots, tn, atom0, eatom, rec_base,
                              D, e_acc);
    }
}

template <int KRT, int KAT, bool EXACT, int MODE, bool BATCH, int HB, int NW = kPWarps>
// (the list-build mode keeps no per-warp state: 32 registers give it eight CTAs per SM)
__global__ void __launch_bounds__(NW * 32, MODE == kBuildList ? 8 : (NW == kPWarps ? 2 : 1))
    k_potential(Basis B, FusedNet net, Grid g_one, const StructInfo *__restrict__ sinfo, int n_struct, Caps caps,
                const float4 *__restrict__ pos4,
                const int *__restrict__ cell_start, const float *__restrict__ params, const float *__restrict__ shift,
                const float *__restrict__ scale, float4 *__restrict__ F4, float *__restrict__ eatom,
                float *__restrict__ G_out, const float *__restrict__ dEdG_in, double *__restrict__ e_part,
                double *__restrict__ vir_part, unsigned long long *__restrict__ stats, unsigned *__restrict__ err,
                unsigned *__restrict__ work, const int *__restrict__ order, int n_items, int *__restrict__ vl_out,
                int *__restrict__ vl_count, int split, int split_from, TcNet tc) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float s_tw[kMaxSpecies];
    __shared__ float s_sh[sh_angular<KRT, KAT, EXACT>() ? kShTab : 1];  // spherical-harmonic form's table
    __shared__ float s_vir[NW][9];
    __shared__ double s_e[NW];
    __shared__ int s_next, s_item;
    __shared__ int s_kept, s_wcnt[NW];  // staged image-atoms of the chunk; per-warp counts while staging
    // tensor-core form: per species of the sub-item, atoms through phase A and
    // network done; the sub-item's atoms in species order, and each species'
    // first position and count in that order
    __shared__ int s_tc_done_a[kMaxSpecies], s_tc_done_b[kMaxSpecies];
    __shared__ int s_tc_order[kTcMaxAtoms], s_tc_first[kMaxSpecies], s_tc_count[kMaxSpecies];
    constexpr bool kTC = is_tc_mode(MODE);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = caps.tile;
    // one layout for every cell: sized for the largest image-offset table
    // (g_one.n_off is that maximum in a batch)
    // (the list-build form keeps no per-warp lists: its CTAs are small)
    constexpr bool kLists = MODE != kBuildList;
    const PLayout L = make_playout(g_one.n_off, tile, kLists ? caps.nb : 0, kLists ? caps.ang : 0,
                                   (MODE == kFused || kTC) ? B.n_species : 0, kTC ? kTcParStride : net.stride, NW,
                                   kTC);
    int *off_start = reinterpret_cast<int *>(smem + L.off_start);
    int *off_count = reinterpret_cast<int *>(smem + L.off_count);
    int *off_prefix = reinterpret_cast<int *>(smem + L.off_prefix);
    float4 *off_shift = reinterpret_cast<float4 *>(smem + L.off_shift);
    float4 *s_pos = reinterpret_cast<float4 *>(smem + L.s_pos);
    int *s_idx = reinterpret_cast<int *>(smem + L.s_idx);
    float *s_par = reinterpret_cast<float *>(smem + L.params);
    unsigned char *wb = smem + L.warp_base + L.warp_bytes * warp;
    WarpLists W;
    W.e_d = reinterpret_cast<float4 *>(wb + L.e_d);
    W.e_j = reinterpret_cast<int *>(wb + L.e_j);
    W.e_fx = reinterpret_cast<float *>(wb + L.e_fx);
    W.e_fy = reinterpret_cast<float *>(wb + L.e_fy);
    W.e_fz = reinterpret_cast<float *>(wb + L.e_fz);
    W.a_u = reinterpret_cast<float4 *>(wb + L.a_u);
    W.a_x = reinterpret_cast<float4 *>(wb + L.a_x);
    W.a_s = reinterpret_cast<float *>(wb + L.a_s);
    W.coef = reinterpret_cast<float *>(wb + L.coef);
    float *s_g = reinterpret_cast<float *>(smem + L.tc_g);
    int *s_cl = reinterpret_cast<int *>(smem + L.tc_cl);
    int *s_nnb = reinterpret_cast<int *>(smem + L.tc_nnb);

#pragma unroll
    for (int t = 0; t < kMaxSpecies; ++t)
        if (tid == t) s_tw[t] = B.type_weight[t];
    if constexpr (sh_angular<KRT, KAT, EXACT>()) load_sh_table(B.sh_b, s_sh, tid);

    // ---- network parameters of every species into the shared-memory layout
    if constexpr (MODE == kFused) load_net_params<KRT, KAT, EXACT>(B, net, params, shift, scale, s_par, tid, NW * 32);
    if constexpr (kTC) load_tc_params<KRT, KAT, EXACT>(B, shift, scale, s_par, tid, NW * 32);

    unsigned long long st_nb = 0, st_ang = 0, st_pairs = 0;
    // Work items are cells: one per CTA (work == NULL), or, in the persistent
    // form, taken from a global counter -- in a batch in the order given by
    // `order` (heaviest cells first); for one structure cells 0 .. split_from-1
    // whole and every later cell as `split` parts (consecutive ranges of its
    // atoms, each part staging the whole neighbourhood), so that the last wave
    // is made of small items and does not leave most SMs idle.
    for (int item_pass = 0;; ++item_pass) {
    int cell, part = 0, nparts = 1, item;
    if (work) {
        __syncthreads();  // the previous item's shared-memory use is over
        if (tid == 0) s_item = (int)atomicAdd(work, 1u);
        __syncthreads();
        item = s_item;
        if (item >= n_items) break;
        if (order) {
            cell = order[item];
        } else if (item < split_from) {
            cell = item;
        } else {
            const int k = item - split_from;
            cell = split_from + k / split;
            part = k - (cell - split_from) * split;
            nparts = split;
        }
    } else {
        if (item_pass) break;
        cell = item = blockIdx.x;
    }
    // the cell grid of this cell's structure: the kernel parameter, or in a batch
    // the grid of the structure that owns the cell (read in place, not copied)
    int sidx = 0;
    if constexpr (BATCH) {
        int lo = 0, hi = n_struct - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sinfo[mid].cell0 <= cell) lo = mid; else hi = mid - 1;
        }
        sidx = lo;
    }
    const Grid &g = BATCH ? sinfo[sidx].g : g_one;
    const int cell0 = BATCH ? sinfo[sidx].cell0 : 0;
    const int n_off = g.n_off;
    if (tid == 0) s_next = 0;
    if (kTC && tid < kMaxSpecies) s_tc_done_a[tid] = s_tc_done_b[tid] = 0;

    // ---- neighbour-cell table: start, count and image shift of every offset
    const int lcell = cell - cell0;         // cell inside its structure's grid
    const int cx = lcell % g.nc[0], cy = (lcell / g.nc[0]) % g.nc[1], cz = lcell / (g.nc[0] * g.nc[1]);
    const int wx = 2 * g.m[0] + 1, wy = 2 * g.m[1] + 1;
    for (int o = tid; o < n_off; o += NW * 32) {
        const int ox = o % wx - g.m[0], oy = (o / wx) % wy - g.m[1], oz = o / (wx * wy) - g.m[2];
        const int ux = cx + ox, uy = cy + oy, uz = cz + oz;
        const int vx = ux - floor_div(ux, g.nc[0]) * g.nc[0];
        const int vy = uy - floor_div(uy, g.nc[1]) * g.nc[1];
        const int vz = uz - floor_div(uz, g.nc[2]) * g.nc[2];
        const int nc = cell0 + (vz * g.nc[1] + vy) * g.nc[0] + vx;
        const int s0 = cell_start[nc];
        off_start[o] = s0;
        off_count[o] = cell_start[nc + 1] - s0;
        // image shift ox A + oy B + oz C (the tilt terms are zero in an orthorhombic box)
        off_shift[o] = make_float4(ox * g.hf[0] + oy * g.htf[0] + oz * g.htf[1], oy * g.hf[1] + oz * g.htf[2],
                                   oz * g.hf[2], __int_as_float((ox | oy | oz) != 0 ? 1 : 0));
    }
    __syncthreads();
    if (warp == 0) {
        int carry = 0;
        for (int base = 0; base < n_off; base += 32) {
            const int o = base + lane;
            const int v = o < n_off ? off_count[o] : 0;
            int x = v;
#pragma unroll
            for (int s = 1; s < 32; s <<= 1) {
                const int y = __shfl_up_sync(kFull, x, s);
                if (lane >= s) x += y;
            }
            if (o < n_off) off_prefix[o] = carry + x - v;
            carry += __shfl_sync(kFull, x, 31);
        }
        if (lane == 0) off_prefix[n_off] = carry;
    }
    __syncthreads();

    const int total = off_prefix[n_off];
    const int cell_first = cell_start[cell], cell_cnt = cell_start[cell + 1] - cell_first;
    const int a_lo = part * cell_cnt / nparts, a_hi = (part + 1) * cell_cnt / nparts;
    const int c0 = cell_first + a_lo;  // this item's atoms: c0 .. c0 + cnt - 1
    const int cnt = a_hi - a_lo;
    const int slot = order ? cell : item;  // row of this item's energy / virial partials (per cell in a batch)
    const int n_chunks = (total + tile - 1) / tile;
    // list-build mode: the entry of the atom itself (zero image offset) is excluded
    const int self_code = (g.m[0] + wx * (g.m[1] + wy * g.m[2])) << caps.vl_jbits;
    const float rc2list = caps.rc_list * caps.rc_list;
    // Staging of chunk `chunk` of the item's neighbourhood into s_pos / s_idx;
    // the number of staged image-atoms is in s_kept after the next barrier.
    // In an orthorhombic cell the item's cell is the box [0, h) of the staged
    // frame, and an image-atom farther than the cutoff from every point of that
    // box is no atom's neighbour: it is not staged (about 28% of a 27-cell
    // neighbourhood). The kept atoms stay in their enumeration order (a block
    // prefix over ballots), so every atom's list is deterministic. The
    // tensor-core modes keep every image-atom: their compact lists refer to
    // the unfiltered enumeration.
    const bool filter = !kTC && !g.tri;
    // (a relative margin of 1e-5 keeps pairs at the cutoff to the last ulp)
    const float rc2stage = (MODE == kBuildList ? rc2list : B.rc_max * B.rc_max) * 1.00001f;
    const unsigned lt_mask = (1u << lane) - 1u;
    auto stage = [&](int chunk) {
        const int base = chunk * tile;
        const int len = min(tile, total - base);
        int kept = 0;  // uniform across the block
        for (int r0 = 0; r0 < len; r0 += NW * 32) {
            const int t = r0 + tid;
            bool keep = false;
            float4 sp = make_float4(0.f, 0.f, 0.f, 0.f);
            int code = 0;
            if (t < len) {
                const int q = base + t;
                int lo = 0, hi = n_off - 1;  // largest o with off_prefix[o] <= q
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (off_prefix[mid] <= q) lo = mid; else hi = mid - 1;
                }
                const int j = off_start[lo] + (q - off_prefix[lo]);
                const float4 p = pos4[j];
                const float4 sh = off_shift[lo];
                sp = make_float4(p.x + sh.x, p.y + sh.y, p.z + sh.z, p.w);
                if constexpr (MODE == kBuildList)
                    code = j | (lo << caps.vl_jbits);  // the Verlet-list entry: index and image offset
                else
                    code = j | (__float_as_int(sh.w) ? kShiftBit : 0);
                keep = true;
                if (filter) {
                    const float dx = fmaxf(fmaxf(-sp.x, sp.x - g.hf[0]), 0.f);
                    const float dy = fmaxf(fmaxf(-sp.y, sp.y - g.hf[1]), 0.f);
                    const float dz = fmaxf(fmaxf(-sp.z, sp.z - g.hf[2]), 0.f);
                    keep = dx * dx + dy * dy + dz * dz <= rc2stage;
                }
            }
            const unsigned mk = __ballot_sync(kFull, keep);
            if (lane == 0) s_wcnt[warp] = __popc(mk);
            __syncthreads();
            int off = kept, round_total = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const int c = s_wcnt[w];
                if (w < warp) off += c;
                round_total += c;
            }
            if (keep) {
                const int slot = off + __popc(mk & lt_mask);
                s_pos[slot] = sp;
                s_idx[slot] = code;
            }
            kept += round_total;
            __syncthreads();  // s_wcnt is written again in the next round
        }
        if (tid == 0) s_kept = kept;
    };

    float vir[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) vir[k] = 0.f;
    double e_acc = 0.0;

    auto finish_list = [&](int &nnb, int &nang) {
        if (nnb > caps.nb) {  // entries past the capacity were dropped
            if (lane == 0) atomicOr(err, kErrNbCap);
            nnb = caps.nb;
        }
        __syncwarp();
        complete_list(B, s_tw, caps, W, lane, nnb, nang, err);
        if (nang > caps.ang) {
            if (lane == 0) atomicOr(err, kErrAngCap);
            nang = caps.ang;
        }
        st_nb += nnb;
        st_ang += nang;
        st_pairs += (unsigned long long)(nang * (nang - 1) / 2);
        __syncwarp();
    };

    if constexpr (kTC) {
    // ---- tensor-core form. The item's atoms are taken in sub-items of at most
    // kTcMaxAtoms, grouped by species (largest group first). Phase A of an atom (neighbour list,
    // descriptor, standardisation) leaves its g row and a compact copy of its
    // list (staging indices) in shared memory; the warp that completes the last
    // phase A of a species runs that species' networks on the tensor cores
    // (16-row tiles), which turn the g rows into dE/dG rows; phase C of an atom
    // (its list rebuilt from the compact copy, the chain rule to forces and
    // virial) waits only for its own species' networks. When the neighbourhood
    // fits one staged chunk the phases are tasks taken in the order A (group
    // by group), then C in the same order, so a group's networks run while
    // other warps still work (the largest group's while the smaller groups'
    // phase A runs, the last group's while the earlier groups' phase C runs); otherwise phase A runs in rounds over the staged
    // chunks and the networks between two block barriers.
    constexpr bool X3 = MODE == kFusedTCx3;
    if (n_chunks <= 1) {
        if (total > 0) stage(0);
        __syncthreads();
    }
    auto tc_phase_a_finish = [&](int a, int i_s, int nnb, int nang) {
        float G0, G1;
        atom_descriptor<KRT, KAT, EXACT>(nnb, nang, B, s_tw, s_sh, W, lane, G0, G1);
        const float *P = s_par + __float_as_int(pos4[i_s].w) * kTcParStride;
        const int g0 = desc_slot0<KRT, KAT>(lane), g1 = desc_slot1<KRT, KAT>(lane);
        s_g[a * kSlots + g0] = (G0 - P[g0]) * P[kSlots + g0];
        s_g[a * kSlots + g1] = (G1 - P[g1]) * P[kSlots + g1];
        if (lane == 0) s_nnb[a] = nnb;
    };
    auto tc_phase_c = [&](int a, int i_s, bool staged) {
        const float4 ui = pos4[i_s];
        const int nnb = s_nnb[a];
        const int *cl = s_cl + a * caps.nb;
        for (int k = lane; k < nnb; k += 32) {
            const int q = cl[k];
            float4 p;
            int j;
            if (staged) {
                p = s_pos[q];
                j = s_idx[q] & ~kShiftBit;
            } else {  // entry q of the concatenated neighbourhood: offset o, atom j
                int lo = 0, hi = n_off - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (off_prefix[mid] <= q) lo = mid; else hi = mid - 1;
                }
                j = off_start[lo] + (q - off_prefix[lo]);
                const float4 pj = pos4[j];
                const float4 sh = off_shift[lo];
                p = make_float4(pj.x + sh.x, pj.y + sh.y, pj.z + sh.z, pj.w);
            }
            const float dx = p.x - ui.x, dy = p.y - ui.y, dz = p.z - ui.z;
            W.e_d[k] = make_float4(dx, dy, dz, dx * dx + dy * dy + dz * dz);
            W.e_j[k] = j | (__float_as_int(p.w) << 28);
        }
        __syncwarp();
        int nang = 0;
        complete_list(B, s_tw, caps, W, lane, nnb, nang, err);
        nang = min(nang, caps.ang);  // an overflow was reported in phase A
        __syncwarp();
        // (the spherical-harmonic form needs its atom's component sums again:
        // the warp's scratch has served other atoms since phase A)
        if constexpr (sh_angular<KRT, KAT, EXACT>()) sh_component_sums(nang, W, lane);
        atom_chain_rule<KRT, KAT, EXACT>(i_s, nnb, nang, B, s_tw, s_sh, W, s_g + a * kSlots, lane, F4, vir);
    };
    for (int sub0 = 0; sub0 < cnt; sub0 += kTcMaxAtoms) {
        const int m = min(kTcMaxAtoms, cnt - sub0);
        const int atom0 = c0 + sub0;
        if (warp == 0) {  // the sub-item's atoms grouped by species, largest group first
            const int ts = lane < m ? __float_as_int(pos4[atom0 + lane].w) : -1;
            // lane t < n_species: its species' count; rank = place of the group in the order
            int cnt_t = 0;
            for (int t = 0; t < B.n_species; ++t) {
                const int c = __popc(__ballot_sync(kFull, ts == t));
                if (lane == t) cnt_t = c;
            }
            int rank = 0;
            for (int u = 0; u < B.n_species; ++u) {
                const int cu = __shfl_sync(kFull, cnt_t, u);
                if (lane < B.n_species && (cu > cnt_t || (cu == cnt_t && u < lane))) ++rank;
            }
            // first position of species t = sum of the counts of the groups ranked before it
            int first_t = 0;
            for (int u = 0; u < B.n_species; ++u) {
                const int cu = __shfl_sync(kFull, cnt_t, u), ru = __shfl_sync(kFull, rank, u);
                if (lane < B.n_species && ru < rank) first_t += cu;
            }
            if (lane < B.n_species) {
                s_tc_first[lane] = first_t;
                s_tc_count[lane] = cnt_t;
            }
            const int my_first = __shfl_sync(kFull, first_t, ts >= 0 ? ts : 0);
            for (int t = 0; t < B.n_species; ++t) {
                const unsigned mk = __ballot_sync(kFull, ts == t);
                if (ts == t) s_tc_order[my_first + __popc(mk & ((1u << lane) - 1u))] = lane;
            }
        }
        __syncthreads();
        auto run_network = [&](int t) {
            tc_species_network<HB, X3>(t, s_tc_order + s_tc_first[t], s_tc_count[t], atom0, lane, s_g, s_par, tc,
                                       eatom, G_out, B.D, e_acc);
        };
        if (n_chunks <= 1) {
            for (;;) {
                int task = 0;
                if (lane == 0) task = atomicAdd(&s_next, 1);
                task = __shfl_sync(kFull, task, 0);
                if (task >= 2 * m) break;
                const int a = s_tc_order[task < m ? task : task - m];
                const int i_s = atom0 + a;
                const int t = __float_as_int(pos4[i_s].w);
                if (task < m) {
                    int nnb = 0, nang = 0;
                    scan_tile<true>(s_pos, s_idx, total, pos4[i_s], i_s, B, caps, W, lane, nnb, s_cl + a * caps.nb, 0);
                    finish_list(nnb, nang);
                    tc_phase_a_finish(a, i_s, nnb, nang);
                    __syncwarp();
                    __threadfence_block();
                    int done = 0;
                    if (lane == 0) done = atomicAdd(&s_tc_done_a[t], 1);
                    done = __shfl_sync(kFull, done, 0);
                    if (done == s_tc_count[t] - 1) {  // the species' last phase A: its networks
                        __threadfence_block();
                        run_network(t);
                        __threadfence_block();
                        __syncwarp();
                        if (lane == 0) atomicExch(&s_tc_done_b[t], 1);
                    }
                } else {
                    if (lane == 0) {  // wait for this species' networks (bounded)
                        int it = 0;
                        while (atomicAdd(&s_tc_done_b[t], 0) == 0) {
                            if (++it > kTcSpin) {
                                atomicOr(err, kErrTimeout);
                                break;
                            }
                            __nanosleep(128);
                        }
                    }
                    __syncwarp();
                    __threadfence_block();
                    tc_phase_c(a, i_s, true);
                }
            }
        } else {
            const int n_rounds = (m + NW - 1) / NW;
            for (int round = 0; round < n_rounds; ++round) {
                const int k = round * NW + warp;
                const bool active = k < m;
                const int a = active ? s_tc_order[k] : 0;
                const int i_s = atom0 + a;
                const float4 ui = active ? pos4[i_s] : make_float4(0.f, 0.f, 0.f, 0.f);
                int nnb = 0, nang = 0;
                for (int chunk = 0; chunk < n_chunks; ++chunk) {
                    __syncthreads();
                    stage(chunk);
                    __syncthreads();
                    if (active)
                        scan_tile<true>(s_pos, s_idx, min(tile, total - chunk * tile), ui, i_s, B, caps, W, lane, nnb,
                                        s_cl + a * caps.nb, chunk * tile);
                }
                if (active) {
                    finish_list(nnb, nang);
                    tc_phase_a_finish(a, i_s, nnb, nang);
                }
            }
            __syncthreads();
            for (int t = warp; t < B.n_species; t += NW)
                if (s_tc_count[t] > 0) run_network(t);
            __syncthreads();
            for (;;) {
                int a = 0;
                if (lane == 0) a = atomicAdd(&s_next, 1);
                a = __shfl_sync(kFull, a, 0);
                if (a >= m) break;
                tc_phase_c(a, atom0 + a, false);
            }
        }
        __syncthreads();  // every task of the sub-item is done
        if (tid == 0) s_next = 0;
        if (tid < kMaxSpecies) s_tc_done_a[tid] = s_tc_done_b[tid] = 0;
        __syncthreads();
    }
    } else if (n_chunks <= 1) {
        if (tid == 0) s_kept = 0;
        if (total > 0) stage(0);
        __syncthreads();
        const int staged = s_kept;
        if constexpr (MODE == kBuildList) {  // two atoms per warp: one pass over the tile serves both
            for (;;) {
                int a = 0;
                if (lane == 0) a = atomicAdd(&s_next, 2);
                a = __shfl_sync(kFull, a, 0);
                if (a >= cnt) break;
                const bool two = a + 1 < cnt;
                const int i0 = c0 + a, i1 = two ? i0 + 1 : i0;
                int n0 = 0, n1 = 0;
                scan_tile_build2(s_pos, s_idx, staged, pos4[i0], pos4[i1], i0 | self_code, i1 | self_code, two,
                                 rc2list, vl_out + (size_t)i0 * caps.vl_cap, vl_out + (size_t)i1 * caps.vl_cap,
                                 caps.vl_cap, lane, n0, n1);
                store_list_count(vl_count, i0, n0, caps.vl_cap, lane, err);
                if (two) store_list_count(vl_count, i1, n1, caps.vl_cap, lane, err);
            }
        } else {
            for (;;) {
                int a = 0;
                if (lane == 0) a = atomicAdd(&s_next, 1);
                a = __shfl_sync(kFull, a, 0);
                if (a >= cnt) break;
                const int i_s = c0 + a;
                const float4 ui = pos4[i_s];
                int nnb = 0, nang = 0;
                scan_tile(s_pos, s_idx, staged, ui, i_s, B, caps, W, lane, nnb);
                finish_list(nnb, nang);
                process_atom<KRT, KAT, EXACT, MODE, HB>(i_s, nnb, nang, B, net, s_par, s_tw, s_sh, W, lane, pos4, F4,
                                                        eatom, G_out, dEdG_in, e_acc, vir);
            }
        }
    } else {
        const int n_rounds = (cnt + NW - 1) / NW;
        for (int round = 0; round < n_rounds; ++round) {
            const int a = round * NW + warp;
            const bool active = a < cnt;
            const int i_s = c0 + a;
            const float4 ui = active ? pos4[i_s] : make_float4(0.f, 0.f, 0.f, 0.f);
            int nnb = 0, nang = 0;
            for (int chunk = 0; chunk < n_chunks; ++chunk) {
                __syncthreads();
                stage(chunk);
                __syncthreads();
                if (active) {
                    const int len = s_kept;
                    if constexpr (MODE == kBuildList)
                        scan_tile_build(s_pos, s_idx, len, ui, i_s | self_code, rc2list,
                                        vl_out + (size_t)i_s * caps.vl_cap, caps.vl_cap, lane, nnb);
                    else
                        scan_tile(s_pos, s_idx, len, ui, i_s, B, caps, W, lane, nnb);
                }
            }
            if (active) {
                if constexpr (MODE == kBuildList) {
                    store_list_count(vl_count, i_s, nnb, caps.vl_cap, lane, err);
                } else {
                    finish_list(nnb, nang);
                    process_atom<KRT, KAT, EXACT, MODE, HB>(i_s, nnb, nang, B, net, s_par, s_tw, s_sh, W, lane, pos4, F4,
                                                            eatom, G_out, dEdG_in, e_acc, vir);
                }
            }
        }
    }

    // ---- cell partials: energy (FP64), virial (FP32 lanes -> FP64)
    if constexpr (MODE == kFused || MODE == kForces || kTC) {
    #pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float v = warp_sum(vir[k]);
            if (lane == 0) s_vir[warp][k] = v;
        }
        if (lane == 0) s_e[warp] = e_acc;
        __syncthreads();
        if (tid < 9) {
            float s = 0.f;
    #pragma unroll
            for (int w = 0; w < NW; ++w) s += s_vir[w][tid];
            vir_part[(size_t)slot * 9 + tid] = (double)s;
        }
        if ((MODE == kFused || kTC) && tid == 0) {  // FP64 sum over the warps' energies, fixed order
            double v = 0.0;
            for (int w = 0; w < NW; ++w) v += s_e[w];
            e_part[slot] = v;
        }
    }
    }  // work items
    if (work && tid == 0) release_work_counter(work);  // every thread has left the loop
    if (MODE != kForces && lane == 0 && st_nb) {  // statistics
        atomicAdd(&stats[0], st_nb);
        atomicAdd(&stats[1], st_ang);
        atomicAdd(&stats[2], st_pairs);
    }
}

// The fused potential over the Verlet list (MD steps between list builds).
// Persistent CTAs (the network parameters are staged once per CTA); each warp
// takes the next sorted atom from a global counter, forms its neighbour list
// from its Verlet-list row (scan_list) and then runs the same descriptor,
// network and chain rule as k_potential. Energy and virial partials per CTA.
template <int KRT, int KAT, bool EXACT, int HB>
__global__ void __launch_bounds__(kPThreads, 2)
    k_potential_list(Basis B, FusedNet net, Grid g, Caps caps, int n, const float4 *__restrict__ pos4,
                     const int *__restrict__ vl, const int *__restrict__ vl_count, const float *__restrict__ params,
                     const float *__restrict__ shift, const float *__restrict__ scale, float4 *__restrict__ F4,
                     float *__restrict__ eatom, double *__restrict__ e_part, double *__restrict__ vir_part,
                     unsigned long long *__restrict__ stats, unsigned *__restrict__ err,
                     unsigned *__restrict__ work) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float s_tw[kMaxSpecies];
    __shared__ float s_sh[sh_angular<KRT, KAT, EXACT>() ? kShTab : 1];  // spherical-harmonic form's table
    __shared__ float s_vir[kPWarps][9];
    __shared__ double s_e[kPWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const PLayout L = make_playout(g.n_off, 0, caps.nb, caps.ang, B.n_species, net.stride);
    float4 *off_shift = reinterpret_cast<float4 *>(smem + L.off_shift);
    float *s_par = reinterpret_cast<float *>(smem + L.params);
    unsigned char *wb = smem + L.warp_base + L.warp_bytes * warp;
    WarpLists W;
    W.e_d = reinterpret_cast<float4 *>(wb + L.e_d);
    W.e_j = reinterpret_cast<int *>(wb + L.e_j);
    W.e_fx = reinterpret_cast<float *>(wb + L.e_fx);
    W.e_fy = reinterpret_cast<float *>(wb + L.e_fy);
    W.e_fz = reinterpret_cast<float *>(wb + L.e_fz);
    W.a_u = reinterpret_cast<float4 *>(wb + L.a_u);
    W.a_x = reinterpret_cast<float4 *>(wb + L.a_x);
    W.a_s = reinterpret_cast<float *>(wb + L.a_s);
    W.coef = reinterpret_cast<float *>(wb + L.coef);
#pragma unroll
    for (int t = 0; t < kMaxSpecies; ++t)
        if (tid == t) s_tw[t] = B.type_weight[t];
    if constexpr (sh_angular<KRT, KAT, EXACT>()) load_sh_table(B.sh_b, s_sh, tid);
    load_net_params<KRT, KAT, EXACT>(B, net, params, shift, scale, s_par, tid, kPThreads);
    const int wx = 2 * g.m[0] + 1, wy = 2 * g.m[1] + 1;
    for (int o = tid; o < g.n_off; o += kPThreads) {  // image offset of every list code
        const int ox = o % wx - g.m[0], oy = (o / wx) % wy - g.m[1], oz = o / (wx * wy) - g.m[2];
        off_shift[o] = make_float4(ox * g.hf[0] + oy * g.htf[0] + oz * g.htf[1], oy * g.hf[1] + oz * g.htf[2],
                                   oz * g.hf[2], 0.f);
    }
    __syncthreads();

    float vir[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) vir[k] = 0.f;
    double e_acc = 0.0;
    unsigned long long st_nb = 0, st_ang = 0, st_pairs = 0;
    for (;;) {
        int a = 0;
        if (lane == 0) a = (int)atomicAdd(work, 1u);
        a = __shfl_sync(kFull, a, 0);
        if (a >= n) break;
        const int i_s = a;
        const float4 ui = pos4[i_s];
        int nnb = 0, nang = 0;
        scan_list(vl + (size_t)i_s * caps.vl_cap, vl_count[i_s], pos4, off_shift, ui, caps.vl_jbits, B, caps, W,
                  lane, nnb);
        if (nnb > caps.nb) {
            if (lane == 0) atomicOr(err, kErrNbCap);
            nnb = caps.nb;
        }
        __syncwarp();
        complete_list(B, s_tw, caps, W, lane, nnb, nang, err);
        if (nang > caps.ang) {
            if (lane == 0) atomicOr(err, kErrAngCap);
            nang = caps.ang;
        }
        st_nb += nnb;
        st_ang += nang;
        st_pairs += (unsigned long long)(nang * (nang - 1) / 2);
        __syncwarp();
        process_atom<KRT, KAT, EXACT, kFused, HB>(i_s, nnb, nang, B, net, s_par, s_tw, s_sh, W, lane, pos4, F4, eatom,
                                                  nullptr, nullptr, e_acc, vir);
    }
    __syncthreads();  // every warp has left the loop
    if (tid == 0) release_work_counter(work);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float v = warp_sum(vir[k]);
        if (lane == 0) s_vir[warp][k] = v;
    }
    if (lane == 0) s_e[warp] = e_acc;
    if (lane == 0 && st_nb) {
        atomicAdd(&stats[0], st_nb);
        atomicAdd(&stats[1], st_ang);
        atomicAdd(&stats[2], st_pairs);
    }
    __syncthreads();
    if (tid < 9) {
        float sv = 0.f;
#pragma unroll
        for (int w = 0; w < kPWarps; ++w) sv += s_vir[w][tid];
        vir_part[(size_t)blockIdx.x * 9 + tid] = (double)sv;
    }
    if (warp == 0) {
        double v = lane < kPWarps ? s_e[lane] : 0.0;
#pragma unroll
        for (int o = kPWarps / 2; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if (lane == 0) e_part[blockIdx.x] = v;
    }
}

}  // namespace
}  // namespace aenet
