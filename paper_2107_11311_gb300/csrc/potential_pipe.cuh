// Pipelined form of the fused FP32 potential kernel (descriptor, network and
// chain rule of Sec. II.A-B in one pass, as k_potential): one CTA of 16 warps
// per SM, with no block barrier between work items.
//
// k_potential stages an item's neighbourhood with the whole CTA and closes
// every item with a block barrier, so a CTA idles while it stages and while its
// last atoms finish (an item of 24 atoms on 8 warps leaves most warps waiting
// for the slowest one). Here the CTA keeps kPipeBufs staging buffers, each
// holding one item (cell or part of a cell) of the CTA's sequence k = 0, 1, 2,
// ... (buffer k % kPipeBufs). Warps move through that sequence on their own:
// a warp takes the next atom of its current item; when the item has none left
// it moves on to the next one while other warps finish the previous item's
// atoms. Before taking an atom, a warp first helps prepare the next item: it
// claims the item from the global counter and builds its image-offset table
// (one warp), or stages one unit of 32 image-atoms of it. A buffer is refilled
// (for item k + kPipeBufs) once the last atom of its item is done.
//
// Per buffer, the item's sequence number and phase (free, set-up, staging,
// ready, end) share one word, so a warp reads a consistent pair; atom and unit
// claims are 64-bit words tagged with the sequence number and taken by CAS, so
// a claim can never land on a buffer that has moved on to a later item. Every
// wait is bounded (kErrTimeout). Image-atoms are staged unfiltered at fixed
// positions (unit u writes entries 32u .. 32u + 31), so the units need no
// ordering among themselves; an item whose neighbourhood exceeds the buffer is
// scanned straight from global memory.
//
// Energy and virial partials are per CTA (a warp's atoms span items); each
// warp sums its atoms' FP32 energies in FP64.
//
// Measured on GB300 (water, 331,776 and 12,288 atoms): the barrier stalls of
// k_potential vanish, but the kernel runs 25% and 6% slower. With no barrier
// the 16 warps of an SM spread over the whole (large) body of the atom loop,
// and the instruction-cache hit rate falls from 96% to 79%; k_potential's
// per-item barriers keep its warps in step. The form is therefore opt-in
// (AENET_OPT_PIPELINE).
#pragma once

#include "potential_kernels.cuh"

namespace aenet {
namespace detail {

constexpr int kPipeWarps = 16;
constexpr int kPipeBufs = 3;
constexpr int kPipeSpin = 1 << 22;  // waits of a warp (x ~100 ns) before kErrTimeout

enum : int { kBufFree = 0, kBufSetup = 1, kBufStaging = 2, kBufReady = 3, kBufEnd = 4 };

struct PipeLayout {
    // inside one buffer: image-offset table and staged image-atoms
    size_t off_start, off_count, off_prefix, off_shift, s_pos, s_idx, buf_bytes;
    size_t params, warp_base, total;
    PLayout w;  // offsets of the per-warp lists inside a warp's region, and its size (w.warp_bytes)
};

__host__ __device__ inline PipeLayout make_pipe_layout(int n_off, int tile, int cap, int acap, int n_species,
                                                       int stride) {
    PipeLayout P{};
    size_t p = 0;
    P.off_start = p;
    p = align16(p + sizeof(int) * n_off);
    P.off_count = p;
    p = align16(p + sizeof(int) * n_off);
    P.off_prefix = p;
    p = align16(p + sizeof(int) * (n_off + 1));
    P.off_shift = p;
    p = align16(p + sizeof(float4) * n_off);
    P.s_pos = p;
    p = align16(p + sizeof(float4) * tile);
    P.s_idx = p;
    p = align16(p + sizeof(int) * tile);
    P.buf_bytes = p;
    size_t q = P.buf_bytes * kPipeBufs;
    P.params = q;
    q = align16(q + sizeof(float) * (size_t)n_species * stride);
    P.warp_base = q;
    P.w = make_playout(0, 0, cap, acap, 0, 0, 1);
    P.total = q + P.w.warp_bytes * kPipeWarps;
    return P;
}

__device__ __forceinline__ int vload(const int *p) { return *reinterpret_cast<const volatile int *>(p); }
__device__ __forceinline__ unsigned long long vload64(const unsigned long long *p) {
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

// Claim the next index below `limit` from a tagged counter (tag = sequence
// number k in the high word): -1 when exhausted or when the word carries
// another tag (the buffer has moved on).
__device__ __forceinline__ int take_tagged(unsigned long long *word, int k, int limit) {
    for (;;) {
        const unsigned long long w = vload64(word);
        if ((int)(w >> 32) != k) return -1;
        const int next = (int)(unsigned)(w & 0xffffffffull);
        if (next >= limit) return -1;
        if (atomicCAS(word, w, w + 1ull) == w) return next;
    }
}

// Phase 1 of the list build straight from global memory (an item whose
// neighbourhood exceeds the staging buffer): as scan_tile, with candidate q of
// the item's image-offset enumeration fetched through the offset table.
__device__ __forceinline__ void scan_direct(const int *off_start, const int *off_prefix, const float4 *off_shift,
                                            int n_off, int total, const float4 *__restrict__ pos4, float4 ui,
                                            int i_s, const Basis &B, const Caps &caps, const WarpLists &W, int lane,
                                            int &nnb) {
    const float rc2max = B.rc_max * B.rc_max;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int base = 0; base < total; base += 32) {
        const int q = base + lane;
        bool in = false;
        float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
        int jid = 0, typ = 0;
        if (q < total) {
            int lo = 0, hi = n_off - 1;  // largest o with off_prefix[o] <= q
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (off_prefix[mid] <= q) lo = mid; else hi = mid - 1;
            }
            const int j = off_start[lo] + (q - off_prefix[lo]);
            const float4 p = pos4[j];
            const float4 sh = off_shift[lo];
            dx = (p.x + sh.x) - ui.x;
            dy = (p.y + sh.y) - ui.y;
            dz = (p.z + sh.z) - ui.z;
            r2 = dx * dx + dy * dy + dz * dz;
            typ = __float_as_int(p.w);
            jid = j;
            in = (r2 <= rc2max) && !(j == i_s && __float_as_int(sh.w) == 0);
        }
        const unsigned m = __ballot_sync(kFull, in);
        if (in) {
            const int slot = nnb + __popc(m & lt_mask);
            if (slot < caps.nb) {
                W.e_d[slot] = make_float4(dx, dy, dz, r2);
                W.e_j[slot] = jid | (typ << 28);
            }
        }
        nnb += __popc(m);
    }
}

template <int KRT, int KAT, bool EXACT, int HB>
__global__ void __launch_bounds__(kPipeWarps * 32, 1)
    k_potential_pipe(Basis B, FusedNet net, Grid g, Caps caps, const float4 *__restrict__ pos4,
                     const int *__restrict__ cell_start, const float *__restrict__ params,
                     const float *__restrict__ shift, const float *__restrict__ scale, float4 *__restrict__ F4,
                     float *__restrict__ eatom, float *__restrict__ rec_out, double *__restrict__ e_part,
                     double *__restrict__ vir_part, unsigned long long *__restrict__ stats,
                     unsigned *__restrict__ err, unsigned *__restrict__ work, int n_items, int split,
                     int split_from) {
    constexpr int NW = kPipeWarps, NB = kPipeBufs;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float s_tw[kMaxSpecies];
    __shared__ float s_sh[sh_angular<KRT, KAT, EXACT>() ? kShTab : 1];  // spherical-harmonic form's table
    __shared__ float s_vir[NW][9];
    __shared__ double s_e[NW];
    __shared__ int b_state[NB];                  // sequence number * 8 + phase
    __shared__ unsigned long long b_atom[NB];    // tagged claim of the item's next atom
    __shared__ unsigned long long b_unit[NB];    // tagged claim of the item's next staging unit
    __shared__ int b_unit_done[NB], b_atom_done[NB];
    __shared__ int b_c0[NB], b_cnt[NB], b_total[NB], b_units[NB];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const PipeLayout P = make_pipe_layout(g.n_off, caps.tile, caps.nb, caps.ang, B.n_species, net.stride);
    float *s_par = reinterpret_cast<float *>(smem + P.params);
    unsigned char *wb = smem + P.warp_base + P.w.warp_bytes * warp;
    WarpLists W;
    W.e_d = reinterpret_cast<float4 *>(wb + P.w.e_d);
    W.e_j = reinterpret_cast<int *>(wb + P.w.e_j);
    W.e_fx = reinterpret_cast<float *>(wb + P.w.e_fx);
    W.e_fy = reinterpret_cast<float *>(wb + P.w.e_fy);
    W.e_fz = reinterpret_cast<float *>(wb + P.w.e_fz);
    W.a_u = reinterpret_cast<float4 *>(wb + P.w.a_u);
    W.a_x = reinterpret_cast<float4 *>(wb + P.w.a_x);
    W.a_s = reinterpret_cast<float *>(wb + P.w.a_s);
    W.coef = reinterpret_cast<float *>(wb + P.w.coef);
    auto buf = [&](int b) { return smem + P.buf_bytes * b; };

#pragma unroll
    for (int t = 0; t < kMaxSpecies; ++t)
        if (tid == t) s_tw[t] = B.type_weight[t];
    if constexpr (sh_angular<KRT, KAT, EXACT>()) load_sh_table(B.sh_b, s_sh, tid);
    if (tid < NB) {
        b_state[tid] = tid * 8 + kBufFree;
        b_atom[tid] = (unsigned long long)tid << 32;
        b_unit[tid] = (unsigned long long)tid << 32;
        b_unit_done[tid] = b_atom_done[tid] = 0;
    }
    load_net_params<KRT, KAT, EXACT>(B, net, params, shift, scale, s_par, tid, NW * 32);
    __syncthreads();

    const int n_off = g.n_off;
    const int wx = 2 * g.m[0] + 1, wy = 2 * g.m[1] + 1;

    // Set-up of buffer b for item k (one warp, after winning free -> set-up):
    // claim an item with atoms from the global counter, build its image-offset
    // table and publish it as staging (or ready, or end when none is left).
    auto setup = [&](int b, int k) {
        int item = 0, cnt = 0, first = 0, cell = 0;
        for (;;) {
            if (lane == 0) item = (int)atomicAdd(work, 1u);
            item = __shfl_sync(kFull, item, 0);
            if (item >= n_items) break;
            int part = 0, nparts = 1;
            if (item < split_from) {
                cell = item;
            } else {
                const int kk = item - split_from;
                cell = split_from + kk / split;
                part = kk - (cell - split_from) * split;
                nparts = split;
            }
            const int cs = cell_start[cell], cc = cell_start[cell + 1] - cs;
            const int lo = part * cc / nparts, hi = (part + 1) * cc / nparts;
            cnt = hi - lo;
            first = cs + lo;
            if (cnt > 0) break;
        }
        if (item >= n_items) {
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                atomicExch(&b_state[b], k * 8 + kBufEnd);
            }
            __syncwarp();
            return;
        }
        unsigned char *bb = buf(b);
        int *off_start = reinterpret_cast<int *>(bb + P.off_start);
        int *off_count = reinterpret_cast<int *>(bb + P.off_count);
        int *off_prefix = reinterpret_cast<int *>(bb + P.off_prefix);
        float4 *off_shift = reinterpret_cast<float4 *>(bb + P.off_shift);
        const int cx = cell % g.nc[0], cy = (cell / g.nc[0]) % g.nc[1], cz = cell / (g.nc[0] * g.nc[1]);
        int carry = 0;
        for (int base = 0; base < n_off; base += 32) {
            const int o = base + lane;
            int v = 0;
            if (o < n_off) {
                const int ox = o % wx - g.m[0], oy = (o / wx) % wy - g.m[1], oz = o / (wx * wy) - g.m[2];
                const int ux = cx + ox, uy = cy + oy, uz = cz + oz;
                const int vx = ux - floor_div(ux, g.nc[0]) * g.nc[0];
                const int vy = uy - floor_div(uy, g.nc[1]) * g.nc[1];
                const int vz = uz - floor_div(uz, g.nc[2]) * g.nc[2];
                const int nc = (vz * g.nc[1] + vy) * g.nc[0] + vx;
                const int s0 = cell_start[nc];
                v = cell_start[nc + 1] - s0;
                off_start[o] = s0;
                off_count[o] = v;
                // image shift ox A + oy B + oz C (the tilt terms are zero in an orthorhombic box)
                off_shift[o] = make_float4(ox * g.hf[0] + oy * g.htf[0] + oz * g.htf[1],
                                           oy * g.hf[1] + oz * g.htf[2], oz * g.hf[2],
                                           __int_as_float((ox | oy | oz) != 0 ? 1 : 0));
            }
            int x = v;
#pragma unroll
            for (int s = 1; s < 32; s <<= 1) {
                const int y = __shfl_up_sync(kFull, x, s);
                if (lane >= s) x += y;
            }
            if (o < n_off) off_prefix[o] = carry + x - v;
            carry += __shfl_sync(kFull, x, 31);
        }
        if (lane == 0) {
            off_prefix[n_off] = carry;
            const int units = carry <= caps.tile ? (carry + 31) >> 5 : 0;
            b_c0[b] = first;
            b_cnt[b] = cnt;
            b_total[b] = carry;
            b_units[b] = units;
            __threadfence_block();
            atomicExch(&b_state[b], k * 8 + (units > 0 ? kBufStaging : kBufReady));
        }
        __syncwarp();
    };

    // Staging unit u of buffer b (item k): image-atoms 32u .. 32u + 31 of the
    // item's enumeration at their own positions; the last unit publishes ready.
    auto stage_unit = [&](int b, int k, int u) {
        unsigned char *bb = buf(b);
        const int *off_start = reinterpret_cast<const int *>(bb + P.off_start);
        const int *off_prefix = reinterpret_cast<const int *>(bb + P.off_prefix);
        const float4 *off_shift = reinterpret_cast<const float4 *>(bb + P.off_shift);
        float4 *s_pos = reinterpret_cast<float4 *>(bb + P.s_pos);
        int *s_idx = reinterpret_cast<int *>(bb + P.s_idx);
        const int total = b_total[b];
        const int q = 32 * u + lane;
        if (q < total) {
            int lo = 0, hi = n_off - 1;  // largest o with off_prefix[o] <= q
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (off_prefix[mid] <= q) lo = mid; else hi = mid - 1;
            }
            const int j = off_start[lo] + (q - off_prefix[lo]);
            const float4 p = pos4[j];
            const float4 sh = off_shift[lo];
            s_pos[q] = make_float4(p.x + sh.x, p.y + sh.y, p.z + sh.z, p.w);
            s_idx[q] = j | (__float_as_int(sh.w) ? kShiftBit : 0);
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            if (atomicAdd(&b_unit_done[b], 1) == b_units[b] - 1) {
                __threadfence_block();
                atomicExch(&b_state[b], k * 8 + kBufReady);
            }
        }
        __syncwarp();
    };

    float vir[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) vir[k] = 0.f;
    double e_acc = 0.0;
    unsigned long long st_nb = 0, st_ang = 0, st_pairs = 0;

    // Atom a of buffer b (item k): list, descriptor, network, chain rule; the
    // item's last atom releases the buffer for item k + NB.
    auto do_atom = [&](int b, int k, int a) {
        unsigned char *bb = buf(b);
        const int total = b_total[b];
        const int i_s = b_c0[b] + a;
        const float4 ui = pos4[i_s];
        int nnb = 0, nang = 0;
        if (total <= caps.tile)
            scan_tile(reinterpret_cast<const float4 *>(bb + P.s_pos), reinterpret_cast<const int *>(bb + P.s_idx),
                      total, ui, i_s, B, caps, W, lane, nnb);
        else
            scan_direct(reinterpret_cast<const int *>(bb + P.off_start),
                        reinterpret_cast<const int *>(bb + P.off_prefix),
                        reinterpret_cast<const float4 *>(bb + P.off_shift), n_off, total, pos4, ui, i_s, B, caps, W,
                        lane, nnb);
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
        process_atom<KRT, KAT, EXACT, kFused, HB>(i_s, nnb, nang, B, net, s_par, s_tw, s_sh, W, lane, pos4, F4, eatom,
                                                  rec_out, nullptr, e_acc, vir);
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();  // this atom's reads of the buffer are done
            if (atomicAdd(&b_atom_done[b], 1) == b_cnt[b] - 1) {
                const unsigned long long tag = (unsigned long long)(k + NB) << 32;
                b_unit_done[b] = 0;
                b_atom_done[b] = 0;
                atomicExch(&b_atom[b], tag);
                atomicExch(&b_unit[b], tag);
                __threadfence_block();
                atomicExch(&b_state[b], (k + NB) * 8 + kBufFree);
            }
        }
        __syncwarp();
    };

    enum : int { kActWait, kActAdvance, kActSetup, kActStage, kActAtom, kActExit };
    int k = 0;      // this warp's current item in the CTA's sequence
    int waits = 0;  // bounded
    for (;;) {
        int act = kActWait, ab = 0, ak = k, arg = 0;
        if (lane == 0) {
            const int b = k % NB;
            const int st = vload(&b_state[b]);
            const int seq = st >> 3, ph = st & 7;
            __threadfence_block();
            if (seq > k) {
                act = kActAdvance;  // item k is complete
            } else if (seq == k) {
                if (ph == kBufEnd) {
                    act = kActExit;
                } else if (ph == kBufFree) {
                    if (atomicCAS(&b_state[b], st, k * 8 + kBufSetup) == st) {
                        act = kActSetup;
                        ab = b;
                    }
                } else if (ph == kBufStaging) {
                    const int u = take_tagged(&b_unit[b], k, b_units[b]);
                    if (u >= 0) {
                        act = kActStage;
                        ab = b;
                        arg = u;
                    }
                } else if (ph == kBufReady) {
                    // first help to prepare item k + 1, then take an atom of item k
                    const int b1 = (k + 1) % NB;
                    const int st1 = vload(&b_state[b1]);
                    __threadfence_block();
                    if ((st1 >> 3) == k + 1) {
                        if ((st1 & 7) == kBufFree) {
                            if (atomicCAS(&b_state[b1], st1, (k + 1) * 8 + kBufSetup) == st1) {
                                act = kActSetup;
                                ab = b1;
                                ak = k + 1;
                            }
                        } else if ((st1 & 7) == kBufStaging) {
                            const int u = take_tagged(&b_unit[b1], k + 1, b_units[b1]);
                            if (u >= 0) {
                                act = kActStage;
                                ab = b1;
                                ak = k + 1;
                                arg = u;
                            }
                        }
                    }
                    if (act == kActWait) {
                        const int a = take_tagged(&b_atom[b], k, b_cnt[b]);
                        if (a >= 0) {
                            act = kActAtom;
                            ab = b;
                            arg = a;
                        } else {
                            act = kActAdvance;  // no atom left: on to item k + 1
                        }
                    }
                }
            }
        }
        act = __shfl_sync(kFull, act, 0);
        ab = __shfl_sync(kFull, ab, 0);
        ak = __shfl_sync(kFull, ak, 0);
        arg = __shfl_sync(kFull, arg, 0);
        __syncwarp();
        if (act == kActExit) break;
        if (act == kActAdvance) {
            ++k;
        } else if (act == kActSetup) {
            setup(ab, ak);
        } else if (act == kActStage) {
            stage_unit(ab, ak, arg);
        } else if (act == kActAtom) {
            do_atom(ab, k, arg);
        } else {
            if (++waits > kPipeSpin) {
                if (lane == 0) atomicOr(err, kErrTimeout);
                break;
            }
            __nanosleep(100);
        }
    }

    // ---- CTA partials: energy (FP64, fixed warp order), virial (FP32 lanes -> FP64)
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const float v = warp_sum(vir[q]);
        if (lane == 0) s_vir[warp][q] = v;
    }
    if (lane == 0) s_e[warp] = e_acc;
    __syncthreads();
    if (tid < 9) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < NW; ++w) s += s_vir[w][tid];
        vir_part[(size_t)blockIdx.x * 9 + tid] = (double)s;
    }
    if (tid == 0) {
        double v = 0.0;
        for (int w = 0; w < NW; ++w) v += s_e[w];
        e_part[blockIdx.x] = v;
    }
    if (tid == 0) release_work_counter(work);  // every thread has left the loop
    if (lane == 0 && st_nb) {
        atomicAdd(&stats[0], st_nb);
        atomicAdd(&stats[1], st_ang);
        atomicAdd(&stats[2], st_pairs);
    }
}

}  // namespace detail
}  // namespace aenet
