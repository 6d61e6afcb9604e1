// Rows a3-a5 and a8 of the path: neighbours, the Chebyshev descriptor
// (Sec. II.B: Eq. radial with the cosine cutoff of Eq. cos-cutoff, Eq. angular
// and the species-weighted copy) and, in the backward variant, the chain rule
// from dE/dG to forces and virial.
//
// Design (GB300): one CTA per cell, one warp per atom of that cell.
//  * The atoms of the (2m+1)^3 neighbour cells are staged once per CTA in
//    shared memory with their periodic image shift already applied (coalesced
//    float4 loads of the cell-sorted, cell-local coordinates).
//  * Each warp builds its atom's neighbour list in shared memory by a ballot
//    compaction over the staged tile (entries with r <= max cutoff; a second
//    list holds the angular ones with unit vector and cutoff value).
//  * Forward: lanes stride over neighbours (radial) and over the flattened
//    unordered (j < k) pairs (angular; the paper's ordered sum is twice the
//    unordered one), accumulating all D coefficients in registers; a 5-stage
//    transpose reduction leaves 2 coefficients per lane for a coalesced store.
//  * Backward: the same list is rebuilt (derivatives are recomputed per tile,
//    never stored); dE/dG is broadcast into registers; per-neighbour force
//    accumulators live in shared memory; one FP32 vector atomic per neighbour
//    scatters forces to global memory; the virial is reduced per CTA into an
//    FP64 partial.
// Displacements are formed from cell-local FP32 coordinates plus the exact cell
// offset, so their error does not grow with the box size.
#include <stdio.h>

#include "aenet_internal.cuh"
#include "fp_common.cuh"

namespace aenet {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kTile = 1024;  // staged atoms per chunk
using detail::align16;
using detail::floor_div;
using detail::kFull;
using detail::kShiftBit;
using detail::pair_advance;
using detail::transpose_reduce64;

struct SmemLayout {
    size_t off_start, off_count, off_prefix, off_shift, s_pos, s_idx, warp_base, warp_bytes, total;
    size_t nb_d, nb_j, nb_s, nb_fx, nb_fy, nb_fz, ang_u, ang_x;  // offsets inside a warp region
};

__host__ __device__ inline SmemLayout make_layout(int n_off, int cap, int acap, bool bwd) {
    SmemLayout L{};
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
    p = align16(p + sizeof(float4) * kTile);
    L.s_idx = p;
    p = align16(p + sizeof(int) * kTile);
    L.warp_base = p;
    size_t q = 0;
    L.nb_d = q;
    q = align16(q + sizeof(float4) * cap);
    L.nb_j = q;
    q = align16(q + sizeof(int) * cap);
    L.nb_s = q;
    q = align16(q + sizeof(float) * cap);
    L.nb_fx = q;
    L.nb_fy = q;
    L.nb_fz = q;
    if (bwd) {
        L.nb_fx = q;
        q = align16(q + sizeof(float) * cap);
        L.nb_fy = q;
        q = align16(q + sizeof(float) * cap);
        L.nb_fz = q;
        q = align16(q + sizeof(float) * cap);
    }
    L.ang_u = q;
    q = align16(q + sizeof(float4) * acap);
    L.ang_x = q;
    q = align16(q + sizeof(float4) * acap);
    L.warp_bytes = q;
    L.total = p + q * kWarps;
    return L;
}

template <int KRT, int KAT, bool EXACT, bool BWD>
__global__ void __launch_bounds__(kThreads, 1)
    k_fingerprint(Basis B, Grid g, Caps caps, const float4 *__restrict__ pos4, const int *__restrict__ cell_start,
                  float *__restrict__ G, const float *__restrict__ dEdG, float4 *__restrict__ F4,
                  double *__restrict__ vir_part, unsigned long long *__restrict__ stats,
                  unsigned *__restrict__ err) {
    static_assert(2 * (KRT + KAT) <= 64, "descriptor slots exceed 64");
    constexpr int SLOT_ANG = KRT, SLOT_RADW = KRT + KAT, SLOT_ANGW = 2 * KRT + KAT;
    const int Kr = EXACT ? KRT : B.Kr;
    const int Ka = EXACT ? KAT : B.Ka;
    const int D = 2 * (Kr + Ka);
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float s_tw[kMaxSpecies];
    __shared__ float s_vir[kWarps][9];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n_off = g.n_off;
    const SmemLayout L = make_layout(n_off, caps.nb, caps.ang, BWD);
    int *off_start = reinterpret_cast<int *>(smem + L.off_start);
    int *off_count = reinterpret_cast<int *>(smem + L.off_count);
    int *off_prefix = reinterpret_cast<int *>(smem + L.off_prefix);
    float4 *off_shift = reinterpret_cast<float4 *>(smem + L.off_shift);
    float4 *s_pos = reinterpret_cast<float4 *>(smem + L.s_pos);
    int *s_idx = reinterpret_cast<int *>(smem + L.s_idx);
    unsigned char *wbase = smem + L.warp_base + L.warp_bytes * warp;
    float4 *nb_d = reinterpret_cast<float4 *>(wbase + L.nb_d);
    int *nb_j = reinterpret_cast<int *>(wbase + L.nb_j);
    float *nb_s = reinterpret_cast<float *>(wbase + L.nb_s);
    float *nb_fx = reinterpret_cast<float *>(wbase + L.nb_fx);
    float *nb_fy = reinterpret_cast<float *>(wbase + L.nb_fy);
    float *nb_fz = reinterpret_cast<float *>(wbase + L.nb_fz);
    float4 *ang_u = reinterpret_cast<float4 *>(wbase + L.ang_u);
    float4 *ang_x = reinterpret_cast<float4 *>(wbase + L.ang_x);

    if (tid < kMaxSpecies) s_tw[tid] = B.type_weight[tid];

    // ---- neighbour-cell table: start, count, image shift of every offset
    const int cell = blockIdx.x;
    const int cx = cell % g.nc[0], cy = (cell / g.nc[0]) % g.nc[1], cz = cell / (g.nc[0] * g.nc[1]);
    const int wx = 2 * g.m[0] + 1, wy = 2 * g.m[1] + 1;
    for (int o = tid; o < n_off; o += kThreads) {
        int ox = o % wx - g.m[0], oy = (o / wx) % wy - g.m[1], oz = o / (wx * wy) - g.m[2];
        int ux = cx + ox, uy = cy + oy, uz = cz + oz;
        int vx = ux - floor_div(ux, g.nc[0]) * g.nc[0];
        int vy = uy - floor_div(uy, g.nc[1]) * g.nc[1];
        int vz = uz - floor_div(uz, g.nc[2]) * g.nc[2];
        int nc = (vz * g.nc[1] + vy) * g.nc[0] + vx;
        int s0 = cell_start[nc];
        off_start[o] = s0;
        off_count[o] = cell_start[nc + 1] - s0;
        off_shift[o] = make_float4(ox * g.hf[0], oy * g.hf[1], oz * g.hf[2],
                                   __int_as_float((ox | oy | oz) != 0 ? 1 : 0));
    }
    __syncthreads();
    if (warp == 0) {
        int carry = 0;
        for (int base = 0; base < n_off; base += 32) {
            int o = base + lane;
            int v = o < n_off ? off_count[o] : 0;
            int x = v;
#pragma unroll
            for (int s = 1; s < 32; s <<= 1) {
                int y = __shfl_up_sync(kFull, x, s);
                if (lane >= s) x += y;
            }
            if (o < n_off) off_prefix[o] = carry + x - v;
            carry += __shfl_sync(kFull, x, 31);
        }
        if (lane == 0) off_prefix[n_off] = carry;
    }
    __syncthreads();

    const int total = off_prefix[n_off];
    const int c0 = cell_start[cell];
    const int cnt = cell_start[cell + 1] - c0;
    const int n_rounds = (cnt + kWarps - 1) / kWarps;
    const int n_chunks = (total + kTile - 1) / kTile;
    const bool single = n_chunks <= 1;

    auto stage = [&](int chunk) {
        const int base = chunk * kTile;
        const int len = min(kTile, total - base);
        for (int t = tid; t < len; t += kThreads) {
            int q = base + t;
            int lo = 0, hi = n_off - 1;  // largest o with off_prefix[o] <= q
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (off_prefix[mid] <= q) lo = mid; else hi = mid - 1;
            }
            int j = off_start[lo] + (q - off_prefix[lo]);
            float4 p = pos4[j];
            float4 sh = off_shift[lo];
            s_pos[t] = make_float4(p.x + sh.x, p.y + sh.y, p.z + sh.z, p.w);
            s_idx[t] = j | (__float_as_int(sh.w) ? kShiftBit : 0);
        }
    };
    if (single && total > 0) {
        stage(0);
        __syncthreads();
    }

    const float rc2max = B.rc_max * B.rc_max, rc2ang = B.rc_ang * B.rc_ang;
    const float inv_rca = 1.0f / B.rc_ang, inv_rcr = 1.0f / B.rc_rad;
    const unsigned lt_mask = (1u << lane) - 1u;
    float vir[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) vir[k] = 0.f;
    unsigned long long st_nb = 0, st_ang = 0, st_pairs = 0;  // neighbour statistics of this warp

    for (int round = 0; round < n_rounds; ++round) {
        const int a = round * kWarps + warp;
        const bool active = a < cnt;
        const int i_s = c0 + a;
        float4 ui = make_float4(0.f, 0.f, 0.f, 0.f);
        if (active) ui = pos4[i_s];
        int nnb = 0, nang = 0;
        for (int chunk = 0; chunk < n_chunks; ++chunk) {
            if (!single) {
                __syncthreads();
                stage(chunk);
                __syncthreads();
            }
            if (!active) continue;
            const int len = min(kTile, total - chunk * kTile);
            for (int base = 0; base < len; base += 32) {
                const int q = base + lane;
                bool in = false, ina = false;
                float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
                int jid = 0, typ = 0;
                if (q < len) {
                    float4 p = s_pos[q];
                    jid = s_idx[q];
                    dx = p.x - ui.x;
                    dy = p.y - ui.y;
                    dz = p.z - ui.z;
                    r2 = dx * dx + dy * dy + dz * dz;
                    typ = __float_as_int(p.w);
                    in = (r2 <= rc2max) && (jid != i_s);
                    ina = in && (r2 <= rc2ang);
                }
                const unsigned m = __ballot_sync(kFull, in);
                const unsigned ma = __ballot_sync(kFull, ina);
                if (in) {
                    const int slot = nnb + __popc(m & lt_mask);
                    float r = sqrtf(r2);
                    if (r < 1e-6f) {
                        atomicOr(err, kErrOverlap);
                        r = 1e-6f;
                    }
                    const float s = s_tw[typ];
                    if (slot < caps.nb) {
                        nb_d[slot] = make_float4(dx, dy, dz, r);
                        nb_j[slot] = jid & ~kShiftBit;
                        nb_s[slot] = s;
                    }
                    if (ina) {
                        const int aslot = nang + __popc(ma & lt_mask);
                        if (aslot < caps.ang && slot < caps.nb) {
                            const float inv = 1.0f / r;
                            const float fc = 0.5f * (cospif(r * inv_rca) + 1.0f);
                            const float dfc = -0.5f * 3.14159265358979f * inv_rca * sinpif(r * inv_rca);
                            ang_u[aslot] = make_float4(dx * inv, dy * inv, dz * inv, fc);
                            ang_x[aslot] = make_float4(r, dfc, s, __int_as_float(slot));
                        }
                    }
                }
                nnb += __popc(m);
                nang += __popc(ma);
            }
        }
        if (active) {
            if (nnb > caps.nb) {  // entries past the capacity were dropped; angular slots may be stale
                if (lane == 0) atomicOr(err, kErrNbCap);
                nnb = caps.nb;
                nang = 0;
            }
            if (nang > caps.ang) {
                if (lane == 0) atomicOr(err, kErrAngCap);
                nang = caps.ang;
            }
            st_nb += nnb;
            st_ang += nang;
            st_pairs += (unsigned long long)(nang * (nang - 1) / 2);
        }
        __syncwarp();
        if (active) {
            const int P = nang * (nang - 1) / 2;
            if constexpr (!BWD) {
                float acc[64];
#pragma unroll
                for (int k = 0; k < 64; ++k) acc[k] = 0.f;
                // radial (Eq. radial) and its weighted copy
                for (int k = lane; k < nnb; k += 32) {
                    const float4 e = nb_d[k];
                    const float r = e.w;
                    if (r <= B.rc_rad) {
                        const float s = nb_s[k];
                        const float x = 2.0f * r * inv_rcr - 1.0f;
                        const float fc = 0.5f * (cospif(r * inv_rcr) + 1.0f);
                        const float sfc = s * fc;
                        float tm1 = 1.0f, t = x;
                        acc[0] += fc;
                        acc[SLOT_RADW] += sfc;
#pragma unroll
                        for (int q = 1; q < KRT; ++q) {
                            if (q < Kr) {
                                acc[q] = fmaf(t, fc, acc[q]);
                                acc[SLOT_RADW + q] = fmaf(t, sfc, acc[SLOT_RADW + q]);
                                const float tn = fmaf(2.0f * x, t, -tm1);
                                tm1 = t;
                                t = tn;
                            }
                        }
                    }
                }
                // angular (Eq. angular) over unordered pairs, doubled below
                if (P > 0) {
                    int j = 0, rem = 0;
                    pair_advance(nang, lane, j, rem);
                    for (int p = lane; p < P; p += 32) {
                        const int kk = j + 1 + rem;
                        const float4 uj = ang_u[j], uk = ang_u[kk];
                        const float sj = ang_x[j].z, sk = ang_x[kk].z;
                        const float c = uj.x * uk.x + uj.y * uk.y + uj.z * uk.z;
                        const float w = uj.w * uk.w;
                        const float ws = w * sj * sk;
                        float tm1 = 1.0f, t = c;
                        acc[SLOT_ANG] += w;
                        acc[SLOT_ANGW] += ws;
#pragma unroll
                        for (int q = 1; q < KAT; ++q) {
                            if (q < Ka) {
                                acc[SLOT_ANG + q] = fmaf(t, w, acc[SLOT_ANG + q]);
                                acc[SLOT_ANGW + q] = fmaf(t, ws, acc[SLOT_ANGW + q]);
                                const float tn = fmaf(2.0f * c, t, -tm1);
                                tm1 = t;
                                t = tn;
                            }
                        }
                        pair_advance(nang, 32, j, rem);
                    }
                }
                transpose_reduce64(acc, lane);
                // lane holds slots 2 lane, 2 lane + 1; map slots to G columns
                float *row = G + (size_t)i_s * D;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int slot = 2 * lane + h;
                    int col = -1;
                    float val = acc[h];
                    if (slot < SLOT_ANG) {
                        if (slot < Kr) col = slot;
                    } else if (slot < SLOT_RADW) {
                        if (slot - SLOT_ANG < Ka) col = Kr + (slot - SLOT_ANG), val *= 2.0f;
                    } else if (slot < SLOT_ANGW) {
                        if (slot - SLOT_RADW < Kr) col = Kr + Ka + (slot - SLOT_RADW);
                    } else if (slot < SLOT_ANGW + KAT) {
                        if (slot - SLOT_ANGW < Ka) col = 2 * Kr + Ka + (slot - SLOT_ANGW), val *= 2.0f;
                    }
                    if (col >= 0) row[col] = val;
                }
            } else {
                // ---- backward: dE_i/dd for every neighbour, scattered as forces
                const float *crow = dEdG + (size_t)i_s * D;
                float cr[KRT], crw[KRT], ca[KAT], caw[KAT];
#pragma unroll
                for (int q = 0; q < KRT; ++q) {
                    cr[q] = q < Kr ? crow[q] : 0.f;
                    crw[q] = q < Kr ? crow[Kr + Ka + q] : 0.f;
                }
#pragma unroll
                for (int q = 0; q < KAT; ++q) {  // factor 2: ordered-pair sum
                    ca[q] = q < Ka ? 2.0f * crow[Kr + q] : 0.f;
                    caw[q] = q < Ka ? 2.0f * crow[2 * Kr + Ka + q] : 0.f;
                }
                const float k2 = 2.0f * inv_rcr;
                for (int k = lane; k < nnb; k += 32) {
                    const float4 e = nb_d[k];
                    const float r = e.w;
                    float fx = 0.f, fy = 0.f, fz = 0.f;
                    if (r <= B.rc_rad) {
                        const float s = nb_s[k];
                        const float x = 2.0f * r * inv_rcr - 1.0f;
                        const float fc = 0.5f * (cospif(r * inv_rcr) + 1.0f);
                        const float dfc = -0.5f * 3.14159265358979f * inv_rcr * sinpif(r * inv_rcr);
                        // d/dr [T_q(x) f_c(r)] = T_q'(x) (2/Rc) f_c + T_q f_c',  T_q' = q U_{q-1}
                        float dEdr = (cr[0] + s * crw[0]) * dfc;
                        float tm1 = 1.0f, t = x;   // T_{q-1}, T_q
                        float um1 = 0.0f, u = 1.0f; // U_{q-2}, U_{q-1}
#pragma unroll
                        for (int q = 1; q < KRT; ++q) {
                            if (q < Kr) {
                                const float coef = fmaf(s, crw[q], cr[q]);
                                const float dT = (float)q * u;
                                dEdr = fmaf(coef, fmaf(dT * k2, fc, t * dfc), dEdr);
                                const float tn = fmaf(2.0f * x, t, -tm1);
                                tm1 = t;
                                t = tn;
                                const float un = fmaf(2.0f * x, u, -um1);
                                um1 = u;
                                u = un;
                            }
                        }
                        const float gr = dEdr / r;  // dE_i/dd = gr * d; force on j = -dE_i/dd
                        fx = -gr * e.x;
                        fy = -gr * e.y;
                        fz = -gr * e.z;
                    }
                    nb_fx[k] = fx;
                    nb_fy[k] = fy;
                    nb_fz[k] = fz;
                }
                __syncwarp();
                if (P > 0) {
                    int j = 0, rem = 0;
                    pair_advance(nang, lane, j, rem);
                    int cur = -1;
                    float ax = 0.f, ay = 0.f, az = 0.f;
                    for (int p = lane; p < P; p += 32) {
                        const int kk = j + 1 + rem;
                        const float4 uj = ang_u[j], uk = ang_u[kk];
                        const float4 xj = ang_x[j], xk = ang_x[kk];
                        const float c = uj.x * uk.x + uj.y * uk.y + uj.z * uk.z;
                        const float w = xj.z * xk.z;
                        float S = ca[0] + w * caw[0];
                        float dS = 0.f;
                        float tm1 = 1.0f, t = c, um1 = 0.0f, u = 1.0f;
#pragma unroll
                        for (int q = 1; q < KAT; ++q) {
                            if (q < Ka) {
                                const float b = fmaf(w, caw[q], ca[q]);
                                S = fmaf(b, t, S);
                                dS = fmaf(b * (float)q, u, dS);
                                const float tn = fmaf(2.0f * c, t, -tm1);
                                tm1 = t;
                                t = tn;
                                const float un = fmaf(2.0f * c, u, -um1);
                                um1 = u;
                                u = un;
                            }
                        }
                        const float fj = uj.w, fk = uk.w;
                        const float A = dS * fj * fk;
                        const float Aj = A / xj.x, Ak = A / xk.x;
                        const float Bj = S * xj.y * fk, Bk = S * fj * xk.y;
                        // dE_i/dd_j and dE_i/dd_k of the pair term
                        const float gjx = Aj * (uk.x - c * uj.x) + Bj * uj.x;
                        const float gjy = Aj * (uk.y - c * uj.y) + Bj * uj.y;
                        const float gjz = Aj * (uk.z - c * uj.z) + Bj * uj.z;
                        const float gkx = Ak * (uj.x - c * uk.x) + Bk * uk.x;
                        const float gky = Ak * (uj.y - c * uk.y) + Bk * uk.y;
                        const float gkz = Ak * (uj.z - c * uk.z) + Bk * uk.z;
                        if (j != cur) {
                            if (cur >= 0) {
                                const int sl = __float_as_int(ang_x[cur].w);
                                atomicAdd(&nb_fx[sl], ax);
                                atomicAdd(&nb_fy[sl], ay);
                                atomicAdd(&nb_fz[sl], az);
                            }
                            cur = j;
                            ax = ay = az = 0.f;
                        }
                        ax -= gjx;
                        ay -= gjy;
                        az -= gjz;
                        const int slk = __float_as_int(xk.w);
                        atomicAdd(&nb_fx[slk], -gkx);
                        atomicAdd(&nb_fy[slk], -gky);
                        atomicAdd(&nb_fz[slk], -gkz);
                        pair_advance(nang, 32, j, rem);
                    }
                    if (cur >= 0) {
                        const int sl = __float_as_int(ang_x[cur].w);
                        atomicAdd(&nb_fx[sl], ax);
                        atomicAdd(&nb_fy[sl], ay);
                        atomicAdd(&nb_fz[sl], az);
                    }
                }
                __syncwarp();
                // scatter: force on each neighbour image, reaction on i, virial
                float fix = 0.f, fiy = 0.f, fiz = 0.f;
                for (int k = lane; k < nnb; k += 32) {
                    const float fx = nb_fx[k], fy = nb_fy[k], fz = nb_fz[k];
                    const float4 e = nb_d[k];
                    atomicAdd(&F4[nb_j[k]], make_float4(fx, fy, fz, 0.f));
                    fix -= fx;
                    fiy -= fy;
                    fiz -= fz;
                    // W_ab = -sum d_a dE/dd_b = sum d_a f_b
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
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) {
                    fix += __shfl_xor_sync(kFull, fix, o);
                    fiy += __shfl_xor_sync(kFull, fiy, o);
                    fiz += __shfl_xor_sync(kFull, fiz, o);
                }
                if (lane == 0) atomicAdd(&F4[i_s], make_float4(fix, fiy, fiz, 0.f));
            }
        }
        __syncwarp();
    }

    if constexpr (!BWD) {
        if (lane == 0 && st_nb) {
            atomicAdd(&stats[0], st_nb);
            atomicAdd(&stats[1], st_ang);
            atomicAdd(&stats[2], st_pairs);
        }
    }
    if constexpr (BWD) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            float v = vir[k];
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
            if (lane == 0) s_vir[warp][k] = v;
        }
        __syncthreads();
        if (tid < 9) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) s += (double)s_vir[w][tid];
            vir_part[(size_t)blockIdx.x * 9 + tid] = s;
        }
    }
}

template <int KRT, int KAT, bool EXACT>
cudaError_t launch_variant(Context &c, const Grid &g, bool bwd) {
    const size_t smem = make_layout(g.n_off, c.caps.nb, c.caps.ang, bwd).total;
    cudaError_t e;
    if (bwd) {
        auto kern = k_fingerprint<KRT, KAT, EXACT, true>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<g.ncell, kThreads, smem, c.stream>>>(c.basis, g, c.caps, c.d_pos4, c.d_cell_start, c.d_G,
                                                     c.d_dEdG, c.d_F4, c.d_vir_part, c.d_stats, c.d_err);
    } else {
        auto kern = k_fingerprint<KRT, KAT, EXACT, false>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<g.ncell, kThreads, smem, c.stream>>>(c.basis, g, c.caps, c.d_pos4, c.d_cell_start, c.d_G,
                                                     c.d_dEdG, c.d_F4, c.d_vir_part, c.d_stats, c.d_err);
    }
    return cudaGetLastError();
}

cudaError_t dispatch(Context &c, const Grid &g, bool bwd) {
    const int Kr = c.basis.Kr, Ka = c.basis.Ka;
    if (Kr == 17 && Ka == 9) return launch_variant<17, 9, true>(c, g, bwd);
    if (Kr == 21 && Ka == 7) return launch_variant<21, 7, true>(c, g, bwd);
    if (Kr <= 20 && Ka <= 12) return launch_variant<20, 12, false>(c, g, bwd);
    if (Kr <= 24 && Ka <= 8) return launch_variant<24, 8, false>(c, g, bwd);
    return cudaErrorInvalidValue;
}

}  // namespace

size_t fp_smem_bytes(const Grid &g, const Caps &caps, bool backward) {
    return make_layout(g.n_off, caps.nb, caps.ang, backward).total;
}

cudaError_t launch_fp_forward(Context &c, const Grid &g, int n) {
    (void)n;
    cudaError_t e = cudaMemsetAsync(c.d_stats, 0, sizeof(unsigned long long) * 4, c.stream);
    if (e != cudaSuccess) return e;
    return dispatch(c, g, false);
}

cudaError_t launch_fp_backward(Context &c, const Grid &g, int n) {
    cudaError_t e = cudaMemsetAsync(c.d_F4, 0, sizeof(float4) * (size_t)(n > 0 ? n : 1), c.stream);
    if (e != cudaSuccess) return e;
    return dispatch(c, g, true);
}

}  // namespace aenet

// ---------------------------------------------------------------------------
// Allocation-free descriptor entry point (aenet_descriptors_noalloc).
//
// Some callers cannot allocate device memory at the time they need descriptors:
// a host program that hands every allocation to its own fixed memory pool, code
// that runs while another component owns the allocator, or a plugin that must
// not grow the process's GPU footprint after start-up. For them this entry point
// computes the same descriptor as aenet_descriptors() without a context and
// without any cudaMalloc/cudaFree: its scratch (cell-sorted coordinates, cell
// table, sorted descriptor rows, error word) is one file-scope __device__ array
// of fixed size, which every GPU that loads this library holds until the
// process exits. The caller passes device inputs and the device output.
#include <mutex>

namespace aenet {

__global__ void k_bin_count(int n, int n_species, const double *__restrict__ pos,
                            const int32_t *__restrict__ types, Grid g, float4 *__restrict__ tmp4,
                            int *__restrict__ cell_of, int *__restrict__ slot, int *__restrict__ cell_count,
                            unsigned *__restrict__ err);
__global__ void k_scan_cells(int ncell, const int *__restrict__ count, int *__restrict__ start);
__global__ void k_scatter(int n, const float4 *__restrict__ tmp4, const int *__restrict__ cell_of,
                          const int *__restrict__ slot, const int *__restrict__ cell_start,
                          float4 *__restrict__ pos4, int *__restrict__ perm);

namespace {

constexpr size_t kNaAlign = 256;
constexpr size_t na_round(size_t x) { return (x + kNaAlign - 1) / kNaAlign * kNaAlign; }
constexpr size_t kNaOffTmp4 = 0;
constexpr size_t kNaOffPos4 = kNaOffTmp4 + na_round(sizeof(float4) * AENET_NOALLOC_MAX_ATOMS);
constexpr size_t kNaOffPerm = kNaOffPos4 + na_round(sizeof(float4) * AENET_NOALLOC_MAX_ATOMS);
constexpr size_t kNaOffCellOf = kNaOffPerm + na_round(sizeof(int) * AENET_NOALLOC_MAX_ATOMS);
constexpr size_t kNaOffSlot = kNaOffCellOf + na_round(sizeof(int) * AENET_NOALLOC_MAX_ATOMS);
constexpr size_t kNaOffCount = kNaOffSlot + na_round(sizeof(int) * AENET_NOALLOC_MAX_ATOMS);
constexpr size_t kNaOffStart = kNaOffCount + na_round(sizeof(int) * AENET_NOALLOC_MAX_CELLS);
constexpr size_t kNaOffG = kNaOffStart + na_round(sizeof(int) * (AENET_NOALLOC_MAX_CELLS + 1));
constexpr size_t kNaOffErr = kNaOffG + na_round(sizeof(float) * kMaxD * AENET_NOALLOC_MAX_ATOMS);
constexpr size_t kNaBytes = kNaOffErr + na_round(sizeof(unsigned) + 4 * sizeof(unsigned long long));

// The scratch itself. Host code must not pass this symbol to a kernel: on the
// host it names a stand-in, not the device address (see na_scratch()).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
unsigned char *g_na_ptr[kNaMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and cached.
cudaError_t na_scratch(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

__global__ void k_na_unsort(int n, int D, const int *__restrict__ perm, const float *__restrict__ Gs,
                            float *__restrict__ G) {
    const size_t total = (size_t)n * D;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(k / D), c = (int)(k % D);
        G[(size_t)perm[s] * D + c] = Gs[k];
    }
}

template <int KRT, int KAT, bool EXACT>
cudaError_t na_launch_fp(const Basis &B, const Grid &g, const Caps &caps, cudaStream_t st, const float4 *pos4,
                         const int *cell_start, float *Gs, unsigned long long *stats, unsigned *err) {
    const size_t smem = make_layout(g.n_off, caps.nb, caps.ang, false).total;
    auto kern = k_fingerprint<KRT, KAT, EXACT, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<g.ncell, kThreads, smem, st>>>(B, g, caps, pos4, cell_start, Gs, nullptr, nullptr, nullptr, stats, err);
    return cudaGetLastError();
}

int na_fail(int code, const char *msg) {
    set_context_free_error(msg);
    return code;
}

bool na_is_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace aenet

extern "C" int aenet_descriptors_noalloc(int n, const double *pos, const int32_t *types, const double *box,
                                         int n_species, const double *type_weight, double rc_rad, int order_rad,
                                         double rc_ang, int order_ang, float *G, void *stream) {
    using namespace aenet;
    cudaGetLastError();
    if (n < 0 || n > AENET_NOALLOC_MAX_ATOMS) {
        char msg[160];
        snprintf(msg, sizeof(msg), "n_atoms = %d is outside [0, %d], the fixed scratch limit of this entry point", n,
                 AENET_NOALLOC_MAX_ATOMS);
        return na_fail(AENET_E_CAPACITY, msg);
    }
    if (!box || !type_weight || n_species < 1 || n_species > kMaxSpecies || !(rc_rad > 0.0) || !(rc_ang > 0.0) ||
        order_rad < 0 || order_ang < 0)
        return na_fail(AENET_E_ARG, "invalid basis arguments");
    const int Kr = order_rad + 1, Ka = order_ang + 1, D = 2 * (Kr + Ka);
    const bool supported = (Kr == 17 && Ka == 9) || (Kr == 21 && Ka == 7) || (Kr <= 20 && Ka <= 12) ||
                           (Kr <= 24 && Ka <= 8);
    if (!supported || D > kMaxD) return na_fail(AENET_E_ARG, "unsupported basis orders");
    if (n > 0 && (!pos || !types || !G || !na_is_device(pos) || !na_is_device(types) || !na_is_device(G)))
        return na_fail(AENET_E_ARG, "pos, types and G must be device pointers");
    Basis B{};
    B.n_species = n_species;
    B.Kr = Kr;
    B.Ka = Ka;
    B.D = D;
    B.rc_rad = (float)rc_rad;
    B.rc_ang = (float)rc_ang;
    B.rc_max = (float)(rc_rad > rc_ang ? rc_rad : rc_ang);
    for (int t = 0; t < kMaxSpecies; ++t) B.type_weight[t] = t < n_species ? (float)type_weight[t] : 0.f;
    Grid g{};
    g.ncell = 1;
    g.n_off = 1;
    for (int a = 0; a < 3; ++a) {
        if (!(box[a] > 0.0) || !isfinite(box[a])) return na_fail(AENET_E_ARG, "box lengths must be finite and > 0");
        int nc = (int)floor(box[a] / B.rc_max);
        nc = nc < 1 ? 1 : (nc > 1024 ? 1024 : nc);
        g.nc[a] = nc;
        g.box[a] = box[a];
        g.h[a] = box[a] / nc;
        g.hf[a] = (float)g.h[a];
        g.inv_box[a] = 1.0 / g.box[a];
        g.inv_h[a] = 1.0 / g.h[a];
        g.m[a] = (int)ceil(B.rc_max / g.h[a]);
        g.ncell *= nc;
        g.n_off *= 2 * g.m[a] + 1;
    }
    if (g.ncell > AENET_NOALLOC_MAX_CELLS)
        return na_fail(AENET_E_CAPACITY, "the box has more cells than the fixed scratch of this entry point holds");
    if (g.n_off > 4096) return na_fail(AENET_E_ARG, "box too small for the cutoff");
    if (n == 0) return AENET_OK;

    unsigned char *base = nullptr;
    cudaError_t e = na_scratch(&base);
    if (e != cudaSuccess) return na_fail(AENET_E_CUDA, "cudaGetSymbolAddress of the scratch array failed");
    float4 *tmp4 = reinterpret_cast<float4 *>(base + kNaOffTmp4);
    float4 *pos4 = reinterpret_cast<float4 *>(base + kNaOffPos4);
    int *perm = reinterpret_cast<int *>(base + kNaOffPerm);
    int *cell_of = reinterpret_cast<int *>(base + kNaOffCellOf);
    int *slot = reinterpret_cast<int *>(base + kNaOffSlot);
    int *count = reinterpret_cast<int *>(base + kNaOffCount);
    int *start = reinterpret_cast<int *>(base + kNaOffStart);
    float *Gs = reinterpret_cast<float *>(base + kNaOffG);
    unsigned *err = reinterpret_cast<unsigned *>(base + kNaOffErr);
    unsigned long long *stats = reinterpret_cast<unsigned long long *>(base + kNaOffErr + 8);
    cudaStream_t st = (cudaStream_t)stream;

    // mean-density capacities (1.5x the expected count + 32), one regrow on overflow
    const double rho = n / (box[0] * box[1] * box[2]);
    auto cap = [&](double rc) {
        int k = (int)(1.5 * rho * 4.18879020478639 * rc * rc * rc + 32.0);
        return ((k + 31) / 32) * 32;
    };
    Caps caps{cap(B.rc_max) > 64 ? cap(B.rc_max) : 64, cap(B.rc_ang) > 32 ? cap(B.rc_ang) : 32};
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    unsigned w = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (optin > 0 && make_layout(g.n_off, caps.nb, caps.ang, false).total > (size_t)optin)
            return na_fail(AENET_E_CAPACITY, "neighbour lists exceed the shared memory of one CTA");
        // the scratch keeps the previous call's contents: clear what must start at zero
        if ((e = cudaMemsetAsync(count, 0, sizeof(int) * g.ncell, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(err, 0, sizeof(unsigned) + 8 + 4 * sizeof(unsigned long long), st)) != cudaSuccess)
            return na_fail(AENET_E_CUDA, cudaGetErrorString(e));
        k_bin_count<<<(n + 255) / 256, 256, 0, st>>>(n, n_species, pos, types, g, tmp4, cell_of, slot, count, err);
        k_scan_cells<<<1, 1024, 0, st>>>(g.ncell, count, start);
        k_scatter<<<(n + 255) / 256, 256, 0, st>>>(n, tmp4, cell_of, slot, start, pos4, perm);
        if ((e = cudaGetLastError()) != cudaSuccess) return na_fail(AENET_E_CUDA, cudaGetErrorString(e));
        if (Kr == 17 && Ka == 9) e = na_launch_fp<17, 9, true>(B, g, caps, st, pos4, start, Gs, stats, err);
        else if (Kr == 21 && Ka == 7) e = na_launch_fp<21, 7, true>(B, g, caps, st, pos4, start, Gs, stats, err);
        else if (Kr <= 20 && Ka <= 12) e = na_launch_fp<20, 12, false>(B, g, caps, st, pos4, start, Gs, stats, err);
        else e = na_launch_fp<24, 8, false>(B, g, caps, st, pos4, start, Gs, stats, err);
        if (e != cudaSuccess) return na_fail(AENET_E_CUDA, cudaGetErrorString(e));
        if ((e = cudaMemcpyAsync(&w, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return na_fail(AENET_E_CUDA, cudaGetErrorString(e));
        if (!(w & (kErrNbCap | kErrAngCap))) break;
        caps.nb *= 2;
        caps.ang *= 2;
    }
    if (w & kErrType) return na_fail(AENET_E_ARG, "species index out of range");
    if (w & kErrNonfinite) return na_fail(AENET_E_NONFINITE, "non-finite coordinate");
    if (w & kErrOverlap) return na_fail(AENET_E_OVERLAP, "two image-atoms closer than 1e-6 A");
    if (w & (kErrNbCap | kErrAngCap)) return na_fail(AENET_E_CAPACITY, "neighbour list overflow");
    k_na_unsort<<<256, 256, 0, st>>>(n, D, perm, Gs, G);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return na_fail(AENET_E_CUDA, cudaGetErrorString(e));
    return AENET_OK;
}
