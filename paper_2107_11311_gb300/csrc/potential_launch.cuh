// Launch of the cell-list potential kernel in any of its modes (shared by the
// translation units that instantiate them: potential.cu for the FP32 fused,
// descriptor and force modes, potential_tc.cu for the tensor-core modes, so
// that the two compile in parallel).
#pragma once

#include <algorithm>

#include "potential_kernels.cuh"

namespace aenet {
namespace {

using namespace detail;

// Shared memory of one CTA that still lets two CTAs share an SM (228 KB per SM,
// 1 KB of it reserved per CTA).
constexpr size_t kTwoCtaSmem = 113 * 1024;

// The tensor-core form's network: packed BF16 weights and FP32 biases of the
// context (prepare_bf16_weights), hidden widths and the activation record.
TcNet make_tc_net(const Context &c, const FusedNet &net) {
    TcNet tn;
    tn.pk = make_packed(c.net.widths[1], c.net.widths[2]);
    tn.wpk = reinterpret_cast<const uint32_t *>(c.d_wbf);
    tn.bias = reinterpret_cast<const float *>(reinterpret_cast<const uint32_t *>(c.d_wbf) + c.wbf_elems);
    tn.H1 = c.net.widths[1];
    tn.H2 = c.net.widths[2];
    tn.rec_len = net.rec_len;
    return tn;
}

template <int KRT, int KAT, bool EXACT, int MODE>
cudaError_t launch_mode(Context &c, const Grid &g, const FusedNet &net) {
    constexpr bool tc = is_tc_mode(MODE);
    const int n_sp = (MODE == kFused || tc) ? c.basis.n_species : 0;
    size_t smem = make_playout(g.n_off, c.caps.tile, c.caps.nb, c.caps.ang, n_sp, tc ? kTcParStride : net.stride,
                               kPWarps, tc)
                      .total;
    // the network's hidden-width bound is a template argument of the fused forms only
    auto kern = c.batch_sinfo ? k_potential<KRT, KAT, EXACT, MODE, true, 32> : k_potential<KRT, KAT, EXACT, MODE, false, 32>;
    int nw = kPWarps;
    if constexpr (tc) {
        if (net.hb == 16)
            kern = c.batch_sinfo ? k_potential<KRT, KAT, EXACT, MODE, true, 16>
                                 : k_potential<KRT, KAT, EXACT, MODE, false, 16>;
    }
    if constexpr (MODE == kFused) {
        if (net.hb == 16) {
            kern = c.batch_sinfo ? k_potential<KRT, KAT, EXACT, MODE, true, 16>
                                 : k_potential<KRT, KAT, EXACT, MODE, false, 16>;
        } else if (smem > kTwoCtaSmem) {
            // one CTA per SM anyway (wide networks of several species): give it
            // 12 warps instead of 8 if their lists fit
            int dev = 0, optin = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            const size_t smem12 = make_playout(g.n_off, c.caps.tile, c.caps.nb, c.caps.ang, n_sp, net.stride, 12).total;
            if (smem12 + 1024 <= (size_t)optin) {
                nw = 12;
                smem = smem12;
                kern = c.batch_sinfo ? k_potential<KRT, KAT, EXACT, MODE, true, 32, 12>
                                     : k_potential<KRT, KAT, EXACT, MODE, false, 32, 12>;
            }
        }
    }
    cudaError_t e = allow_max_smem(kern);
    if (e != cudaSuccess) return e;
    // activation records (fused forms) / G rows
    float *rows = (MODE == kFused || tc) ? (c.keep_act ? c.d_act : nullptr) : c.d_G;
    const TcNet tn = tc ? make_tc_net(c, net) : TcNet{};
    // one structure: (some) cells split into parts (persistent CTAs); batches: whole cells
    int split_from = 0;
    const int split = c.batch_sinfo ? 1 : potential_split(c, g, &split_from);
    const int n_items = split_from + (g.ncell - split_from) * split;
    int grid = g.ncell;
    unsigned *work = nullptr;
    if (((c.persist && c.batch_sinfo) || split > 1) && c.d_work && g.ncell > 0) {
        // persistent form: as many CTAs as stay resident (or the tuned count)
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nw * 32, smem)) != cudaSuccess)
            return e;
        const int resident = std::max(1, per_sm) * c.n_sm;
        grid = std::min(n_items, c.persist_ctas > 0 ? std::min(c.persist_ctas, resident) : resident);
        work = c.d_work;  // left at zero by the previous persistent launch
    }
    kern<<<grid, nw * 32, smem, c.stream>>>(c.basis, net, g, c.batch_sinfo, c.batch_n, c.caps, c.d_pos4,
                                              c.d_cell_start, c.d_params,
                                              c.d_shift, c.d_scale, c.d_F4, c.d_eatom, rows, c.d_dEdG,
                                              c.d_e_part, c.d_vir_part, c.d_stats, c.d_err, work,
                                              (work && c.batch_sinfo) ? c.batch_order : nullptr, n_items, nullptr,
                                              nullptr, split, split_from, tn);
    c.last_grid = grid;
    c.pot_parts = n_items;
    return cudaGetLastError();
}

template <int MODE>
cudaError_t dispatch(Context &c, const Grid &g) {
    const FusedNet net = make_fused_net(c.net);
    const int Kr = c.basis.Kr, Ka = c.basis.Ka;
    if constexpr (is_tc_mode(MODE)) {  // the bases whose slots are the G columns
        if (Kr == 17 && Ka == 9) return launch_mode<17, 9, true, MODE>(c, g, net);
        if (Kr == 21 && Ka == 7) return launch_mode<21, 7, true, MODE>(c, g, net);
        return cudaErrorInvalidValue;
    } else {
    if (Kr == 17 && Ka == 9) return launch_mode<17, 9, true, MODE>(c, g, net);
    if (Kr == 21 && Ka == 7) return launch_mode<21, 7, true, MODE>(c, g, net);
    // small bases (e.g. D = 20) get their own bound, so that the fixed-trip
    // order loops do not run the masked orders of the (20, 12) form
    if (Kr <= 8 && Ka <= 6) return launch_mode<8, 6, false, MODE>(c, g, net);
    if (Kr <= 20 && Ka <= 12) return launch_mode<20, 12, false, MODE>(c, g, net);
    if (Kr <= 24 && Ka <= 8) return launch_mode<24, 8, false, MODE>(c, g, net);
    return cudaErrorInvalidValue;
    }
}

}  // namespace
}  // namespace aenet
