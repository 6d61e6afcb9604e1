// MD with a Verlet list: launch of the list-building form of the potential
// kernel and of the list-driven kernel k_potential_list (kernels in
// potential_kernels.cuh).
#include <algorithm>

#include "potential_kernels.cuh"

namespace aenet {
namespace {

using namespace detail;

template <int KRT, int KAT, bool EXACT>
cudaError_t launch_build(Context &c, const Grid &g) {
    const size_t smem = make_playout(g.n_off, c.caps.tile, 0, 0, 0, 0).total;  // no per-warp lists
    auto kern = k_potential<KRT, KAT, EXACT, kBuildList, false, 32>;
    cudaError_t e = allow_max_smem(kern);
    if (e != cudaSuccess) return e;
    const FusedNet net{};
    kern<<<g.ncell, kPThreads, smem, c.stream>>>(c.basis, net, g, nullptr, 0, c.caps, c.d_pos4, c.d_cell_start,
                                                 nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                 nullptr, nullptr, c.d_stats, c.d_err, nullptr, nullptr, g.ncell,
                                                 c.d_vl, c.d_vl_count, 1, 0, TcNet{});
    return cudaGetLastError();
}

size_t potential_list_smem(const Context &c, const Grid &g, const FusedNet &net) {
    return make_playout(g.n_off, 0, c.caps.nb, c.caps.ang, c.basis.n_species, net.stride).total;
}

template <int KRT, int KAT, bool EXACT>
cudaError_t launch_list(Context &c, const Grid &g, int n) {
    const FusedNet net = make_fused_net(c.net);
    const size_t smem = potential_list_smem(c, g, net);
    auto kern = net.hb == 16 ? k_potential_list<KRT, KAT, EXACT, 16> : k_potential_list<KRT, KAT, EXACT, 32>;
    cudaError_t e = allow_max_smem(kern);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPThreads, smem)) != cudaSuccess) return e;
    const int grid = std::max(1, std::min(std::min(std::max(1, per_sm), 4) * c.n_sm, (n + kPWarps - 1) / kPWarps));
    kern<<<grid, kPThreads, smem, c.stream>>>(c.basis, net, g, c.caps, n, c.d_pos4, c.d_vl, c.d_vl_count, c.d_params,
                                              c.d_shift, c.d_scale, c.d_F4, c.d_eatom, c.d_vl_epart, c.d_vl_vpart,
                                              c.d_stats, c.d_err, c.d_work);
    c.last_epart = c.d_vl_epart;
    c.last_vpart = c.d_vl_vpart;
    c.last_eparts = grid;
    c.last_vparts = grid;
    return cudaGetLastError();
}

}  // namespace

int potential_list_max_ctas(const Context &c) { return 4 * std::max(1, c.n_sm); }

cudaError_t launch_vl_build(Context &c, const Grid &g, int n) {
    (void)n;
    const int Kr = c.basis.Kr, Ka = c.basis.Ka;
    if (Kr == 17 && Ka == 9) return launch_build<17, 9, true>(c, g);
    if (Kr == 21 && Ka == 7) return launch_build<21, 7, true>(c, g);
    if (Kr <= 8 && Ka <= 6) return launch_build<8, 6, false>(c, g);
    if (Kr <= 20 && Ka <= 12) return launch_build<20, 12, false>(c, g);
    if (Kr <= 24 && Ka <= 8) return launch_build<24, 8, false>(c, g);
    return cudaErrorInvalidValue;
}

cudaError_t launch_potential_list(Context &c, const Grid &g, int n) {
    if (!c.md_prezeroed) {
        cudaError_t e = cudaMemsetAsync(c.d_stats, 0, sizeof(unsigned long long) * 4, c.stream);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(c.d_F4, 0, sizeof(float4) * (size_t)(n > 0 ? n : 1), c.stream);
        if (e != cudaSuccess) return e;
    }
    const int Kr = c.basis.Kr, Ka = c.basis.Ka;
    if (Kr == 17 && Ka == 9) return launch_list<17, 9, true>(c, g, n);
    if (Kr == 21 && Ka == 7) return launch_list<21, 7, true>(c, g, n);
    if (Kr <= 8 && Ka <= 6) return launch_list<8, 6, false>(c, g, n);
    if (Kr <= 20 && Ka <= 12) return launch_list<20, 12, false>(c, g, n);
    if (Kr <= 24 && Ka <= 8) return launch_list<24, 8, false>(c, g, n);
    return cudaErrorInvalidValue;
}

}  // namespace aenet
