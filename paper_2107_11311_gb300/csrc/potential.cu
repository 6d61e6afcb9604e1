// Cell-list evaluation with the potential kernel: launch of its fused,
// descriptor-only and forces-only forms (single structures and batches), and
// the allocation-free descriptor entry point. The kernels themselves are in
// potential_kernels.cuh.
#include <stdio.h>

#include <algorithm>

#include "potential_launch.cuh"
#include "potential_pipe.cuh"

namespace aenet {

// How a single-structure evaluation divides cells into work items for the
// persistent CTAs. Cells split_from .. ncell-1 are split into `split` parts
// (consecutive ranges of their atoms; each part restages the cell's
// neighbourhood), the others stay whole:
//  * fewer cells than one wave of resident CTAs (2 per SM, or `wave`): every cell, into
//    enough parts to fill the wave (at most kMaxSplit, no part with fewer than 8
//    atoms -- one per warp -- on average): 1,536 atoms in 64 cells run 23% faster;
//  * more cells: the last wave's worth of cells into 2 parts, so that the tail
//    is made of half-size items (also the persistent form, which stages the
//    network parameters once per CTA: water 98,304 and 331,776 atoms run 9%
//    and 12% faster than with one CTA per cell).
int potential_split(const Context &c, const Grid &g, int *split_from, int wave) {
    if (wave <= 0) wave = 2 * std::max(1, c.n_sm);
    *split_from = 0;
    if (g.ncell <= 0) return 1;
    const double per_cell = c.cap_atoms > 0 ? (double)c.cap_atoms / g.ncell : 8.0;
    const int most = std::max(1, (int)(per_cell / 8.0));
    if (g.ncell < wave) {
        const int want = (wave + g.ncell - 1) / g.ncell;
        return std::max(1, std::min(std::min(want, kMaxSplit), most));
    }
    if (most >= 2) {
        *split_from = g.ncell - wave;
        return 2;
    }
    return 1;
}

bool fused_supported(const Context &c) {
    if (c.precision != AENET_FP32) return false;
    for (int l = 1; l < c.net.n_layers; ++l)
        if (c.net.widths[l] > 32) return false;
    return true;
}

bool tc_fused_supported(const Context &c) {
    if (c.precision == AENET_FP32 || !c.fuse_network || !bf16_supported(c.net) || !c.d_wbf) return false;
    return (c.basis.Kr == 17 && c.basis.Ka == 9) || (c.basis.Kr == 21 && c.basis.Ka == 7);
}

// The pipelined form (k_potential_pipe): FP32 fused evaluation of one
// structure on the exact bases, when its layout fits one CTA per SM.
static size_t pipe_smem_bytes(const Context &c, const Grid &g) {
    const FusedNet net = make_fused_net(c.net);
    return make_pipe_layout(g.n_off, c.caps.tile, c.caps.nb, c.caps.ang, c.basis.n_species, net.stride).total;
}

bool pipe_supported(const Context &c, const Grid &g) {
    if (!c.pipeline || !fused_supported(c) || c.batch_sinfo || !c.d_work || c.n_sm <= 0) return false;
    if (!((c.basis.Kr == 17 && c.basis.Ka == 9) || (c.basis.Kr == 21 && c.basis.Ka == 7))) return false;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return pipe_smem_bytes(c, g) + 1024 <= (size_t)optin;  // + the kernel's static shared memory
}

template <int KRT, int KAT, int HB>
static cudaError_t launch_pipe_form(Context &c, const Grid &g, const FusedNet &net) {
    auto kern = k_potential_pipe<KRT, KAT, true, HB>;
    const size_t smem = pipe_smem_bytes(c, g);
    cudaError_t e = allow_max_smem(kern);
    if (e != cudaSuccess) return e;
    // one CTA per SM; the last wave's worth of cells in halves (short tail items)
    int split_from = 0;
    const int split = potential_split(c, g, &split_from, c.n_sm);
    const int n_items = split_from + (g.ncell - split_from) * split;
    const int grid = std::max(1, std::min(c.n_sm, n_items));
    kern<<<grid, kPipeWarps * 32, smem, c.stream>>>(c.basis, net, g, c.caps, c.d_pos4, c.d_cell_start, c.d_params,
                                                    c.d_shift, c.d_scale, c.d_F4, c.d_eatom,
                                                    c.keep_act ? c.d_act : nullptr, c.d_e_part, c.d_vir_part,
                                                    c.d_stats, c.d_err, c.d_work, n_items, split, split_from);
    c.last_grid = grid;
    c.pot_parts = grid;  // energy / virial partial rows: one per CTA
    return cudaGetLastError();
}

static cudaError_t launch_pipe(Context &c, const Grid &g) {
    const FusedNet net = make_fused_net(c.net);
    if (c.basis.Kr == 17 && c.basis.Ka == 9)
        return net.hb == 16 ? launch_pipe_form<17, 9, 16>(c, g, net) : launch_pipe_form<17, 9, 32>(c, g, net);
    return net.hb == 16 ? launch_pipe_form<21, 7, 16>(c, g, net) : launch_pipe_form<21, 7, 32>(c, g, net);
}

size_t potential_smem_bytes(const Context &c, const Grid &g) {
    const FusedNet net = make_fused_net(c.net);
    if (pipe_supported(c, g)) return pipe_smem_bytes(c, g);
    if (tc_fused_supported(c))
        return make_playout(g.n_off, c.caps.tile, c.caps.nb, c.caps.ang, c.basis.n_species, kTcParStride, kPWarps,
                            true)
            .total;
    return make_playout(g.n_off, c.caps.tile, c.caps.nb, c.caps.ang, fused_supported(c) ? c.basis.n_species : 0,
                        net.stride)
        .total;
}

cudaError_t launch_fused_potential(Context &c, const Grid &g, int n) {
    if (!c.md_prezeroed) {
        cudaError_t e = cudaMemsetAsync(c.d_stats, 0, sizeof(unsigned long long) * 4, c.stream);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(c.d_F4, 0, sizeof(float4) * (size_t)(n > 0 ? n : 1), c.stream);
        if (e != cudaSuccess) return e;
    }
    c.last_pipe = g.ncell > 0 && pipe_supported(c, g);
    if (c.last_pipe) return launch_pipe(c, g);
    return dispatch<kFused>(c, g);
}

cudaError_t launch_fp_forward(Context &c, const Grid &g, int n) {
    (void)n;
    cudaError_t e = cudaMemsetAsync(c.d_stats, 0, sizeof(unsigned long long) * 4, c.stream);
    if (e != cudaSuccess) return e;
    return dispatch<kDescriptor>(c, g);
}

cudaError_t launch_fp_backward(Context &c, const Grid &g, int n) {
    cudaError_t e = cudaMemsetAsync(c.d_F4, 0, sizeof(float4) * (size_t)(n > 0 ? n : 1), c.stream);
    if (e != cudaSuccess) return e;
    return dispatch<kForces>(c, g);
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
__global__ void k_scan_cells(int ncell, int *__restrict__ count, int *__restrict__ start);
__global__ void k_scatter(int n, const float4 *__restrict__ tmp4, const int *__restrict__ cell_of,
                          int *__restrict__ slot, const int *__restrict__ cell_start,
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
    const FusedNet net{};  // no network in descriptor mode
    const size_t smem = make_playout(g.n_off, caps.tile, caps.nb, caps.ang, 0, 0).total;
    auto kern = k_potential<KRT, KAT, EXACT, kDescriptor, false, 32>;
    cudaError_t e = allow_max_smem(kern);
    if (e != cudaSuccess) return e;
    kern<<<g.ncell, kPThreads, smem, st>>>(B, net, g, nullptr, 0, caps, pos4, cell_start, nullptr, nullptr, nullptr,
                                           nullptr,
                                           nullptr, Gs, nullptr, nullptr, nullptr, stats, err, nullptr, nullptr,
                                           g.ncell, nullptr, nullptr, 1, 0, TcNet{});
    return cudaGetLastError();
}

// Attributes (static shared memory) of the descriptor kernel form for (Kr, Ka).
cudaError_t na_kernel_attributes(int Kr, int Ka, cudaFuncAttributes *fa) {
    if (Kr == 17 && Ka == 9) return cudaFuncGetAttributes(fa, k_potential<17, 9, true, kDescriptor, false, 32>);
    if (Kr == 21 && Ka == 7) return cudaFuncGetAttributes(fa, k_potential<21, 7, true, kDescriptor, false, 32>);
    if (Kr <= 20 && Ka <= 12) return cudaFuncGetAttributes(fa, k_potential<20, 12, false, kDescriptor, false, 32>);
    return cudaFuncGetAttributes(fa, k_potential<24, 8, false, kDescriptor, false, 32>);
}

int na_fail(int code, const char *msg) {
    set_context_free_error(msg);
    return code;
}

// Device memory of the current device, or managed memory (reachable from it).
// Device memory of another GPU is refused: the kernels run on the current
// device and would fault on it unless peer access happened to be enabled.
bool na_is_device(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
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
    int cur_dev = 0;
    if (cudaGetDevice(&cur_dev) != cudaSuccess) return na_fail(AENET_E_CUDA, "cudaGetDevice failed");
    if (n > 0 && (!pos || !types || !G || !na_is_device(pos, cur_dev) || !na_is_device(types, cur_dev) ||
                  !na_is_device(G, cur_dev)))
        return na_fail(AENET_E_ARG, "pos, types and G must be device pointers of the current device");
    Basis B{};
    B.n_species = n_species;
    B.Kr = Kr;
    B.Ka = Ka;
    B.D = D;
    B.rc_rad = (float)rc_rad;
    B.rc_ang = (float)rc_ang;
    B.rc_max = (float)(rc_rad > rc_ang ? rc_rad : rc_ang);
    detail::sh_legendre_of_chebyshev(B.sh_b);
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

    // mean-density capacities (as for a context), one regrow on overflow
    const double rho = n / (box[0] * box[1] * box[2]);
    auto cap = [&](double rc, double margin) {
        int k = (int)(1.3 * rho * 4.18879020478639 * rc * rc * rc + margin);
        return ((k + 15) / 16) * 16;
    };
    Caps caps{};
    caps.nb = cap(B.rc_max, 32.0) > 64 ? cap(B.rc_max, 32.0) : 64;
    caps.ang = cap(B.rc_ang, 24.0) > 32 ? cap(B.rc_ang, 24.0) : 32;
    int tl = (int)(1.25 * ((double)n / g.ncell) * g.n_off + 64.0);
    tl = ((tl + 31) / 32) * 32;
    caps.tile = tl < 128 ? 128 : (tl > 1024 ? 1024 : tl);
    // dynamic shared memory available to the descriptor kernel: the opt-in
    // limit minus its static shared memory (what allow_max_smem grants)
    int optin = 0;
    cudaFuncAttributes fa{};
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, cur_dev) != cudaSuccess ||
        na_kernel_attributes(Kr, Ka, &fa) != cudaSuccess)
        return na_fail(AENET_E_CUDA, "device attributes of the descriptor kernel");
    const size_t smem_avail = optin > (int)fa.sharedSizeBytes ? (size_t)(optin - (int)fa.sharedSizeBytes) : 0;
    unsigned w = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (make_playout(g.n_off, caps.tile, caps.nb, caps.ang, 0, 0).total > smem_avail)
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
        caps.tile = 1024;
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

namespace aenet {
int activation_record_len(const Net &net) { return make_fused_net(net).rec_len; }
}  // namespace aenet
