// C ABI of the library (declared in include/aenet_gpu.h): context set-up, the
// energy/force/virial evaluation, the descriptor-only entry point and the
// graph-captured velocity-Verlet NVE propagator.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <new>

#include "aenet_internal.cuh"
#include "sh_angular.cuh"

struct aenet_ctx {
    aenet::Context c;
};

namespace aenet {

cudaError_t prepare_bf16_weights(Context &c);

namespace {

thread_local std::string g_setup_error;

int fail(Context *c, int code, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(Context *c, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf; else g_setup_error = buf;
    return code;
}

int cuda_fail(Context *c, cudaError_t e, const char *where) {
    return fail(c, AENET_E_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call, where)                                  \
    do {                                                 \
        cudaError_t _e = (call);                         \
        if (_e != cudaSuccess) return cuda_fail(&c, _e, where); \
    } while (0)

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <class T>
cudaError_t grow(T *&p, size_t have, size_t need) {
    if (need <= have && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    return cudaMalloc(&p, sizeof(T) * (need > 0 ? need : 1));
}

// Cell grid of a box: cells at least rc_cut (default: the largest cutoff) thick
// along each lattice direction, and the (2m+1)^3 image-cell window that covers
// rc_cut. tilt (xy, xz, yz) or NULL: the restricted triclinic cell. A
// displacement of length <= rc has a fractional component along lattice
// vector k of at most rc / w_k (w_k the distance between the cell's faces
// across k), so cell indices differ by at most m_k = ceil(rc nc_k / w_k).
int make_grid(Context &c, const double *box, Grid &g, double rc_cut = 0.0, const double *tilt = nullptr) {
    const double rc = rc_cut > 0.0 ? rc_cut : c.basis.rc_max;
    g.ncell = 1;
    g.n_off = 1;
    for (int a = 0; a < 3; ++a) {
        if (!(box[a] > 0.0) || !isfinite(box[a])) return fail(&c, AENET_E_ARG, "box[%d] must be finite and > 0", a);
        g.tilt[a] = tilt ? tilt[a] : 0.0;
        if (!isfinite(g.tilt[a])) return fail(&c, AENET_E_ARG, "box tilt %d must be finite", a);
    }
    g.tri = g.tilt[0] != 0.0 || g.tilt[1] != 0.0 || g.tilt[2] != 0.0;
    double w[3] = {box[0], box[1], box[2]};
    if (g.tri) {  // face distances: volume / |b x c|, volume / |c x a|, L_z
        const double xy = g.tilt[0], xz = g.tilt[1], yz = g.tilt[2];
        const double V = box[0] * box[1] * box[2];
        w[0] = V / sqrt(box[1] * box[2] * box[1] * box[2] + xy * box[2] * xy * box[2] +
                        (xy * yz - box[1] * xz) * (xy * yz - box[1] * xz));
        w[1] = V / (box[0] * sqrt(box[2] * box[2] + yz * yz));
        w[2] = box[2];
    }
    for (int a = 0; a < 3; ++a) {
        int nc = (int)floor(w[a] / rc);
        if (nc < 1) nc = 1;
        if (nc > 1024) nc = 1024;
        g.nc[a] = nc;
        g.box[a] = box[a];
        g.h[a] = box[a] / nc;
        g.hf[a] = (float)g.h[a];
        g.inv_box[a] = 1.0 / g.box[a];
        g.inv_h[a] = 1.0 / g.h[a];
        g.m[a] = g.tri ? (int)ceil(rc * nc / w[a]) : (int)ceil(rc / g.h[a]);
        g.ncell *= nc;
        g.n_off *= 2 * g.m[a] + 1;
    }
    g.ht[0] = g.tilt[0] / g.nc[1];
    g.ht[1] = g.tilt[1] / g.nc[2];
    g.ht[2] = g.tilt[2] / g.nc[2];
    for (int a = 0; a < 3; ++a) g.htf[a] = (float)g.ht[a];
    if (g.n_off > 4096)
        return fail(&c, AENET_E_ARG, "box too small for the cutoff: %d image cells per atom (limit 4096)", g.n_off);
    return AENET_OK;
}

// Neighbour-list capacities from the mean density: 1.3x the expected count plus
// a margin, rounded to 16; the staging tile holds 1.25x the mean neighbourhood
// of a cell (at most 1024 atoms; larger neighbourhoods are staged in chunks).
Caps estimate_caps(const Context &c, int n, const Grid &g) {
    const double V = g.box[0] * g.box[1] * g.box[2];
    const double rho = n / V;
    auto cap = [&](double rc, double margin) {
        double e = rho * 4.18879020478639 * rc * rc * rc;
        int k = (int)(1.3 * e + margin);
        return ((k + 15) / 16) * 16;
    };
    Caps k;
    k.nb = std::max(64, cap(c.basis.rc_max, 32.0));
    k.ang = std::max(32, cap(c.basis.rc_ang, 24.0));
    const double per_cell = (double)n / g.ncell;
    int tile = (int)(1.25 * per_cell * g.n_off + 64.0);
    tile = ((tile + 31) / 32) * 32;
    k.tile = std::min(1024, std::max(128, tile));
    return k;
}

int ensure(Context &c, int n, const Grid &g) {
    if (n > c.cap_atoms || !c.d_pos4) {
        n = std::max(n, 1);
        size_t N = (size_t)n;
        const int D = c.basis.D;
        CK(grow(c.d_pos4, 0, N), "cudaMalloc");
        CK(grow(c.d_tmp4, 0, N), "cudaMalloc");
        CK(grow(c.d_perm, 0, N), "cudaMalloc");
        CK(grow(c.d_cell_of, 0, N), "cudaMalloc");
        CK(grow(c.d_slot, 0, N), "cudaMalloc");
        CK(grow(c.d_G, 0, N * D), "cudaMalloc");
        CK(grow(c.d_dEdG, 0, N * D), "cudaMalloc");
        CK(grow(c.d_eatom, 0, N), "cudaMalloc");
        CK(grow(c.d_F4, 0, N), "cudaMalloc");
        CK(grow(c.d_ke_part, 0, 11 * ((N + 255) / 256 + 1)), "cudaMalloc");  // an 11-entry row per MD CTA
        CK(grow(c.d_sp_rank, 0, N), "cudaMalloc");
        CK(grow(c.d_sp_list, 0, N), "cudaMalloc");
        c.cap_atoms = n;
        ++c.buf_gen;
    }
    if (g.ncell > c.cap_cells) {
        CK(grow(c.d_cell_count, 0, (size_t)g.ncell), "cudaMalloc");
        // zero from the start: every scan clears the counts it reads, so the MD
        // step's binning relies on finding them zero
        CK(cudaMemsetAsync(c.d_cell_count, 0, sizeof(int) * (size_t)g.ncell, c.stream), "cudaMemsetAsync");
        CK(grow(c.d_cell_start, 0, (size_t)g.ncell + 1), "cudaMalloc");
        CK(grow(c.d_vir_part, 0, (size_t)g.ncell * kMaxSplit * 9), "cudaMalloc");  // a row per cell part
        c.cap_cells = g.ncell;
        ++c.buf_gen;
    }
    if (c.keep_act && (n > c.cap_act || !c.d_act)) {
        CK(grow(c.d_act, 0, (size_t)std::max(n, 1) * activation_record_len(c.net)), "cudaMalloc");
        c.cap_act = std::max(n, 1);
        ++c.buf_gen;
    }
    const int need_e =
        std::max(std::max(ann_blocks(std::max(n, 1)), g.ncell * kMaxSplit), tcgen05_tiles(c, std::max(n, 1))) + 1;
    if (need_e > c.cap_blocks || !c.d_e_part) {
        CK(grow(c.d_e_part, 0, (size_t)need_e), "cudaMalloc");
        c.cap_blocks = need_e;
        ++c.buf_gen;
    }
    return AENET_OK;
}

int ensure_stage(Context &c, int n) {
    if (n > c.cap_stage || !c.d_pos) {
        n = std::max(n, 1);
        size_t N = (size_t)n;
        CK(grow(c.d_pos, 0, 3 * N), "cudaMalloc");
        CK(grow(c.d_vel, 0, 3 * N), "cudaMalloc");
        CK(grow(c.d_forces, 0, 3 * N), "cudaMalloc");
        CK(grow(c.d_eatom_out, 0, N), "cudaMalloc");
        CK(grow(c.d_types, 0, N), "cudaMalloc");
        c.cap_stage = n;
        ++c.buf_gen;
    }
    return AENET_OK;
}

int check_smem(Context &c, const Grid &g) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t need = potential_smem_bytes(c, g) + 1024;  // + the kernel's static shared memory
    if (optin > 0 && need > (size_t)optin)
        return fail(&c, AENET_E_CAPACITY, "neighbour lists need %zu B of shared memory (limit %d B)", need, optin);
    return AENET_OK;
}

// Stage event k of the MD step (an event-record node inside the captured graph)
// when c.ev_mask selects it. Each node costs the step ~2 us of device time, so
// the light timing mode records only the events around the potential.
cudaError_t mark(Context &c, int k) {
    if (!((c.ev_mask >> k) & 1u)) return cudaSuccess;
    return cudaEventRecordWithFlags(c.ev[k], c.stream, cudaEventRecordExternal);
}

// Descriptor, networks and forces after the cell list (fused kernel or the
// three split kernels), with stage events 3, 4 (after descriptor, network) and
// 5 (after forces) when selected. *n_eparts = number of energy partials written.
int enqueue_potential(Context &c, const Grid &g, int n, int *n_eparts) {
    if (fused_path(c)) {
        // descriptor, network and forces in one kernel: their stage events coincide
        CK(mark(c, 3), "event");
        CK(mark(c, 4), "event");
        if (fused_supported(c))
            CK(launch_fused_potential(c, g, n), "potential kernel");
        else
            CK(launch_fused_tc(c, g, n), "potential kernel (tensor-core network)");
        *n_eparts = c.pot_parts;
        c.last_epart = c.d_e_part;
        c.last_eparts = c.pot_parts;
        c.last_vpart = c.d_vir_part;
        c.last_vparts = c.pot_parts;
    } else {
        CK(launch_fp_forward(c, g, n), "descriptor kernel");
        CK(mark(c, 3), "event");
        if (c.precision == AENET_FP32) {
            CK(launch_ann(c, n), "network kernel");
            *n_eparts = ann_blocks(n);
        } else {
            CK(launch_ann_tcgen05(c, n), "BF16 network kernel");
            *n_eparts = tcgen05_eparts(c, n);
        }
        CK(mark(c, 4), "event");
        CK(launch_fp_backward(c, g, n), "force kernel");
        c.last_epart = c.d_e_part;
        c.last_eparts = *n_eparts;
        c.last_vpart = c.d_vir_part;
        c.last_vparts = c.pot_parts;
    }
    c.maps_n = n;          // the cell maps now describe this evaluation
    c.vl_valid = false;    // and no Verlet list matches them
    CK(mark(c, 5), "event");
    return AENET_OK;
}

// The whole path on device buffers, enqueued on c.stream (no synchronisation).
// *n_eparts (optional) receives the number of energy partials.
int enqueue_compute(Context &c, const Grid &g, int n, const double *pos, const int32_t *types, double *forces,
                    double *e_atom, int *n_eparts_out = nullptr) {
    int rc = check_smem(c, g);
    if (rc) return rc;
    CK(launch_cells(c, g, n, pos, types), "cell list");
    int n_eparts = 0;
    if ((rc = enqueue_potential(c, g, n, &n_eparts))) return rc;
    CK(launch_finalize(c, g, n, n_eparts, forces, e_atom), "reductions");
    if (n_eparts_out) *n_eparts_out = n_eparts;
    return AENET_OK;
}

int read_error_word(Context &c) {
    unsigned w = 0;
    CK(cudaMemcpyAsync(&w, c.d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream), "cudaMemcpyAsync");
    CK(cudaStreamSynchronize(c.stream), "cudaStreamSynchronize");
    if (w) CK(cudaMemsetAsync(c.d_err, 0, sizeof(unsigned), c.stream), "cudaMemsetAsync");
    if (w & kErrType) return fail(&c, AENET_E_ARG, "species index out of range");
    if (w & kErrNonfinite) return fail(&c, AENET_E_NONFINITE, "non-finite coordinate");
    if (w & kErrOverlap) return fail(&c, AENET_E_OVERLAP, "two image-atoms closer than 1e-6 A");
    if (w & (kErrNbCap | kErrAngCap))
        return fail(&c, AENET_E_CAPACITY, "neighbour list overflow (capacity %d / %d)", c.caps.nb, c.caps.ang);
    if (w & kErrTimeout) return fail(&c, AENET_E_TIMEOUT, "a bounded wait inside the potential kernel gave up");
    return AENET_OK;
}

// Stage a host-or-device array into a device buffer.
template <class T>
int stage_in(Context &c, const T *src, T *dev_buf, size_t count, const T **out) {
    if (!src || count == 0) {
        *out = src;
        return AENET_OK;
    }
    if (is_device_ptr(src)) {
        *out = src;
        return AENET_OK;
    }
    CK(cudaMemcpyAsync(dev_buf, src, sizeof(T) * count, cudaMemcpyHostToDevice, c.stream), "cudaMemcpyAsync");
    *out = dev_buf;
    return AENET_OK;
}

int validate_types_host(Context &c, int n, const int32_t *types) {
    if (is_device_ptr(types)) return AENET_OK;  // device arrays are range-checked by the binning kernel
    for (int i = 0; i < n; ++i)
        if (types[i] < 0 || types[i] >= c.basis.n_species)
            return fail(&c, AENET_E_ARG, "types[%d] = %d out of range [0, %d)", i, types[i], c.basis.n_species);
    return AENET_OK;
}

void destroy_graph(Context &c) {
    if (c.md_exec) cudaGraphExecDestroy(c.md_exec);
    c.md_exec = nullptr;
    c.md_key.n = -1;
}

}  // namespace

void set_context_free_error(const char *msg) { g_setup_error = msg; }

}  // namespace aenet

using namespace aenet;

extern "C" int aenet_setup(aenet_ctx **out, const aenet_model_desc *m, int precision, void *stream) {
    if (!out) return fail(nullptr, AENET_E_ARG, "out is NULL");
    *out = nullptr;
    if (!m) return fail(nullptr, AENET_E_ARG, "model is NULL");
    if (m->n_species < 1 || m->n_species > kMaxSpecies)
        return fail(nullptr, AENET_E_ARG, "n_species must be in [1, %d]", kMaxSpecies);
    if (!m->type_weight || !m->widths || !m->params) return fail(nullptr, AENET_E_ARG, "NULL model array");
    if (!(m->rc_rad > 0.0) || !(m->rc_ang > 0.0)) return fail(nullptr, AENET_E_ARG, "cutoffs must be > 0");
    if (m->order_rad < 0 || m->order_ang < 0 || m->order_rad > kMaxOrder || m->order_ang > kMaxOrder)
        return fail(nullptr, AENET_E_ARG, "orders must be in [0, %d]", kMaxOrder);
    const int Kr = m->order_rad + 1, Ka = m->order_ang + 1, D = 2 * (Kr + Ka);
    const bool supported = (Kr == 17 && Ka == 9) || (Kr == 21 && Ka == 7) || (Kr <= 20 && Ka <= 12) ||
                           (Kr <= 24 && Ka <= 8);
    if (!supported || D > kMaxD)
        return fail(nullptr, AENET_E_ARG,
                    "unsupported basis orders (%d, %d): need (N_r+1, N_a+1) <= (20, 12) or (24, 8)", Kr, Ka);
    if (m->n_layers < 2 || m->n_layers > kMaxLayers)
        return fail(nullptr, AENET_E_ARG, "n_layers must be in [2, %d]", kMaxLayers);
    if (m->widths[0] != D) return fail(nullptr, AENET_E_ARG, "widths[0] = %d but D = %d", m->widths[0], D);
    if (m->widths[m->n_layers] != 1) return fail(nullptr, AENET_E_ARG, "output width must be 1");
    for (int l = 1; l < m->n_layers; ++l)
        if (m->widths[l] < 1 || m->widths[l] > kMaxWidth)
            return fail(nullptr, AENET_E_ARG, "hidden width %d out of [1, %d]", m->widths[l], kMaxWidth);
    if (precision != AENET_FP32 && precision != AENET_BF16 && precision != AENET_BF16X3)
        return fail(nullptr, AENET_E_ARG, "unknown precision %d", precision);
    if (precision != AENET_FP32 && !(m->n_layers == 3 && m->widths[1] <= 32 && m->widths[2] <= 32))
        return fail(nullptr, AENET_E_ARG, "the BF16 forms need two hidden layers of width <= 32");

    aenet_ctx *h = new (std::nothrow) aenet_ctx();
    if (!h) return fail(nullptr, AENET_E_NOMEM, "host allocation failed");
    Context &c = h->c;
    cudaGetDevice(&c.device);
    c.precision = precision;
    c.stream = (cudaStream_t)stream;
    if (!c.stream) {
        cudaError_t e = cudaStreamCreate(&c.stream);
        if (e != cudaSuccess) {
            delete h;
            return fail(nullptr, AENET_E_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        }
        c.own_stream = true;
    }
    c.basis.n_species = m->n_species;
    c.basis.Kr = Kr;
    c.basis.Ka = Ka;
    c.basis.D = D;
    c.basis.rc_rad = (float)m->rc_rad;
    c.basis.rc_ang = (float)m->rc_ang;
    c.basis.rc_max = (float)std::max(m->rc_rad, m->rc_ang);
    detail::sh_legendre_of_chebyshev(c.basis.sh_b);
    for (int t = 0; t < kMaxSpecies; ++t) c.basis.type_weight[t] = t < m->n_species ? (float)m->type_weight[t] : 0.f;
    c.net.n_species = m->n_species;
    c.net.n_layers = m->n_layers;
    c.net.act_len = 0;
    c.net.n_params = 0;
    for (int l = 0; l <= kMaxLayers; ++l) c.net.widths[l] = l <= m->n_layers ? m->widths[l] : 0;
    for (int l = 0; l <= m->n_layers; ++l) c.net.act_len += m->widths[l];
    for (int l = 1; l <= m->n_layers; ++l) c.net.n_params += m->widths[l] * m->widths[l - 1] + m->widths[l];
    if (m->mass) c.mass.assign(m->mass, m->mass + m->n_species);

    const size_t NP = (size_t)m->n_species * c.net.n_params;
    std::vector<float> P(NP), sh((size_t)m->n_species * D, 0.f), sc((size_t)m->n_species * D, 1.f);
    for (size_t k = 0; k < NP; ++k) P[k] = (float)m->params[k];
    for (size_t k = 0; k < sh.size(); ++k) {
        if (m->in_shift) sh[k] = (float)m->in_shift[k];
        if (m->in_scale) sc[k] = (float)m->in_scale[k];
    }
    auto setup_fail = [&](cudaError_t e, const char *what) {
        g_setup_error = std::string(what) + ": " + cudaGetErrorString(e);
        aenet_destroy(h);
        return AENET_E_CUDA;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&c.d_params, sizeof(float) * NP)) != cudaSuccess) return setup_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&c.d_shift, sizeof(float) * sh.size())) != cudaSuccess) return setup_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&c.d_scale, sizeof(float) * sc.size())) != cudaSuccess) return setup_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&c.d_err, sizeof(unsigned))) != cudaSuccess) return setup_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&c.d_stats, sizeof(unsigned long long) * 4)) != cudaSuccess)
        return setup_fail(e, "cudaMalloc");
    for (int k = 0; k <= Context::kStages; ++k)
        if ((e = cudaEventCreate(&c.ev[k])) != cudaSuccess) return setup_fail(e, "cudaEventCreate");
    if ((e = cudaMalloc(&c.d_step, sizeof(int))) != cudaSuccess) return setup_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&c.d_done, sizeof(unsigned))) != cudaSuccess) return setup_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&c.d_sp_cnt, sizeof(int) * kMaxSpecies)) != cudaSuccess) return setup_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&c.d_sp_off, sizeof(int) * kMaxSpecies)) != cudaSuccess) return setup_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&c.d_result, sizeof(double) * 11)) != cudaSuccess) return setup_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&c.d_mass, sizeof(double) * kMaxSpecies)) != cudaSuccess) return setup_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&c.d_work, 2 * sizeof(unsigned))) != cudaSuccess) return setup_fail(e, "cudaMalloc");
    if ((e = cudaMemset(c.d_work, 0, 2 * sizeof(unsigned))) != cudaSuccess) return setup_fail(e, "cudaMemset");
    if ((e = cudaDeviceGetAttribute(&c.n_sm, cudaDevAttrMultiProcessorCount, c.device)) != cudaSuccess)
        return setup_fail(e, "cudaDeviceGetAttribute");
    double masses[kMaxSpecies] = {0};
    for (int t = 0; t < m->n_species && m->mass; ++t) masses[t] = m->mass[t];
    if ((e = cudaMemcpy(c.d_params, P.data(), sizeof(float) * NP, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(c.d_shift, sh.data(), sizeof(float) * sh.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(c.d_scale, sc.data(), sizeof(float) * sc.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(c.d_mass, masses, sizeof(masses), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(c.d_err, 0, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMemset(c.d_done, 0, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMemset(c.d_sp_cnt, 0, sizeof(int) * kMaxSpecies)) != cudaSuccess ||
        (e = cudaMemset(c.d_stats, 0, sizeof(unsigned long long) * 4)) != cudaSuccess ||
        (e = cudaMemset(c.d_result, 0, sizeof(double) * 11)) != cudaSuccess)
        return setup_fail(e, "cudaMemcpy");
    if (precision != AENET_FP32) {
        if ((e = prepare_bf16_weights(c)) != cudaSuccess) return setup_fail(e, "BF16 weights");
    }
    {
        const std::vector<int2> pairs = grad_pairs(c.net);
        if ((e = cudaMalloc(&c.d_wpairs, sizeof(int2) * pairs.size())) != cudaSuccess ||
            (e = cudaMemcpy(c.d_wpairs, pairs.data(), sizeof(int2) * pairs.size(), cudaMemcpyHostToDevice)) !=
                cudaSuccess ||
            (e = cudaMalloc(&c.d_dEdW, sizeof(double) * NP)) != cudaSuccess)
            return setup_fail(e, "gradient tables");
    }
    *out = h;
    return AENET_OK;
}

extern "C" int aenet_set_stream(aenet_ctx *h, void *stream) {
    if (!h) return AENET_E_ARG;
    Context &c = h->c;
    if (!stream) return fail(&c, AENET_E_ARG, "stream must not be NULL");
    if (c.own_stream && c.stream) {
        cudaStreamSynchronize(c.stream);
        cudaStreamDestroy(c.stream);
        c.own_stream = false;
    }
    c.stream = (cudaStream_t)stream;
    destroy_graph(c);
    return AENET_OK;
}

static int compute_impl(Context &c, int n, const double *pos, const int32_t *types, const double *box,
                        double *energy, double *forces, double *virial, double *e_atom, float *G_out) {
    cudaGetLastError();  // a stale error of an unrelated earlier call must not be reported as ours
    if (n < 0) return fail(&c, AENET_E_ARG, "n_atoms < 0");
    if (!box) return fail(&c, AENET_E_ARG, "box is NULL");
    if (n > 0 && (!pos || !types)) return fail(&c, AENET_E_ARG, "pos/types NULL");
    Grid g;
    int rc = make_grid(c, box, g, 0.0, c.tilt);
    if (rc) return rc;
    if ((rc = validate_types_host(c, n, types))) return rc;
    if ((rc = ensure(c, n, g)) || (rc = ensure_stage(c, n))) return rc;
    if (c.caps.nb == 0) c.caps = estimate_caps(c, n, g);
    const double *dpos;
    const int32_t *dtypes;
    if ((rc = stage_in(c, pos, c.d_pos, 3 * (size_t)n, &dpos))) return rc;
    if ((rc = stage_in(c, types, c.d_types, (size_t)n, &dtypes))) return rc;
    const bool f_dev = is_device_ptr(forces), ea_dev = is_device_ptr(e_atom), G_dev = is_device_ptr(G_out);
    double *dF = forces ? (f_dev ? forces : c.d_forces) : nullptr;
    double *dE = e_atom ? (ea_dev ? e_atom : c.d_eatom_out) : nullptr;
    for (int attempt = 0; attempt < 2; ++attempt) {
        CK(cudaMemsetAsync(c.d_err, 0, sizeof(unsigned), c.stream), "cudaMemsetAsync");
        if (G_out) {
            if ((rc = check_smem(c, g))) return rc;
            CK(launch_cells(c, g, n, dpos, dtypes), "cell list");
            CK(launch_fp_forward(c, g, n), "descriptor kernel");
        } else {
            if ((rc = enqueue_compute(c, g, n, dpos, dtypes, dF, dE))) return rc;
        }
        rc = read_error_word(c);
        if (rc != AENET_E_CAPACITY || attempt == 1) break;
        c.caps.nb *= 2;  // regrow once and retry
        c.caps.ang *= 2;
        c.caps.tile = 1024;
        destroy_graph(c);
    }
    if (rc) return rc;
    if (G_out) {
        if (G_dev) {
            CK(launch_unsort_G(c, n, G_out), "unsort");
        } else {
            float *tmp = nullptr;
            CK(cudaMalloc(&tmp, sizeof(float) * (size_t)n * c.basis.D + 4), "cudaMalloc");
            cudaError_t e1 = launch_unsort_G(c, n, tmp);
            cudaError_t e2 = e1 == cudaSuccess ? cudaMemcpyAsync(G_out, tmp, sizeof(float) * (size_t)n * c.basis.D,
                                                                 cudaMemcpyDeviceToHost, c.stream)
                                               : e1;
            cudaError_t e3 = cudaStreamSynchronize(c.stream);
            cudaFree(tmp);
            if (e2 != cudaSuccess) return cuda_fail(&c, e2, "descriptor copy");
            if (e3 != cudaSuccess) return cuda_fail(&c, e3, "cudaStreamSynchronize");
        }
        CK(cudaStreamSynchronize(c.stream), "cudaStreamSynchronize");
        return AENET_OK;
    }
    c.act_valid = c.keep_act;
    c.act_atoms = n;
    if (energy) CK(cudaMemcpyAsync(energy, c.d_result, sizeof(double), cudaMemcpyDefault, c.stream), "energy copy");
    if (virial)
        CK(cudaMemcpyAsync(virial, c.d_result + 1, 9 * sizeof(double), cudaMemcpyDefault, c.stream), "virial copy");
    if (forces && !f_dev)
        CK(cudaMemcpyAsync(forces, c.d_forces, 3 * sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, c.stream),
           "forces copy");
    if (e_atom && !ea_dev)
        CK(cudaMemcpyAsync(e_atom, c.d_eatom_out, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, c.stream),
           "e_atom copy");
    CK(cudaStreamSynchronize(c.stream), "cudaStreamSynchronize");
    return AENET_OK;
}

extern "C" int aenet_compute(aenet_ctx *h, int n, const double *pos, const int32_t *types, const double *box,
                             double *energy, double *forces, double *virial, double *e_atom) {
    if (!h) return fail(nullptr, AENET_E_ARG, "ctx is NULL");
    return compute_impl(h->c, n, pos, types, box, energy, forces, virial, e_atom, nullptr);
}

extern "C" int aenet_compute_async(aenet_ctx *h, int n, const double *pos, const int32_t *types, const double *box,
                                   double *energy, double *forces, double *virial, double *e_atom) {
    if (!h) return fail(nullptr, AENET_E_ARG, "ctx is NULL");
    Context &c = h->c;
    cudaGetLastError();
    if (n < 1) return fail(&c, AENET_E_ARG, "n_atoms < 1");
    if (!box) return fail(&c, AENET_E_ARG, "box is NULL");
    const void *arrays[] = {pos, types, energy, forces, virial, e_atom};
    for (int k = 0; k < 6; ++k)
        if ((k < 2 || arrays[k]) && !is_device_ptr(arrays[k]))
            return fail(&c, AENET_E_ARG, "aenet_compute_async takes device pointers only (argument %d)", k);
    Grid g;
    int rc = make_grid(c, box, g, 0.0, c.tilt);
    if (rc) return rc;
    if ((rc = ensure(c, n, g))) return rc;
    if (c.caps.nb == 0) c.caps = estimate_caps(c, n, g);
    if ((rc = enqueue_compute(c, g, n, pos, types, forces, e_atom))) return rc;
    c.act_valid = c.keep_act;
    c.act_atoms = n;
    if (energy) CK(cudaMemcpyAsync(energy, c.d_result, sizeof(double), cudaMemcpyDeviceToDevice, c.stream), "energy");
    if (virial)
        CK(cudaMemcpyAsync(virial, c.d_result + 1, 9 * sizeof(double), cudaMemcpyDeviceToDevice, c.stream), "virial");
    return AENET_OK;
}

// ------------------------------------------------------------ batched form
// Many periodic structures in one evaluation: per-structure cell grids in one
// global cell index space; one launch of each kernel over all cells.
namespace aenet {
namespace {

struct BatchLayout {
    std::vector<StructInfo> info;  // per structure
    std::vector<int> order;        // cells, heaviest first
    Grid gall{};                   // ncell = all cells, n_off = largest image table
    int n = 0;                     // atoms
    double max_rho = 0.0, max_neigh = 0.0;
};

int batch_layout(Context &c, int n_struct, const int64_t *atom_offset, const double *boxes, BatchLayout &L) {
    if (n_struct < 1 || !atom_offset || !boxes) return fail(&c, AENET_E_ARG, "bad batch description");
    if (atom_offset[0] != 0) return fail(&c, AENET_E_ARG, "atom_offset[0] must be 0");
    for (int s = 0; s < n_struct; ++s)
        if (atom_offset[s + 1] < atom_offset[s]) return fail(&c, AENET_E_ARG, "atom_offset must be non-decreasing");
    if (atom_offset[n_struct] > INT32_MAX / 2) return fail(&c, AENET_E_ARG, "too many atoms");
    L.n = (int)atom_offset[n_struct];
    L.info.assign((size_t)n_struct, StructInfo{});
    int total_cells = 0, max_off = 1;
    std::vector<double> work_of((size_t)n_struct);
    for (int s = 0; s < n_struct; ++s) {
        StructInfo &si = L.info[s];
        int rc = make_grid(c, boxes + 3 * (size_t)s, si.g);
        if (rc) return rc;
        if ((long long)total_cells + si.g.ncell > INT32_MAX / 2) return fail(&c, AENET_E_ARG, "too many cells");
        si.cell0 = total_cells;
        si.ncell = si.g.ncell;
        si.atom0 = (int)atom_offset[s];
        si.natoms = (int)(atom_offset[s + 1] - atom_offset[s]);
        total_cells += si.g.ncell;
        max_off = std::max(max_off, si.g.n_off);
        const double V = boxes[3 * s] * boxes[3 * s + 1] * boxes[3 * s + 2];
        const double per_cell = (double)si.natoms / si.g.ncell;
        L.max_rho = std::max(L.max_rho, si.natoms / V);
        L.max_neigh = std::max(L.max_neigh, per_cell * si.g.n_off);
        // work of one cell ~ its atoms x the image-atoms each of them scans
        work_of[s] = per_cell * (per_cell * si.g.n_off);
    }
    L.gall = Grid{};
    L.gall.ncell = total_cells;
    L.gall.n_off = max_off;
    L.order.resize((size_t)total_cells);
    std::vector<int> sorder((size_t)n_struct);
    for (int s = 0; s < n_struct; ++s) sorder[s] = s;
    std::stable_sort(sorder.begin(), sorder.end(), [&](int a, int b) { return work_of[a] > work_of[b]; });
    int k = 0;
    for (int s : sorder)
        for (int q = 0; q < L.info[s].ncell; ++q) L.order[k++] = L.info[s].cell0 + q;
    return AENET_OK;
}

// Work buffers and neighbour-list capacities for a batch (capacities from the
// densest structure, staging tile from the largest neighbourhood of a cell).
int batch_buffers(Context &c, const BatchLayout &L) {
    int rc;
    if ((rc = ensure(c, L.n, L.gall)) || (rc = ensure_stage(c, L.n))) return rc;
    if (c.caps.nb == 0) {
        Grid dens{};
        dens.box[0] = dens.box[1] = dens.box[2] = 1.0;
        dens.ncell = 1;
        dens.n_off = 1;
        c.caps = estimate_caps(c, 0, dens);
        auto cap = [&](double rcut, double margin) {
            const int k = (int)(1.3 * L.max_rho * 4.18879020478639 * rcut * rcut * rcut + margin);
            return ((k + 15) / 16) * 16;
        };
        c.caps.nb = std::max(64, cap(c.basis.rc_max, 32.0));
        c.caps.ang = std::max(32, cap(c.basis.rc_ang, 24.0));
        c.caps.tile = std::min(1024, std::max(128, (((int)(1.25 * L.max_neigh + 64.0)) + 31) / 32 * 32));
    }
    return AENET_OK;
}

// The batched evaluation on device buffers, enqueued on c.stream: binning,
// cell sort, potential (persistent when c.persist), per-structure reductions,
// forces back in input order. sinfo/order: the layout on the device.
int batch_enqueue(Context &c, const BatchLayout &L, const StructInfo *sinfo, const int *order, const double *dpos,
                  const int32_t *dtypes, double *dF, double *energies, double *virials) {
    int rc = check_smem(c, L.gall);
    if (rc) return rc;
    c.batch_sinfo = sinfo;
    c.batch_order = order;
    c.batch_n = (int)L.info.size();
    cudaError_t e = launch_cells_batch(c, L.n, L.gall.ncell, dpos, dtypes);
    int n_eparts = 0;
    if (e == cudaSuccess) rc = enqueue_potential(c, L.gall, L.n, &n_eparts);
    if (e == cudaSuccess && !rc) e = launch_batch_reduce(c, energies, virials);
    if (e == cudaSuccess && !rc) e = launch_finalize_forces(c, L.n, dF);
    c.batch_sinfo = nullptr;
    c.batch_order = nullptr;
    c.batch_n = 0;
    if (e != cudaSuccess) return cuda_fail(&c, e, "batched evaluation");
    return rc;
}

int grow_order(Context &c, int cells) {
    if (cells > c.cap_order || !c.d_order) {
        CK(grow(c.d_order, 0, (size_t)cells), "cudaMalloc");
        c.cap_order = cells;
        ++c.buf_gen;
    }
    return AENET_OK;
}

}  // namespace
}  // namespace aenet

extern "C" int aenet_compute_batch(aenet_ctx *h, int n_struct, const int64_t *atom_offset, const double *pos,
                                   const int32_t *types, const double *boxes, double *energies, double *forces,
                                   double *virials) {
    if (!h) return fail(nullptr, AENET_E_ARG, "ctx is NULL");
    Context &c = h->c;
    cudaGetLastError();
    BatchLayout L;
    int rc = batch_layout(c, n_struct, atom_offset, boxes, L);
    if (rc) return rc;
    const int n = L.n;
    if (n > 0 && (!pos || !types)) return fail(&c, AENET_E_ARG, "pos/types NULL");
    if ((rc = validate_types_host(c, n, types))) return rc;
    if ((rc = batch_buffers(c, L))) return rc;
    if (n_struct > c.cap_struct) {
        CK(grow(c.d_sinfo, 0, (size_t)n_struct), "cudaMalloc");
        CK(grow(c.d_bres, 0, (size_t)n_struct * 10), "cudaMalloc");
        c.cap_struct = n_struct;
        ++c.buf_gen;
    }
    if ((rc = grow_order(c, L.gall.ncell))) return rc;
    const double *dpos;
    const int32_t *dtypes;
    if ((rc = stage_in(c, pos, c.d_pos, 3 * (size_t)n, &dpos))) return rc;
    if ((rc = stage_in(c, types, c.d_types, (size_t)n, &dtypes))) return rc;
    CK(cudaMemcpyAsync(c.d_sinfo, L.info.data(), sizeof(StructInfo) * n_struct, cudaMemcpyHostToDevice, c.stream),
       "cudaMemcpyAsync");
    CK(cudaMemcpyAsync(c.d_order, L.order.data(), sizeof(int) * L.order.size(), cudaMemcpyHostToDevice, c.stream),
       "cudaMemcpyAsync");
    const bool f_dev = is_device_ptr(forces);
    double *dF = forces ? (f_dev ? forces : c.d_forces) : nullptr;
    const bool persist = c.persist;
    c.persist = true;  // heaviest cells first, resident CTAs
    struct Restore {
        Context &c;
        bool v;
        ~Restore() { c.persist = v; }
    } restore{c, persist};
    for (int attempt = 0; attempt < 2; ++attempt) {
        CK(cudaMemsetAsync(c.d_err, 0, sizeof(unsigned), c.stream), "cudaMemsetAsync");
        if ((rc = batch_enqueue(c, L, c.d_sinfo, c.d_order, dpos, dtypes, dF, nullptr, nullptr))) break;
        rc = read_error_word(c);
        if (rc != AENET_E_CAPACITY || attempt == 1) break;
        c.caps.nb *= 2;
        c.caps.ang *= 2;
        c.caps.tile = 1024;
        destroy_graph(c);
    }
    if (rc) return rc;
    c.act_valid = c.keep_act;
    c.act_atoms = n;
    // outputs: per-structure [energy, virial[9]] rows -> caller layout
    std::vector<double> res((size_t)n_struct * 10);
    CK(cudaMemcpyAsync(res.data(), c.d_bres, sizeof(double) * res.size(), cudaMemcpyDeviceToHost, c.stream),
       "result copy");
    if (forces && !f_dev)
        CK(cudaMemcpyAsync(forces, c.d_forces, 3 * sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, c.stream),
           "forces copy");
    CK(cudaStreamSynchronize(c.stream), "cudaStreamSynchronize");
    std::vector<double> E((size_t)n_struct), W((size_t)n_struct * 9);
    for (int s = 0; s < n_struct; ++s) {
        E[s] = res[(size_t)s * 10];
        for (int k = 0; k < 9; ++k) W[(size_t)s * 9 + k] = res[(size_t)s * 10 + 1 + k];
    }
    if (energies) CK(cudaMemcpy(energies, E.data(), sizeof(double) * E.size(), cudaMemcpyDefault), "energies");
    if (virials) CK(cudaMemcpy(virials, W.data(), sizeof(double) * W.size(), cudaMemcpyDefault), "virials");
    return AENET_OK;
}

// ------------------------------------------------------------ prepared batch
namespace aenet {
namespace {

// Capture the prepared batch's evaluation into c.batch_exec.
int batch_capture(Context &c, const BatchLayout &L) {
    if (c.batch_exec) cudaGraphExecDestroy(c.batch_exec);
    c.batch_exec = nullptr;
    const bool persist = c.persist;
    c.persist = c.plan.persist;
    c.persist_ctas = c.plan.ctas;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    int rc = batch_enqueue(c, L, c.d_psinfo, c.d_porder, c.plan.pos, c.plan.types, c.plan.forces, c.plan.energies,
                           c.plan.virials);
    cudaError_t ce = cudaStreamEndCapture(c.stream, &graph);
    c.persist = persist;
    c.persist_ctas = 0;
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (ce != cudaSuccess) return cuda_fail(&c, ce, "end capture");
    size_t n_nodes = 0;
    c.plan.kernels = 0;
    if (cudaGraphGetNodes(graph, nullptr, &n_nodes) == cudaSuccess && n_nodes > 0) {
        std::vector<cudaGraphNode_t> nodes(n_nodes);
        if (cudaGraphGetNodes(graph, nodes.data(), &n_nodes) == cudaSuccess)
            for (size_t k = 0; k < n_nodes; ++k) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nodes[k], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
                    ++c.plan.kernels;
            }
    }
    ce = cudaGraphInstantiate(&c.batch_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
        c.batch_exec = nullptr;
        return cuda_fail(&c, ce, "graph instantiate");
    }
    c.plan.gen = c.buf_gen;
    c.plan.stream = c.stream;
    c.plan.caps = c.caps;
    return AENET_OK;
}

}  // namespace
}  // namespace aenet

extern "C" int aenet_batch_prepare(aenet_ctx *h, int n_struct, const int64_t *atom_offset, const double *boxes,
                                   const double *pos, const int32_t *types, double *energies, double *forces,
                                   double *virials, int flags) {
    if (!h) return fail(nullptr, AENET_E_ARG, "ctx is NULL");
    Context &c = h->c;
    cudaGetLastError();
    c.plan.valid = false;
    if (c.batch_exec) cudaGraphExecDestroy(c.batch_exec);
    c.batch_exec = nullptr;
    BatchLayout L;
    int rc = batch_layout(c, n_struct, atom_offset, boxes, L);
    if (rc) return rc;
    const int n = L.n;
    if (n > 0 && (!is_device_ptr(pos) || !is_device_ptr(types)))
        return fail(&c, AENET_E_ARG, "a prepared batch needs device pos and types");
    if ((forces && !is_device_ptr(forces)) || (energies && !is_device_ptr(energies)) ||
        (virials && !is_device_ptr(virials)))
        return fail(&c, AENET_E_ARG, "a prepared batch needs device output buffers");
    if ((rc = batch_buffers(c, L))) return rc;
    // the plan's own layout buffers
    if (c.d_psinfo) cudaFree(c.d_psinfo);
    if (c.d_porder) cudaFree(c.d_porder);
    c.d_psinfo = nullptr;
    c.d_porder = nullptr;
    CK(cudaMalloc(&c.d_psinfo, sizeof(StructInfo) * (size_t)n_struct), "cudaMalloc");
    CK(cudaMalloc(&c.d_porder, sizeof(int) * std::max<size_t>(1, L.order.size())), "cudaMalloc");
    CK(cudaMemcpyAsync(c.d_psinfo, L.info.data(), sizeof(StructInfo) * n_struct, cudaMemcpyHostToDevice, c.stream),
       "cudaMemcpyAsync");
    CK(cudaMemcpyAsync(c.d_porder, L.order.data(), sizeof(int) * L.order.size(), cudaMemcpyHostToDevice, c.stream),
       "cudaMemcpyAsync");
    CK(cudaStreamSynchronize(c.stream), "cudaStreamSynchronize");
    c.plan.n_struct = n_struct;
    c.plan.n_atoms = n;
    c.plan.total_cells = L.gall.ncell;
    c.plan.gall = L.gall;
    c.plan.pos = pos;
    c.plan.types = types;
    c.plan.energies = energies;
    c.plan.forces = forces;
    c.plan.virials = virials;

    // Candidate launches: one CTA per cell in index order, or persistent CTAs
    // taking cells heaviest first; staging tiles of 256 ... 2048 image-atoms.
    struct Cand {
        bool persist;
        int tile;
        float ms;
    };
    std::vector<Cand> cands;
    const bool tune = (flags & AENET_BATCH_AUTOTUNE) != 0;
    if (tune) {
        for (int p = 0; p < 2; ++p)
            for (int tile : {256, 512, 1024, 2048}) cands.push_back({p == 1, tile, 0.f});
    } else {
        cands.push_back({true, c.caps.tile, 0.f});
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0), "cudaEventCreate");
    CK(cudaEventCreate(&e1), "cudaEventCreate");
    struct Ev {
        cudaEvent_t a, b;
        ~Ev() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } ev_guard{e0, e1};
    const bool persist0 = c.persist;
    int best = -1;
    for (size_t k = 0; k < cands.size(); ++k) {
        Cand &cd = cands[k];
        c.caps.tile = cd.tile;
        c.persist = cd.persist;
        if (check_smem(c, L.gall)) {  // does not fit: skip
            cd.ms = -1.f;
            continue;
        }
        for (int attempt = 0; attempt < 2; ++attempt) {  // warm-up run; regrow the lists once on overflow
            CK(cudaMemsetAsync(c.d_err, 0, sizeof(unsigned), c.stream), "cudaMemsetAsync");
            if ((rc = batch_enqueue(c, L, c.d_psinfo, c.d_porder, pos, types, forces, energies, virials))) break;
            rc = read_error_word(c);
            if (rc != AENET_E_CAPACITY || attempt == 1) break;
            c.caps.nb *= 2;
            c.caps.ang *= 2;
        }
        if (rc) {
            c.persist = persist0;
            return rc;
        }
        const int reps = tune ? 3 : 1;
        CK(cudaEventRecord(e0, c.stream), "cudaEventRecord");
        for (int r = 0; r < reps && !rc; ++r)
            rc = batch_enqueue(c, L, c.d_psinfo, c.d_porder, pos, types, forces, energies, virials);
        CK(cudaEventRecord(e1, c.stream), "cudaEventRecord");
        CK(cudaEventSynchronize(e1), "cudaEventSynchronize");
        if (rc) {
            c.persist = persist0;
            return rc;
        }
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
        cd.ms = ms / reps;
        if (best < 0 || cd.ms < cands[best].ms) best = (int)k;
    }
    c.persist = persist0;
    if (best < 0) return fail(&c, AENET_E_CAPACITY, "no staging tile fits in shared memory");
    if ((rc = read_error_word(c))) return rc;
    c.plan.persist = cands[best].persist;
    c.plan.tile = cands[best].tile;
    c.plan.ctas = 0;
    c.plan.ms = cands[best].ms;
    c.caps.tile = c.plan.tile;
    if ((rc = batch_capture(c, L))) return rc;
    c.plan.ctas = c.plan.persist ? c.last_grid : L.gall.ncell;
    c.plan.valid = true;
    c.plan_layout = L.info;
    c.plan_order = L.order;
    return AENET_OK;
}

extern "C" int aenet_batch_run(aenet_ctx *h) {
    if (!h) return fail(nullptr, AENET_E_ARG, "ctx is NULL");
    Context &c = h->c;
    cudaGetLastError();
    if (!c.plan.valid || !c.batch_exec) return fail(&c, AENET_E_STATE, "no prepared batch");
    if (c.plan.gen != c.buf_gen || c.plan.stream != c.stream || c.plan.caps.nb != c.caps.nb ||
        c.plan.caps.ang != c.caps.ang) {
        // work buffers, stream or list capacities changed since the capture
        BatchLayout L;
        L.info = c.plan_layout;
        L.order = c.plan_order;
        L.gall = c.plan.gall;
        L.n = c.plan.n_atoms;
        int rc = batch_buffers(c, L);
        if (rc) return rc;
        const int tile = c.caps.tile;
        c.caps.tile = c.plan.tile;
        rc = batch_capture(c, L);
        c.caps.tile = tile;
        if (rc) return rc;
    }
    CK(cudaGraphLaunch(c.batch_exec, c.stream), "graph launch");
    c.maps_n = c.plan.n_atoms;  // the replay rewrote the cell maps
    c.vl_valid = false;
    return AENET_OK;
}

extern "C" int aenet_batch_tuning(aenet_ctx *h, int *persistent, int *tile, int *ctas, int *kernels, float *ms) {
    if (!h) return fail(nullptr, AENET_E_ARG, "ctx is NULL");
    Context &c = h->c;
    if (!c.plan.valid) return fail(&c, AENET_E_STATE, "no prepared batch");
    if (persistent) *persistent = c.plan.persist ? 1 : 0;
    if (tile) *tile = c.plan.tile;
    if (ctas) *ctas = c.plan.ctas;
    if (kernels) *kernels = c.plan.kernels;
    if (ms) *ms = c.plan.ms;
    return AENET_OK;
}

extern "C" int aenet_descriptors(aenet_ctx *h, int n, const double *pos, const int32_t *types, const double *box,
                                 float *G) {
    if (!h) return fail(nullptr, AENET_E_ARG, "ctx is NULL");
    if (!G) return fail(&h->c, AENET_E_ARG, "G is NULL");
    return compute_impl(h->c, n, pos, types, box, nullptr, nullptr, nullptr, nullptr, G);
}

// Whether an MD step without a skin builds the exact neighbour list in every
// step (AENET_OPT_MD_LIST): the FP32 fused form only, not the pipelined form;
// automatic: every basis but the spherical-harmonic one (radial / angular
// coefficient counts 21 / 7), whose fused kernel is the faster there.
static bool md_list_form(const Context &c) {
    if (c.skin > 0.0 || !fused_supported(c) || c.pipeline || c.md_list == AENET_MD_LIST_OFF) return false;
    if (c.md_list == AENET_MD_LIST_ON) return true;
    return !(c.basis.Kr == 21 && c.basis.Ka == 7);
}

// One MD step on device buffers: kick + drift + binning, cell sort (and, in the
// list form, the neighbour-list build), forces at the new positions, closing
// kick with the FP64 reductions (and the record of (E_pot, E_kin) when rec !=
// NULL). With timing, events bracket the 6 stages.
static int enqueue_md_step(Context &c, const Grid &g, int n, double dt, double *pos, double *vel,
                           const int32_t *types, double *rec, bool list_form) {
    int rc = check_smem(c, g);
    if (rc) return rc;
    CK(mark(c, 0), "event");
    CK(launch_md_kick_drift_bin(c, g, n, dt, pos, vel, types), "kick + drift + binning + scan");
    CK(mark(c, 1), "event");
    CK(launch_scatter(c, n), "cell sort");
    // list form: every image-atom within rc_max of each atom, from this step's
    // cells, into the atom's list row (the list kernel of the Verlet path)
    if (list_form) CK(launch_vl_build(c, g, n), "neighbour list");
    CK(mark(c, 2), "event");
    if (list_form) {
        CK(mark(c, 3), "event");
        CK(mark(c, 4), "event");
        c.md_prezeroed = true;  // the kick + drift kernel cleared the forces and statistics
        const cudaError_t pe = launch_potential_list(c, g, n);
        c.md_prezeroed = false;
        CK(pe, "potential kernel (neighbour list)");
        CK(mark(c, 5), "event");
    } else {
        int n_eparts = 0;
        c.md_prezeroed = true;
        rc = enqueue_potential(c, g, n, &n_eparts);
        c.md_prezeroed = false;
        if (rc) return rc;
    }
    CK(launch_md_kick_finish(c, n, dt, vel, types, rec, rec ? rec + c.cap_rec : nullptr), "kick + reductions");
    CK(mark(c, 6), "event");
    return AENET_OK;
}

// One MD step with the Verlet list, enqueued while c.stream is being captured:
// kick + drift (refreshing the FP32 coordinates, setting the rebuild
// conditional), a conditional node whose body rebuilds the list (binning, cell
// sort, list build; captured on the auxiliary stream), the potential over the
// list, and the closing kick with the reductions. Events bracket the stages.
static int enqueue_md_step_verlet(Context &c, const Grid &g, int n, double dt, double *pos, double *vel,
                                  const int32_t *types, double *rec) {
    int rc = check_smem(c, g);
    if (rc) return rc;
    cudaStreamCaptureStatus status;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamGetCaptureInfo(c.stream, &status, nullptr, &graph, nullptr, nullptr, nullptr), "capture info");
    if (status != cudaStreamCaptureStatusActive || !graph) return fail(&c, AENET_E_STATE, "stream is not capturing");
    cudaGraphConditionalHandle cond;
    CK(cudaGraphConditionalHandleCreate(&cond, graph, 0, cudaGraphCondAssignDefault), "conditional handle");
    CK(mark(c, 0), "event");
    CK(launch_md_vl_kick_drift(c, n, dt, pos, vel, types, cond), "kick + drift");
    CK(mark(c, 1), "event");
    // the conditional node after everything captured so far
    const cudaGraphNode_t *deps = nullptr;
    size_t n_deps = 0;
    CK(cudaStreamGetCaptureInfo(c.stream, &status, nullptr, &graph, &deps, nullptr, &n_deps), "capture info");
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    CK(cudaGraphAddNode(&cnode, graph, deps, nullptr, n_deps, &cp), "conditional node");
    CK(cudaStreamUpdateCaptureDependencies(c.stream, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies),
       "capture dependencies");
    // its body: the rebuild, captured on the auxiliary stream
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(c.aux_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
       "body capture");
    cudaStream_t main_stream = c.stream;
    c.stream = c.aux_stream;
    cudaError_t be = launch_md_vl_bin(c, g, n, pos, types);
    if (be == cudaSuccess) be = launch_sort(c, g, n);
    if (be == cudaSuccess) be = launch_vl_build(c, g, n);
    c.stream = main_stream;
    cudaGraph_t body_out = nullptr;
    cudaError_t ee = cudaStreamEndCapture(c.aux_stream, &body_out);
    if (be != cudaSuccess) return cuda_fail(&c, be, "list rebuild");
    if (ee != cudaSuccess) return cuda_fail(&c, ee, "body capture");
    CK(mark(c, 2), "event");
    CK(mark(c, 3), "event");
    CK(mark(c, 4), "event");
    c.md_prezeroed = true;  // the kick + drift kernel cleared the forces and statistics
    const cudaError_t pe = launch_potential_list(c, g, n);
    c.md_prezeroed = false;
    CK(pe, "potential kernel (Verlet list)");
    CK(mark(c, 5), "event");
    CK(launch_md_kick_finish(c, n, dt, vel, types, rec, rec ? rec + c.cap_rec : nullptr, true),
       "kick + reductions");
    CK(mark(c, 6), "event");
    return AENET_OK;
}

// Buffers and list shape of the Verlet path for n atoms on grid g.
static int ensure_verlet(Context &c, int n, const Grid &g) {
    if (!c.aux_stream) CK(cudaStreamCreateWithFlags(&c.aux_stream, cudaStreamNonBlocking), "cudaStreamCreate");
    int code_bits = 0;
    while ((1 << code_bits) < g.n_off) ++code_bits;
    const int jbits = 31 - code_bits;
    if (jbits < 1 || n >= (1 << jbits) || n >= (1 << 28))
        return fail(&c, AENET_E_CAPACITY, "Verlet list: %d atoms x %d image offsets do not fit a 31-bit entry", n,
                    g.n_off);
    const double V = g.box[0] * g.box[1] * g.box[2];
    const double rl = c.caps.rc_list;
    const int need_cap =
        std::max(64, (((int)(1.3 * (n / V) * 4.18879020478639 * rl * rl * rl + 32.0)) + 15) / 16 * 16);
    if (c.caps.vl_cap < need_cap) c.caps.vl_cap = need_cap;
    c.caps.vl_jbits = jbits;
    const size_t N = (size_t)std::max(n, 1);
    if (n > c.cap_vl_atoms || !c.d_vl || (size_t)c.caps.vl_cap * N > (size_t)c.cap_vl_entries) {
        CK(grow(c.d_vl, 0, N * c.caps.vl_cap), "cudaMalloc");
        CK(grow(c.d_vl_count, 0, N), "cudaMalloc");
        CK(grow(c.d_vl_origin, 0, 3 * N), "cudaMalloc");
        CK(grow(c.d_vl_ref, 0, 3 * N), "cudaMalloc");
        c.cap_vl_atoms = n;
        c.cap_vl_entries = (long long)N * c.caps.vl_cap;
        c.vl_valid = false;
        ++c.buf_gen;
    }
    if (!c.d_vl_flag) {
        const size_t P = (size_t)potential_list_max_ctas(c);
        CK(grow(c.d_vl_flag, 0, 2), "cudaMalloc");
        CK(grow(c.d_vl_builds, 0, 1), "cudaMalloc");
        CK(grow(c.d_vl_epart, 0, P + 1), "cudaMalloc");
        CK(grow(c.d_vl_vpart, 0, 9 * P + 9), "cudaMalloc");
        CK(cudaMemsetAsync(c.d_vl_flag, 0, 2 * sizeof(unsigned), c.stream), "cudaMemsetAsync");
        CK(cudaMemsetAsync(c.d_vl_builds, 0, sizeof(unsigned long long), c.stream), "cudaMemsetAsync");
        ++c.buf_gen;
    }
    return AENET_OK;
}

// n_steps MD steps in one fixed cell (edges box, tilts c.tilt).
static int md_fixed_cell(aenet_ctx *h, int n, double *pos, double *vel, const int32_t *types, const double *box,
                         double dt, int n_steps, double *e_pot, double *e_kin, int flags) {
    Context &c = h->c;
    cudaGetLastError();
    if (c.mass.empty()) return fail(&c, AENET_E_ARG, "model has no masses");
    if (n <= 0 || !pos || !vel || !types || !box) return fail(&c, AENET_E_ARG, "bad MD arguments");
    if (n_steps < 0 || !isfinite(dt)) return fail(&c, AENET_E_ARG, "bad n_steps / dt");
    const bool async = (flags & AENET_MD_ASYNC) != 0;
    const bool keep_act = c.keep_act;  // MD steps keep no activation records
    c.keep_act = false;
    c.act_valid = false;
    struct Restore {
        Context &c;
        bool v;
        ~Restore() { c.keep_act = v; }
    } restore{c, keep_act};
    // continuing needs the cell maps and forces of an evaluation of these n atoms
    const bool cont = (flags & AENET_MD_CONTINUE) != 0 && c.maps_n == n;
    // stage events: all 7 (AENET_MD_TIMING), or only those around the potential
    // (AENET_MD_TIMING_POTENTIAL; around each split kernel outside the fused form)
    const unsigned ev_mask = (flags & AENET_MD_TIMING) ? 0x7Fu
                             : (flags & AENET_MD_TIMING_POTENTIAL) ? (fused_path(c) ? 0x30u : 0x3Cu)
                                                                   : 0u;
    const bool timing = ev_mask != 0;
    const bool verlet = c.skin > 0.0 && fused_supported(c);
    const bool list_form = !verlet && md_list_form(c);
    const bool pos_dev = is_device_ptr(pos), vel_dev = is_device_ptr(vel), typ_dev = is_device_ptr(types);
    const bool rec_dev = (!e_pot || is_device_ptr(e_pot)) && (!e_kin || is_device_ptr(e_kin));
    if (async && !(pos_dev && vel_dev && typ_dev && rec_dev))
        return fail(&c, AENET_E_ARG, "AENET_MD_ASYNC needs device pointers");
    Grid g;
    // with a Verlet list the cells must cover the list cutoff rc_max + skin
    int rc = make_grid(c, box, g, verlet ? c.basis.rc_max + c.skin : 0.0, c.tilt);
    if (rc) return rc;
    if ((rc = validate_types_host(c, n, types))) return rc;
    if ((rc = ensure(c, n, g)) || (rc = ensure_stage(c, n))) return rc;
    if (c.caps.nb == 0) c.caps = estimate_caps(c, n, g);
    if (verlet || list_form) {
        // the list form keeps a relative margin of 1e-5 over rc_max: its list is then a
        // superset of the pairs within rc_max, which the list kernel selects exactly
        c.caps.rc_list = (float)(verlet ? c.basis.rc_max + c.skin : c.basis.rc_max * 1.00001);
        if ((rc = ensure_verlet(c, n, g))) return rc;
    }
    double *dpos = pos_dev ? pos : c.d_pos;
    double *dvel = vel_dev ? vel : c.d_vel;
    const int32_t *dtypes = typ_dev ? types : c.d_types;
    if (!pos_dev) CK(cudaMemcpyAsync(dpos, pos, 3 * sizeof(double) * n, cudaMemcpyHostToDevice, c.stream), "pos in");
    if (!vel_dev) CK(cudaMemcpyAsync(dvel, vel, 3 * sizeof(double) * n, cudaMemcpyHostToDevice, c.stream), "vel in");
    if (!typ_dev)
        CK(cudaMemcpyAsync(c.d_types, types, sizeof(int32_t) * n, cudaMemcpyHostToDevice, c.stream), "types in");
    const bool want_rec = e_pot || e_kin;
    if (want_rec && n_steps + 1 > c.cap_rec) {
        if (c.d_rec) cudaFree(c.d_rec);
        c.d_rec = nullptr;
        c.cap_rec = 0;
        CK(cudaMalloc(&c.d_rec, sizeof(double) * 2 * (size_t)(n_steps + 1)), "cudaMalloc");
        c.cap_rec = n_steps + 1;
        ++c.buf_gen;
        destroy_graph(c);
    }
    double *rec = want_rec ? c.d_rec : nullptr;
    if (!async) CK(cudaMemsetAsync(c.d_err, 0, sizeof(unsigned), c.stream), "cudaMemsetAsync");
    if (want_rec) CK(cudaMemsetAsync(c.d_step, 0, sizeof(int), c.stream), "cudaMemsetAsync");
    // frame 0: forces at the initial positions (unless continuing); a
    // neighbour-list overflow here regrows the capacities once before capture
    if (!cont) {
        for (int attempt = 0; attempt < 2; ++attempt) {
            if ((rc = enqueue_compute(c, g, n, dpos, dtypes, nullptr, nullptr))) return rc;
            if (async) break;
            rc = read_error_word(c);
            if (rc != AENET_E_CAPACITY || attempt == 1) break;
            c.caps.nb *= 2;
            c.caps.ang *= 2;
            c.caps.tile = 1024;
            destroy_graph(c);
        }
        if (rc) return rc;
    }
    // thermostat: the coupling factor of each step comes from the closing
    // reductions of the step before (frame 0: the kick with dt = 0 below)
    c.thermo_dt = dt;
    const bool thermo = c.thermo_tau > 0.0;
    if (thermo && !c.d_lambda) {
        CK(cudaMalloc(&c.d_lambda, sizeof(double)), "cudaMalloc");
        ++c.buf_gen;
    }
    if (want_rec || (thermo && (!cont || !c.lambda_valid)))  // kinetic energy and record of frame 0
        CK(launch_md_kick_finish(c, n, 0.0, dvel, dtypes, rec, rec ? rec + c.cap_rec : nullptr), "frame 0");
    if (n_steps > 0) {
        const bool same = c.md_exec && c.md_key.n == n && c.md_key.pos == dpos && c.md_key.vel == dvel &&
                          c.md_key.types == dtypes && c.md_key.box[0] == box[0] && c.md_key.box[1] == box[1] &&
                          c.md_key.box[2] == box[2] && c.md_key.dt == dt && c.md_key.rec == rec &&
                          c.md_key.stream == c.stream && c.md_key.caps.nb == c.caps.nb &&
                          c.md_key.caps.ang == c.caps.ang && c.md_key.caps.tile == c.caps.tile &&
                          c.md_key.ev_mask == ev_mask && c.md_key.gen == c.buf_gen && c.md_key.skin == c.skin &&
                          c.md_key.list_form == list_form && c.md_key.caps.vl_cap == c.caps.vl_cap &&
                          c.md_key.thermo_T0 == c.thermo_T0 &&
                          c.md_key.thermo_tau == c.thermo_tau;
        if (!same) {
            destroy_graph(c);
            cudaGraph_t graph = nullptr;
            CK(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            c.ev_mask = ev_mask;
            int src = verlet ? enqueue_md_step_verlet(c, g, n, dt, dpos, dvel, dtypes, rec)
                             : enqueue_md_step(c, g, n, dt, dpos, dvel, dtypes, rec, list_form);
            c.ev_mask = 0u;
            cudaError_t ce = cudaStreamEndCapture(c.stream, &graph);
            if (src) {
                if (graph) cudaGraphDestroy(graph);
                return src;
            }
            if (ce != cudaSuccess) return cuda_fail(&c, ce, "end capture");
            size_t n_nodes = 0;
            c.md_kernels = 0;
            if (cudaGraphGetNodes(graph, nullptr, &n_nodes) == cudaSuccess && n_nodes > 0) {
                std::vector<cudaGraphNode_t> nodes(n_nodes);
                if (cudaGraphGetNodes(graph, nodes.data(), &n_nodes) == cudaSuccess) {
                    for (size_t k = 0; k < n_nodes; ++k) {
                        cudaGraphNodeType t;
                        if (cudaGraphNodeGetType(nodes[k], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
                            ++c.md_kernels;
                    }
                }
            }
            ce = cudaGraphInstantiate(&c.md_exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) {
                c.md_exec = nullptr;
                return cuda_fail(&c, ce, "graph instantiate");
            }
            c.md_key.n = n;
            c.md_key.pos = dpos;
            c.md_key.vel = dvel;
            c.md_key.types = dtypes;
            for (int a = 0; a < 3; ++a) c.md_key.box[a] = box[a];
            c.md_key.dt = dt;
            c.md_key.rec = rec;
            c.md_key.stream = c.stream;
            c.md_key.caps = c.caps;
            c.md_key.timing = timing;
            c.md_key.ev_mask = ev_mask;
            c.md_key.gen = c.buf_gen;
            c.md_key.skin = c.skin;
            c.md_key.list_form = list_form;
            c.last_list = list_form;
            c.md_key.thermo_T0 = c.thermo_T0;
            c.md_key.thermo_tau = c.thermo_tau;
        }
        // the first step after any other evaluation (or a new list shape) builds the list
        if (verlet && (!cont || !c.vl_valid))
            CK(cudaMemsetAsync(c.d_vl_flag, 0xff, sizeof(unsigned), c.stream), "cudaMemsetAsync");
        for (int s = 0; s < n_steps; ++s) CK(cudaGraphLaunch(c.md_exec, c.stream), "graph launch");
        c.maps_n = n;
        c.vl_valid = verlet;
        c.lambda_valid = thermo;
    }
    if (want_rec) {
        if (e_pot) CK(cudaMemcpyAsync(e_pot, rec, sizeof(double) * (n_steps + 1), cudaMemcpyDefault, c.stream), "e_pot");
        if (e_kin)
            CK(cudaMemcpyAsync(e_kin, rec + c.cap_rec, sizeof(double) * (n_steps + 1), cudaMemcpyDefault, c.stream),
               "e_kin");
    }
    if (!pos_dev) CK(cudaMemcpyAsync(pos, dpos, 3 * sizeof(double) * n, cudaMemcpyDeviceToHost, c.stream), "pos out");
    if (!vel_dev) CK(cudaMemcpyAsync(vel, dvel, 3 * sizeof(double) * n, cudaMemcpyDeviceToHost, c.stream), "vel out");
    if (async) return AENET_OK;
    return read_error_word(c);
}

// Berendsen coupling after a step: the pressure of the frame the step ended on
// (energy, virial and kinetic energy of its closing reduction, d_result),
//     P = (2 E_kin + tr W) / (3 V),  V = L_x L_y L_z,
// then positions, edges and tilts scaled by
//     mu = (1 - (every dt / tau) (P0 - P) / B)^(1/3).
// The cell maps, forces and list of the old cell are invalidated, so the next
// steps start from a fresh evaluation in the scaled cell.
static int barostat_couple(Context &c, int n, double *pos, double *L, double dt) {
    constexpr double kEvPerA3InBar = 1.602176634e6;
    double res[11];
    CK(cudaMemcpyAsync(res, c.d_result, sizeof(res), cudaMemcpyDeviceToHost, c.stream), "pressure copy");
    CK(cudaStreamSynchronize(c.stream), "cudaStreamSynchronize");
    const double V = L[0] * L[1] * L[2];
    const double P = (2.0 * res[10] + res[1] + res[5] + res[9]) / (3.0 * V) * kEvPerA3InBar;
    const double arg = 1.0 - (c.baro_every * dt / c.baro_tau) * (c.baro_P0 - P) / c.baro_modulus;
    if (!(arg > 0.0) || !isfinite(arg))
        return fail(&c, AENET_E_ARG, "barostat: volume factor %g <= 0 (pressure %g bar; lower dt * every / tau)", arg, P);
    const double mu = cbrt(arg);
    const bool pos_dev = is_device_ptr(pos);
    double *dpos = pos_dev ? pos : c.d_pos;  // the device copy holds the final positions either way
    CK(launch_scale(c, dpos, 3LL * n, mu), "scale positions");
    if (!pos_dev) {
        CK(cudaMemcpyAsync(pos, dpos, 3 * sizeof(double) * n, cudaMemcpyDeviceToHost, c.stream), "pos out");
        CK(cudaStreamSynchronize(c.stream), "cudaStreamSynchronize");
    }
    for (int a = 0; a < 3; ++a) {
        L[a] *= mu;
        c.tilt[a] *= mu;
    }
    c.vl_valid = false;
    c.maps_n = -1;
    destroy_graph(c);
    return AENET_OK;
}

extern "C" int aenet_md_nve(aenet_ctx *h, int n, double *pos, double *vel, const int32_t *types,
                            const double *box, double dt, int n_steps, double *e_pot, double *e_kin, int flags) {
    if (!h) return fail(nullptr, AENET_E_ARG, "ctx is NULL");
    Context &c = h->c;
    if (!box) return fail(&c, AENET_E_ARG, "bad MD arguments");
    double L[3] = {box[0], box[1], box[2]};
    int rc = AENET_OK;
    if (c.baro_every <= 0) {
        rc = md_fixed_cell(h, n, pos, vel, types, L, dt, n_steps, e_pot, e_kin, flags);
    } else {
        // runs of baro_every steps between couplings; the records of a coupling
        // step hold the scaled state (its frame is evaluated again)
        if (flags & AENET_MD_ASYNC)
            return fail(&c, AENET_E_ARG, "the barostat reads the pressure at every coupling: no AENET_MD_ASYNC");
        int s0 = 0;
        do {
            const int k = std::min(c.baro_every, n_steps - s0);
            rc = md_fixed_cell(h, n, pos, vel, types, L, dt, k, e_pot ? e_pot + s0 : nullptr,
                               e_kin ? e_kin + s0 : nullptr, s0 == 0 ? flags : (flags & ~AENET_MD_CONTINUE));
            if (rc) break;
            s0 += k;
            if (k == c.baro_every) {
                if ((rc = barostat_couple(c, n, pos, L, dt))) break;
                if (s0 == n_steps)  // the scaled last frame: its forces, energy and records
                    rc = md_fixed_cell(h, n, pos, vel, types, L, dt, 0, e_pot ? e_pot + s0 : nullptr,
                                       e_kin ? e_kin + s0 : nullptr, flags & ~AENET_MD_CONTINUE);
                if (rc) break;
            }
        } while (s0 < n_steps);
    }
    if (rc == AENET_OK) {
        for (int a = 0; a < 3; ++a) c.md_box[a] = L[a];
        c.md_box_valid = true;
    }
    return rc;
}

extern "C" int aenet_set_barostat(aenet_ctx *h, double P0, double tau, double modulus, int every) {
    if (!h) return fail(nullptr, AENET_E_ARG, "ctx is NULL");
    Context &c = h->c;
    if (!isfinite(P0) || !isfinite(tau) || !isfinite(modulus))
        return fail(&c, AENET_E_ARG, "barostat parameters must be finite");
    if (tau <= 0.0) {
        c.baro_every = 0;
        return AENET_OK;
    }
    if (!(modulus > 0.0) || every < 1) return fail(&c, AENET_E_ARG, "barostat: modulus > 0 and every >= 1 required");
    c.baro_P0 = P0;
    c.baro_tau = tau;
    c.baro_modulus = modulus;
    c.baro_every = every;
    return AENET_OK;
}

extern "C" int aenet_md_box(aenet_ctx *h, double *box, double *tilt) {
    if (!h || !box) return fail(h ? &h->c : nullptr, AENET_E_ARG, "NULL argument");
    Context &c = h->c;
    if (!c.md_box_valid) return fail(&c, AENET_E_STATE, "no MD call has run on this context");
    for (int a = 0; a < 3; ++a) {
        box[a] = c.md_box[a];
        if (tilt) tilt[a] = c.tilt[a];
    }
    return AENET_OK;
}

extern "C" int aenet_neighbor_stats(aenet_ctx *h, int64_t *out) {
    if (!h || !out) return fail(h ? &h->c : nullptr, AENET_E_ARG, "NULL argument");
    Context &c = h->c;
    unsigned long long st[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(st, c.d_stats, sizeof(st), cudaMemcpyDeviceToHost, c.stream), "stats copy");
    CK(cudaStreamSynchronize(c.stream), "cudaStreamSynchronize");
    for (int k = 0; k < 3; ++k) out[k] = (int64_t)st[k];
    return AENET_OK;
}

extern "C" int aenet_md_stage_times(aenet_ctx *h, float *ms, int *kernels_per_step, int *path_flags) {
    if (!h || !ms) return fail(h ? &h->c : nullptr, AENET_E_ARG, "NULL argument");
    Context &c = h->c;
    if (!c.md_exec || !c.md_key.timing) return fail(&c, AENET_E_STATE, "no MD step was run with AENET_MD_TIMING");
    CK(cudaStreamSynchronize(c.stream), "cudaStreamSynchronize");
    for (int k = 0; k < Context::kStages; ++k) {
        const unsigned both = (1u << k) | (1u << (k + 1));
        if ((c.md_key.ev_mask & both) == both)
            CK(cudaEventElapsedTime(&ms[k], c.ev[k], c.ev[k + 1]), "elapsed");
        else
            ms[k] = nanf("");  // stage not recorded in the light timing mode
    }
    if (kernels_per_step) *kernels_per_step = c.md_kernels;
    if (path_flags)
        *path_flags = (fused_path(c) ? AENET_PATH_FUSED : 0) | (c.last_pipe ? AENET_PATH_PIPELINED : 0) |
                      (c.last_list ? AENET_PATH_LIST : 0);
    return AENET_OK;
}

extern "C" int aenet_set_option(aenet_ctx *h, int option, int value) {
    if (!h) return fail(nullptr, AENET_E_ARG, "ctx is NULL");
    Context &c = h->c;
    if (option == AENET_OPT_KEEP_ACTIVATIONS) {
        c.keep_act = value != 0;
        c.act_valid = false;
        return AENET_OK;
    }
    if (option == AENET_OPT_FUSED_NETWORK) {
        if (c.fuse_network != (value != 0)) {
            c.fuse_network = value != 0;
            destroy_graph(c);  // the captured MD step holds the other path's kernels
        }
        return AENET_OK;
    }
    if (option == AENET_OPT_PIPELINE) {
        if (c.pipeline != (value != 0)) {
            c.pipeline = value != 0;
            destroy_graph(c);
        }
        return AENET_OK;
    }
    if (option == AENET_OPT_MD_LIST) {
        if (value != AENET_MD_LIST_AUTO && value != AENET_MD_LIST_OFF && value != AENET_MD_LIST_ON)
            return fail(&c, AENET_E_ARG, "AENET_OPT_MD_LIST takes AENET_MD_LIST_AUTO, _OFF or _ON, not %d", value);
        if (c.md_list != value) {
            c.md_list = value;
            destroy_graph(c);
        }
        return AENET_OK;
    }
    return fail(&c, AENET_E_ARG, "unknown option %d", option);
}

extern "C" int aenet_grad_weights(aenet_ctx *h, double *dEdW) {
    if (!h || !dEdW) return fail(h ? &h->c : nullptr, AENET_E_ARG, "NULL argument");
    Context &c = h->c;
    cudaGetLastError();
    if (!c.act_valid)
        return fail(&c, AENET_E_STATE, "no activation records: set AENET_OPT_KEEP_ACTIVATIONS and evaluate first");
    if (c.net.n_params > grad_max_params())
        return fail(&c, AENET_E_ARG, "network has more than %d parameters per species", grad_max_params());
    CK(launch_grad_weights(c, c.act_atoms), "weight gradient");
    CK(cudaMemcpyAsync(dEdW, c.d_dEdW, sizeof(double) * c.basis.n_species * c.net.n_params, cudaMemcpyDefault,
                       c.stream),
       "dE/dW copy");
    if (!is_device_ptr(dEdW)) CK(cudaStreamSynchronize(c.stream), "cudaStreamSynchronize");
    return AENET_OK;
}

namespace aenet {
namespace {
// FP64 parameters (device) to the context's FP32 copy.
__global__ void k_params_to_f32(size_t n, const double *__restrict__ src, float *__restrict__ dst) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        dst[k] = (float)src[k];
}
}  // namespace
}  // namespace aenet

extern "C" int aenet_set_params(aenet_ctx *h, const double *params) {
    if (!h || !params) return fail(h ? &h->c : nullptr, AENET_E_ARG, "NULL argument");
    Context &c = h->c;
    cudaGetLastError();
    const size_t NP = (size_t)c.basis.n_species * c.net.n_params;
    if (is_device_ptr(params)) {
        // on the context's stream, after the work already enqueued: no host round trip
        k_params_to_f32<<<(int)std::min<size_t>((NP + 255) / 256, 1024), 256, 0, c.stream>>>(NP, params, c.d_params);
        CK(cudaGetLastError(), "parameter conversion");
    } else {
        std::vector<float> P(NP);
        for (size_t k = 0; k < NP; ++k) P[k] = (float)params[k];
        CK(cudaStreamSynchronize(c.stream), "cudaStreamSynchronize");
        CK(cudaMemcpy(c.d_params, P.data(), sizeof(float) * NP, cudaMemcpyHostToDevice), "cudaMemcpy");
    }
    if (c.precision != AENET_FP32) CK(prepare_bf16_weights(c), "BF16 weights");
    c.act_valid = false;
    return AENET_OK;
}

extern "C" int aenet_check(aenet_ctx *h) {
    if (!h) return fail(nullptr, AENET_E_ARG, "ctx is NULL");
    return read_error_word(h->c);
}

extern "C" const char *aenet_last_error(const aenet_ctx *h) {
    if (!h) return g_setup_error.c_str();
    return h->c.err.c_str();
}

extern "C" void aenet_destroy(aenet_ctx *h) {
    if (!h) return;
    Context &c = h->c;
    destroy_graph(c);
    if (c.batch_exec) cudaGraphExecDestroy(c.batch_exec);
    c.batch_exec = nullptr;
    if (c.stream) cudaStreamSynchronize(c.stream);
    void *ptrs[] = {c.d_params, c.d_shift, c.d_scale, c.d_wbf, c.d_wtc, c.d_mass, c.d_pos4, c.d_tmp4, c.d_perm,
                    c.d_cell_of, c.d_slot, c.d_cell_count, c.d_cell_start, c.d_G, c.d_dEdG, c.d_eatom, c.d_F4,
                    c.d_vir_part, c.d_e_part, c.d_ke_part, c.d_result, c.d_err, c.d_step, c.d_done, c.d_pos, c.d_vel,
                    c.d_forces, c.d_eatom_out, c.d_types, c.d_rec, c.d_stats, c.d_sp_cnt, c.d_sp_off,
                    c.d_sp_rank, c.d_sp_list, c.d_sinfo, c.d_bres, c.d_act,
                    c.d_wpart, c.d_wpairs, c.d_dEdW, c.d_work, c.d_order, c.d_psinfo, c.d_porder,
                    c.d_vl, c.d_vl_count, c.d_vl_origin, c.d_vl_ref, c.d_vl_flag, c.d_vl_builds,
                    c.d_vl_epart, c.d_vl_vpart, c.d_lambda};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (int k = 0; k <= Context::kStages; ++k)
        if (c.ev[k]) cudaEventDestroy(c.ev[k]);
    if (c.own_stream && c.stream) cudaStreamDestroy(c.stream);
    if (c.aux_stream) cudaStreamDestroy(c.aux_stream);
    delete h;
}

extern "C" int aenet_set_thermostat(aenet_ctx *h, double T0, double tau) {
    if (!h) return fail(nullptr, AENET_E_ARG, "ctx is NULL");
    Context &c = h->c;
    if (!isfinite(T0) || !isfinite(tau) || T0 < 0.0) return fail(&c, AENET_E_ARG, "T0 must be >= 0, tau finite");
    if (tau <= 0.0) T0 = tau = 0.0;
    if (T0 != c.thermo_T0 || tau != c.thermo_tau) {
        c.thermo_T0 = T0;
        c.thermo_tau = tau;
        c.lambda_valid = false;
        destroy_graph(c);
    }
    return AENET_OK;
}

extern "C" int aenet_set_skin(aenet_ctx *h, double skin) {
    if (!h) return fail(nullptr, AENET_E_ARG, "ctx is NULL");
    Context &c = h->c;
    if (!(skin >= 0.0) || !isfinite(skin)) return fail(&c, AENET_E_ARG, "skin must be finite and >= 0");
    if (skin != c.skin) {
        c.skin = skin;
        c.vl_valid = false;
        c.caps.vl_cap = 0;
        destroy_graph(c);
    }
    return AENET_OK;
}

extern "C" int aenet_set_box_tilt(aenet_ctx *h, double xy, double xz, double yz) {
    if (!h) return fail(nullptr, AENET_E_ARG, "ctx is NULL");
    Context &c = h->c;
    if (!isfinite(xy) || !isfinite(xz) || !isfinite(yz)) return fail(&c, AENET_E_ARG, "tilt factors must be finite");
    if (xy != c.tilt[0] || xz != c.tilt[1] || yz != c.tilt[2]) {
        c.tilt[0] = xy;
        c.tilt[1] = xz;
        c.tilt[2] = yz;
        c.vl_valid = false;
        c.maps_n = -1;  // forces and cell maps of the old cell: the next MD call starts from frame 0
        destroy_graph(c);
    }
    return AENET_OK;
}

extern "C" int aenet_md_list_builds(aenet_ctx *h, int64_t *builds) {
    if (!h || !builds) return fail(h ? &h->c : nullptr, AENET_E_ARG, "NULL argument");
    Context &c = h->c;
    unsigned long long v = 0;
    if (c.d_vl_builds) {
        CK(cudaMemcpyAsync(&v, c.d_vl_builds, sizeof(v), cudaMemcpyDeviceToHost, c.stream), "cudaMemcpyAsync");
        CK(cudaStreamSynchronize(c.stream), "cudaStreamSynchronize");
    }
    *builds = (int64_t)v;
    return AENET_OK;
}
