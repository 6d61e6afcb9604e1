// Internal declarations of the GB300 ANN-potential library: device model
// constants, the cell grid, the context, and the launch wrappers of every
// kernel. Only the .cu files of this library include it.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>
#include <vector_types.h>

#include "aenet_gpu.h"

namespace aenet {

constexpr int kMaxSpecies = 8;
constexpr int kMaxD = 64;       // descriptor length handled by the 64-slot warp reduction
constexpr int kMaxWidth = 64;   // hidden-layer width limit
constexpr int kMaxLayers = 5;   // weight layers
constexpr int kMaxOrder = 31;

// Device error word bits (set by kernels, read by the host after a sync).
constexpr unsigned kErrNbCap = 1u;      // neighbour list overflow
constexpr unsigned kErrAngCap = 2u;     // angular list overflow
constexpr unsigned kErrOverlap = 4u;    // |d| < 1e-6 A
constexpr unsigned kErrNonfinite = 8u;  // non-finite coordinate
constexpr unsigned kErrType = 16u;      // species index out of range
constexpr unsigned kErrTimeout = 32u;   // a bounded in-kernel wait ran out

// Descriptor basis and species constants, passed by value to the kernels.
struct Basis {
    int n_species;
    int Kr, Ka, D;          // Kr = order_rad + 1, Ka = order_ang + 1, D = 2 (Kr + Ka)
    float rc_rad, rc_ang, rc_max;
    float type_weight[kMaxSpecies];
    float sh_b[7][7];       // Legendre coefficients of T_a (a, l <= 6): the angular form through spherical harmonics
};

// Network shape (per species identical), passed by value.
struct Net {
    int n_species;
    int n_layers;                  // weight layers
    int widths[kMaxLayers + 1];
    int n_params;                  // floats per species: W^1 b^1 W^2 b^2 ...
    int act_len;                   // sum of widths (activation storage per atom)
};

// Cell grid of one orthorhombic box: nc cells per axis of edge h >= rc_max (or
// a single cell when the box is shorter than the cutoff); neighbour cells are
// scanned over offsets -m..m per axis, each offset one periodic image.
// Cell grid of one periodic box. The box is the restricted triclinic cell of
// LAMMPS, lattice vectors a = (L_x, 0, 0), b = (xy, L_y, 0), c = (xz, yz, L_z)
// (orthorhombic when the tilts are zero): nc[k] cells along lattice vector k,
// so a cell's edge vectors are A = a / nc[0], B = b / nc[1], C = c / nc[2], and
// image-cell offset (ox, oy, oz) is the shift ox A + oy B + oz C.
struct Grid {
    int nc[3];
    int m[3];
    int ncell;
    int n_off;                     // prod(2 m + 1)
    double box[3];                 // L_x, L_y, L_z
    double h[3];                   // diagonal of A, B, C: L_k / nc[k]
    double inv_box[3];             // reciprocals: no FP64 division on the device
    double inv_h[3];
    float hf[3];
    int tri;                       // any tilt != 0
    double tilt[3];                // xy, xz, yz
    double ht[3];                  // off-diagonal of the cell edges: B_x = xy / nc[1], C_x = xz / nc[2], C_y = yz / nc[2]
    float htf[3];
};

// Wrap one position into [0, box) and bin it: returns the cell and the FP32
// coordinates relative to the cell origin (computed in FP64, then rounded).
// FP64 work is a short chain of multiplies and FMAs (no division): FP64 has a
// long latency on this part.
__device__ inline int bin_position(double x0, double x1, double x2, const Grid &g, float *u, bool &finite,
                                   double *ud = nullptr) {
    if (g.tri) {
        // tilted cell: fractional coordinates by back substitution (x = H s, H
        // upper triangular), each wrapped into [0, 1) and binned; the position
        // relative to the cell's centre (c0 + 1/2) A + (c1 + 1/2) B + (c2 + 1/2) C
        // in Cartesian (the centre, not a corner: an oblique cell's long
        // diagonal would double the FP32 coordinates' magnitude and rounding)
        double x[3] = {x0, x1, x2};
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (!isfinite(x[a])) {
                finite = false;
                x[a] = 0.0;
            }
        double s[3];
        s[2] = x[2] * g.inv_box[2];
        s[1] = fma(-g.tilt[2], s[2], x[1]) * g.inv_box[1];
        s[0] = fma(-g.tilt[1], s[2], fma(-g.tilt[0], s[1], x[0])) * g.inv_box[0];
        int ci[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double w = s[a] - floor(s[a]);
            if (w >= 1.0) w -= 1.0;
            if (w < 0.0) w = 0.0;
            s[a] = w;
            int c = (int)(w * g.nc[a]);
            ci[a] = c >= g.nc[a] ? g.nc[a] - 1 : c;
        }
        const double xw[3] = {fma(g.tilt[1], s[2], fma(g.tilt[0], s[1], g.box[0] * s[0])),
                              fma(g.tilt[2], s[2], g.box[1] * s[1]), g.box[2] * s[2]};
        const double k0 = ci[0] + 0.5, k1 = ci[1] + 0.5, k2 = ci[2] + 0.5;
        const double ua[3] = {xw[0] - fma(k2, g.ht[1], fma(k1, g.ht[0], k0 * g.h[0])),
                              xw[1] - fma(k2, g.ht[2], k1 * g.h[1]), xw[2] - k2 * g.h[2]};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            u[a] = (float)ua[a];
            if (ud) ud[a] = ua[a];
        }
        return (ci[2] * g.nc[1] + ci[1]) * g.nc[0] + ci[0];
    }
    const double xs[3] = {x0, x1, x2};
    int ci[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double x = xs[a];
        if (!isfinite(x)) {
            finite = false;
            x = 0.0;
        }
        const double L = g.box[a];
        double w = fma(-floor(x * g.inv_box[a]), L, x);
        if (w >= L) w -= L;
        if (w < 0.0) w = 0.0;
        int c = (int)(w * g.inv_h[a]);
        c = c >= g.nc[a] ? g.nc[a] - 1 : c;
        ci[a] = c;
        const double ua = fma(-(double)c, g.h[a], w);
        u[a] = (float)ua;
        if (ud) ud[a] = ua;  // FP64 cell-relative coordinate (the Verlet list keeps its origin)
    }
    return (ci[2] * g.nc[1] + ci[1]) * g.nc[0] + ci[0];
}

// One structure of a batch: its own cell grid inside a global cell index space
// (cells cell0 .. cell0 + ncell - 1) and its atoms (atom0 .. atom0 + natoms - 1
// in input order).
struct StructInfo {
    Grid g;
    int cell0, ncell, atom0, natoms;
};

// Capacities of the per-warp neighbour lists of the potential kernel, and the
// shape of the Verlet list (MD with a skin).
struct Caps {
    int nb;     // entries with r <= rc_max
    int ang;    // entries with r <= rc_ang
    int tile;   // staged neighbour-cell atoms per chunk (fused kernel)
    int vl_cap = 0;        // Verlet-list entries per atom (r <= rc_max + skin at the build)
    int vl_jbits = 0;      // bits of the sorted atom index in an entry; the rest: image-offset code
    float rc_list = 0.f;   // rc_max + skin
};

struct Context {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int precision = AENET_FP32;
    bool fuse_network = true;      // BF16 forms: tensor-core network inside the fused kernel
    bool pipeline = false;         // FP32 fused form: the pipelined kernel (one CTA of 16 warps per SM)
    Basis basis{};
    Net net{};
    std::vector<double> mass;      // [n_species], empty if none
    std::string err;

    // model on the device
    float *d_params = nullptr;     // [n_species * n_params] FP32
    float *d_shift = nullptr;      // [n_species * D]
    float *d_scale = nullptr;      // [n_species * D]
    uint16_t *d_wbf = nullptr;     // BF16 warp-MMA operand fragments (hi, lo) and biases, see ann_bf16.cu
    unsigned char *d_wtc = nullptr;  // tcgen05 B operands and biases per species, see ann_tcgen05.cu
    size_t wbf_elems = 0;
    double *d_mass = nullptr;      // [n_species]

    // work buffers (grown on demand)
    int cap_atoms = 0;
    int cap_cells = 0;
    int cap_blocks = 0;
    float4 *d_pos4 = nullptr;      // sorted cell-local coordinates, .w = species (int bits)
    float4 *d_tmp4 = nullptr;      // same, input order
    int *d_perm = nullptr;         // sorted slot -> input index
    int *d_cell_of = nullptr;      // input index -> cell
    int *d_slot = nullptr;         // input index -> rank inside its cell
    int *d_cell_count = nullptr;   // [ncell]
    int *d_cell_start = nullptr;   // [ncell + 1]
    float *d_G = nullptr;          // [n * D] sorted order
    float *d_dEdG = nullptr;       // [n * D] sorted order
    float *d_eatom = nullptr;      // [n] sorted order
    float4 *d_F4 = nullptr;        // [n] force accumulators, sorted order
    double *d_vir_part = nullptr;  // [cells * 9]
    double *d_e_part = nullptr;    // [blocks]
    double *d_ke_part = nullptr;   // [MD CTAs * 11] per-CTA energy, virial and kinetic-energy sums
    double *d_result = nullptr;    // [10]: energy, virial[9]
    unsigned *d_err = nullptr;     // device error word
    unsigned long long *d_stats = nullptr;  // [4] radial entries, angular entries, angular pairs
    int *d_step = nullptr;         // MD record counter
    unsigned *d_done = nullptr;    // last-CTA counter of the MD reduction (left at 0)

    // per-atom activation records for dE/dW (optional)
    bool keep_act = false;
    bool act_valid = false;        // records of the last evaluation are in d_act
    int act_atoms = 0;             // atoms of that evaluation
    int cap_act = 0;
    float *d_act = nullptr;        // [n * rec_len] sorted order
    float *d_wpart = nullptr;      // dE/dW partial sums per (species, chunk)
    size_t cap_wpart = 0;
    int2 *d_wpairs = nullptr;      // [n_params] record indices of each weight's factors
    double *d_dEdW = nullptr;      // [n_species * n_params]

    // species grouping of the BF16 network kernel
    int *d_sp_cnt = nullptr;       // [kMaxSpecies], kept at 0 between evaluations
    int *d_sp_off = nullptr;       // [kMaxSpecies]
    int *d_sp_rank = nullptr;      // [n]
    int *d_sp_list = nullptr;      // [n] sorted indices grouped by species

    // staging of host arrays
    int cap_stage = 0;
    double *d_pos = nullptr, *d_vel = nullptr, *d_forces = nullptr, *d_eatom_out = nullptr;
    int32_t *d_types = nullptr;
    int cap_rec = 0;
    double *d_rec = nullptr;       // [2 * cap_rec] e_pot, e_kin records

    Caps caps{};

    // batched evaluation: per-structure grids (device), valid during a batch call
    int cap_struct = 0;
    StructInfo *d_sinfo = nullptr;     // [n_struct]
    double *d_bres = nullptr;          // [n_struct * 10]: energy, virial[9]
    const StructInfo *batch_sinfo = nullptr;  // non-NULL while a batch is enqueued
    int batch_n = 0;

    // Verlet neighbour list with a skin (MD steps of the fused FP32 form; skin 0 =
    // the cell list every step). Entries: sorted index | image-offset code << jbits,
    // built by k_potential's list mode, rebuilt inside the captured step (a graph
    // conditional node) whenever an atom moved more than skin/2 since the build.
    double skin = 0.0;
    // MD steps without a skin: AENET_MD_LIST_AUTO (0), _OFF (1: the fused kernel searches the cells
    // itself) or _ON (2: the exact list is built in every step and the list kernel evaluates it)
    int md_list = 0;
    bool last_list = false;            // the captured MD step builds the exact list in every step
    // tilt factors xy, xz, yz of the restricted triclinic cell of single-structure
    // calls (zero: orthorhombic)
    double tilt[3] = {0.0, 0.0, 0.0};
    int cap_vl_atoms = 0;
    long long cap_vl_entries = 0;
    int *d_vl = nullptr;               // [atoms * vl_cap] sorted order
    int *d_vl_count = nullptr;         // [atoms]
    double *d_vl_origin = nullptr;     // [atoms * 3] origin of atom i's FP32 coordinates (input order)
    double *d_vl_ref = nullptr;        // [atoms * 3] positions at the last build (input order)
    unsigned *d_vl_flag = nullptr;     // [2]: rebuild flag, last-CTA counter
    unsigned long long *d_vl_builds = nullptr;  // list builds so far
    double *d_vl_epart = nullptr;      // [4 * SMs] energy partials of the list-mode kernel
    double *d_vl_vpart = nullptr;      // [4 * SMs * 9] virial partials
    bool vl_valid = false;             // list, origins and cell maps describe the MD state
    cudaStream_t aux_stream = nullptr; // captures the body of the rebuild conditional
    int maps_n = -1;                   // atoms of the evaluation that last wrote the cell maps
    // partials of the last potential evaluation (read by the MD reductions)
    const double *last_epart = nullptr, *last_vpart = nullptr;
    int last_eparts = 0, last_vparts = 0;

    // Berendsen thermostat of the MD path (tau <= 0: NVE). d_lambda holds the
    // velocity scale of the next step, written by the closing kick.
    double thermo_T0 = 0.0, thermo_tau = 0.0, thermo_dt = 0.0;
    double *d_lambda = nullptr;
    bool lambda_valid = false;         // d_lambda was computed with the current settings

    // Berendsen barostat of the MD path (baro_every 0: off): after every
    // baro_every-th step of a call, positions and cell scaled by
    // mu = (1 - (baro_every dt / baro_tau) (baro_P0 - P) / baro_modulus)^(1/3).
    double baro_P0 = 0.0, baro_tau = 0.0, baro_modulus = 0.0;  // bar, ps, bar
    int baro_every = 0;
    double md_box[3] = {0.0, 0.0, 0.0};  // edges of the cell after the last MD call
    bool md_box_valid = false;

    // Generation of the work buffers: bumped whenever one is reallocated, so a
    // captured graph (which holds their addresses) knows it must be re-captured.
    unsigned buf_gen = 0;

    // persistent form of the potential kernel (used by the batched evaluation)
    int n_sm = 0;                      // SMs of the device
    bool persist = false;              // CTAs take cells from a global counter (batches only)
    int persist_ctas = 0;              // CTAs of the persistent launch (0 = all resident)
    unsigned *d_work = nullptr;        // [2] item counter, exit counter (each launch leaves both 0)
    const int *batch_order = nullptr;  // cell order of the batch being enqueued, heaviest first
    int *d_order = nullptr;            // [cap_order] that order for aenet_compute_batch
    int cap_order = 0;
    int last_grid = 0;                 // CTAs of the last potential launch
    bool last_pipe = false;            // the last fused FP32 launch was the pipelined form
    // set while an MD step is enqueued: its kick + drift kernel has already cleared the force
    // accumulators and the neighbour statistics, so the potential launch needs no memset
    bool md_prezeroed = false;
    int pot_parts = 0;                 // energy / virial partial rows of the last potential launch

    // prepared batch (aenet_batch_prepare): its own layout buffers, the tuned
    // launch and the captured evaluation
    cudaGraphExec_t batch_exec = nullptr;
    StructInfo *d_psinfo = nullptr;    // [n_struct]
    int *d_porder = nullptr;           // [total_cells]
    struct {
        bool valid = false;
        int n_struct = 0, n_atoms = 0, total_cells = 0;
        Grid gall{};
        const double *pos = nullptr;
        const int32_t *types = nullptr;
        double *energies = nullptr, *forces = nullptr, *virials = nullptr;
        bool persist = false;
        int tile = 0, ctas = 0, kernels = 0;
        float ms = 0.f;
        Caps caps{};
        unsigned gen = 0;
        cudaStream_t stream = nullptr;
    } plan;
    std::vector<StructInfo> plan_layout;  // host copy of the prepared layout
    std::vector<int> plan_order;

    // captured MD step
    cudaGraphExec_t md_exec = nullptr;
    struct {
        int n = -1;
        double *pos = nullptr, *vel = nullptr;
        const int32_t *types = nullptr;
        double box[3] = {0, 0, 0};
        double dt = 0;
        double *rec = nullptr;
        cudaStream_t stream = nullptr;
        Caps caps{};
        bool timing = false;
        unsigned gen = 0;
        double skin = 0.0;
        bool list_form = false;
        unsigned ev_mask = 0;
        double thermo_T0 = 0.0, thermo_tau = 0.0;
    } md_key;
    unsigned ev_mask = 0;              // stage events recorded while an MD step is captured

    // stage timing of the captured MD step (events recorded inside the graph)
    static constexpr int kStages = 6;  // kick+drift+bin, sort, descriptor, network, forces, kick+reductions
    cudaEvent_t ev[kStages + 1] = {};
    int md_kernels = 0;                // kernel nodes in the captured step
};

// Allow a kernel the device's largest dynamic shared memory. Launches of one
// kernel with different sizes (captured graphs among them) then never depend on
// which size was set last; each launcher still checks its own size.
template <class K>
inline cudaError_t allow_max_smem(K kern) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);  // static shared memory counts against the limit
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
    return e;
}

// ---------------------------------------------------------------- launchers
// All launchers enqueue on ctx.stream and return the launch status.

// Wrap, bin and sort atoms by cell (the periodic cell list).
cudaError_t launch_cells(Context &c, const Grid &g, int n, const double *pos, const int32_t *types);
// The scan + scatter half of launch_cells (after the counts are in place).
cudaError_t launch_scan(Context &c, const Grid &g);  // cell counts -> cell starts (k_scan_cells)
cudaError_t launch_scatter(Context &c, int n);  // the sort after a binning kernel that also scanned
cudaError_t launch_sort(Context &c, const Grid &g, int n);
// Binning of a batch: every atom into the cell grid of its structure.
cudaError_t launch_cells_batch(Context &c, int n, int total_cells, const double *pos, const int32_t *types);
// Per-structure energy (FP64 sum of E_i) and virial (FP64 sum of cell partials)
// into c.d_bres rows, or (when given) straight into energies[S], virials[S*9].
cudaError_t launch_batch_reduce(Context &c, double *energies = nullptr, double *virials = nullptr);

// Descriptor of every atom into c.d_G (Sec. II.B; k_potential, descriptor mode).
cudaError_t launch_fp_forward(Context &c, const Grid &g, int n);

// Per-species networks: E_i and dE/dG_i (Sec. II.A, Eq. ANN-layer), energy block partials.
cudaError_t launch_ann(Context &c, int n);

// Forces and virial partials from c.d_dEdG (the chain rule; k_potential, forces mode).
cudaError_t launch_fp_backward(Context &c, const Grid &g, int n);

// Energy and virial reductions (E = sum_i E_i, Sec. II.A) over n_eparts energy partials and the
// cells' virial partials, and outputs in input order.
cudaError_t launch_finalize(Context &c, const Grid &g, int n, int n_eparts, double *forces, double *e_atom);

// BF16 tensor-core networks (precision forms; two hidden layers <= 32).
bool bf16_supported(const Net &net);
// The three-kernel path's network kernel: tcgen05 (TMEM accumulators) over
// 128-atom species tiles. Energy partials: one per CTA.
int tcgen05_tiles(const Context &c, int n);
int tcgen05_eparts(const Context &c, int n);
cudaError_t launch_ann_tcgen05(Context &c, int n);
// Its weights, packed into the B-operand layout (c.d_wtc) from c.d_params.
cudaError_t pack_tcgen05_weights(Context &c);

// Length of the per-atom activation record (g, then x_l and delta_l per hidden layer).
int activation_record_len(const Net &net);
// Group the sorted atoms by species (d_sp_list, d_sp_off).
cudaError_t launch_species_group(Context &c, int n);
// dE/dW and dE/db of every species from the activation records (FP64 result in d_dEdW).
cudaError_t launch_grad_weights(Context &c, int n);
std::vector<int2> grad_pairs(const Net &net);
int grad_max_params();

// Work items per cell of a single-structure potential launch (persistent CTAs
// take cell parts from a counter); partial buffers hold kMaxSplit rows per cell.
constexpr int kMaxSplit = 4;
int potential_split(const Context &c, const Grid &g, int *split_from, int wave = 0);
bool pipe_supported(const Context &c, const Grid &g);

// Fused descriptor + network + forces kernel (FP32 form, hidden widths <= 32).
bool fused_supported(const Context &c);
cudaError_t launch_fused_potential(Context &c, const Grid &g, int n);
// Fused kernel with the networks on the tensor cores (BF16 forms; two hidden
// layers <= 32 wide; the water (16, 8) and solid (20, 6) bases), unless the
// context asked for the three-kernel path (AENET_OPT_FUSED_NETWORK 0).
bool tc_fused_supported(const Context &c);
cudaError_t launch_fused_tc(Context &c, const Grid &g, int n);
// Either fused form: descriptor, networks and forces in one kernel.
inline bool fused_path(const Context &c) { return fused_supported(c) || tc_fused_supported(c); }
int ann_blocks(int n);

// Forces to input order (FP64) only.
cudaError_t launch_finalize_forces(Context &c, int n, double *forces);

// Descriptor rows to input order (float).
cudaError_t launch_unsort_G(Context &c, int n, float *G);

// Velocity Verlet (the propagation step of the MD cycle, Fig. 1).
// One MD half: kick (v += dt/2 F/m c) + drift (x += dt v) fused with the binning
// of the new positions (integration and cell list); the scan and scatter follow.
cudaError_t launch_md_kick_drift_bin(Context &c, const Grid &g, int n, double dt, double *pos, double *vel,
                                     const int32_t *types);
// The closing kick (v += dt/2 F/m c) with the kinetic energy, fused with the
// FP64 reduction of energy, virial and kinetic energy (last-CTA pattern) into
// c.d_result and, when rec_pot != NULL, the record of step *c.d_step. The
// partials are those of the last potential evaluation (c.last_*). With
// clear_vl, the last CTA also counts a list build and clears the rebuild flag.
cudaError_t launch_md_kick_finish(Context &c, int n, double dt, double *vel, const int32_t *types,
                                  double *rec_pot, double *rec_kin, bool clear_vl = false);
// x *= mu for count doubles (the barostat's isotropic scaling of positions).
cudaError_t launch_scale(Context &c, double *x, long long count, double mu);

// Verlet form of the opening half-kick and drift (no binning): refresh the FP32
// coordinates relative to the origins of the last list build, raise the rebuild
// flag if an atom moved more than skin/2, and set the graph conditional.
cudaError_t launch_md_vl_kick_drift(Context &c, int n, double dt, double *pos, double *vel, const int32_t *types,
                                    cudaGraphConditionalHandle cond);
// Rebuild, part 1: bin the current positions, record each atom's origin and
// reference position (then launch_sort and launch_vl_build).
cudaError_t launch_md_vl_bin(Context &c, const Grid &g, int n, const double *pos, const int32_t *types);
// Rebuild, part 2: the Verlet list of every atom (k_potential, list-build mode).
cudaError_t launch_vl_build(Context &c, const Grid &g, int n);
// The fused potential over the Verlet list (persistent CTAs, atoms from a
// counter); sets c.last_* to its partials.
cudaError_t launch_potential_list(Context &c, const Grid &g, int n);
// Largest CTA count of launch_potential_list (sizes its partial buffers).
int potential_list_max_ctas(const Context &c);

// Message reported by aenet_last_error(NULL) for calls made without a context.
void set_context_free_error(const char *msg);

// Dynamic shared memory bytes of the potential kernel in the context's mode.
size_t potential_smem_bytes(const Context &c, const Grid &g);
size_t ann_smem_bytes(const Context &c);

}  // namespace aenet
