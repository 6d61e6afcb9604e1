/*
 * aenet_gpu.h -- C ABI of the GB300 (sm_103a) ANN-potential hot path.
 *
 * The library evaluates an atomic-energy-network potential of the
 * Behler-Parrinello form E = sum_i ANN_{t_i}(g_i) (Sec. II.A, Eq. ANN-layer and
 * the atomic-energy sum) on the Chebyshev descriptor of Sec. II.B (Eq. radial,
 * Eq. angular, Eq. cos-cutoff and the species-weighted copy), plus the forces
 * and virial that the MD engines of Sec. III consume and a velocity-Verlet NVE
 * propagator (the MD cycle of Fig. 1). One context drives one GPU on one stream.
 *
 * Units: eV, Angstrom, amu, ps (LAMMPS "metal", Sec. III).
 *
 * Pointers: every array argument marked "host or device" may point to host
 * memory or to device memory of the context's GPU; the library inspects it with
 * cudaPointerGetAttributes and stages host data through its own device buffers.
 * The caller owns all arrays it passes; the library copies what it keeps.
 *
 * Errors: every int-returning call returns an aenet_status. Nothing aborts or
 * traps: device-side problems (neighbour-list overflow, coincident atoms,
 * non-finite coordinates) are recorded in a device error word and reported by
 * the next call that synchronises. aenet_last_error() gives a message.
 *
 * Thread safety: a context is not thread-safe; use one context per host thread
 * and stream.
 */
#ifndef AENET_GPU_H
#define AENET_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct aenet_ctx aenet_ctx;

typedef enum {
    AENET_OK = 0,
    AENET_E_ARG = -1,       /* invalid argument (sizes, NULL, types out of range, box) */
    AENET_E_CUDA = -2,      /* a CUDA runtime call failed */
    AENET_E_CAPACITY = -3,  /* a neighbour list exceeded its capacity even after one regrow */
    AENET_E_NONFINITE = -4, /* non-finite coordinate */
    AENET_E_OVERLAP = -5,   /* two image-atoms closer than 1e-6 A */
    AENET_E_TIMEOUT = -6,   /* a bounded device wait gave up */
    AENET_E_NOMEM = -7,     /* device allocation failed */
    AENET_E_STATE = -8      /* call out of order (e.g. gradient before compute) */
} aenet_status;

typedef enum {
    AENET_FP32 = 0,         /* network layers in FP32 on the CUDA cores */
    AENET_BF16 = 1,         /* network layers as BF16 tensor-core products, FP32 accumulate */
    AENET_BF16X3 = 2        /* split-BF16 (hi*hi + hi*lo + lo*hi) tensor-core products */
} aenet_precision;

/*
 * Model description (copied at setup; the caller may free it afterwards).
 *
 * Descriptor (Sec. II.B): for atom i with neighbours j (all periodic images
 * within the cutoff, excluding only the zero-shift self)
 *   radial  c_a = sum_j T_a(2 r_ij / rc_rad - 1) f_c(r_ij),      a = 0..order_rad
 *   angular c_a = sum_{j != k} T_a(cos theta_ijk) f_c(r_ij) f_c(r_ik), a = 0..order_ang
 *             (ordered pairs of distinct image-atoms, f_c with rc_ang)
 * and the same two sums with every neighbour term weighted by type_weight[t_j]
 * (angular: type_weight[t_j] * type_weight[t_k]). G = [radial, angular,
 * radial_w, angular_w], D = 2 (order_rad + 1 + order_ang + 1) <= 64.
 * The network input is g = (G - in_shift[t]) * in_scale[t].
 *
 * Network (Eq. ANN-layer): widths[0] = D, widths[n_layers] = 1, hidden widths
 * <= 64; tanh on hidden layers, linear output. params holds, per species, the
 * concatenation W^1 b^1 W^2 b^2 ... with W^l row-major [widths[l] x widths[l-1]].
 */
typedef struct {
    int n_species;               /* >= 1, <= 8 */
    const double *type_weight;   /* [n_species] s_t of the weighted copy */
    const double *mass;          /* [n_species] amu; NULL if no MD is run */
    double rc_rad;               /* radial cutoff (A) */
    int order_rad;               /* radial Chebyshev order N_r (0..31) */
    double rc_ang;               /* angular cutoff (A) */
    int order_ang;               /* angular Chebyshev order N_a (0..31) */
    int n_layers;                /* weight layers, 2..5 (at least one hidden layer) */
    const int *widths;           /* [n_layers + 1] */
    const double *params;        /* [n_species * n_params] */
    const double *in_shift;      /* [n_species * D] or NULL (zeros) */
    const double *in_scale;      /* [n_species * D] or NULL (ones) */
} aenet_model_desc;

/*
 * Create a context on the current CUDA device. `stream` is a cudaStream_t
 * (NULL: the context creates a blocking stream of its own, which the legacy
 * default stream orders implicitly); all work of the context is ordered on it.
 * precision: an aenet_precision. Returns AENET_OK and *out, or an error and
 * *out = NULL.
 */
int aenet_setup(aenet_ctx **out, const aenet_model_desc *model, int precision, void *stream);

/* Change the stream of a context (the captured MD graph is rebuilt lazily). */
int aenet_set_stream(aenet_ctx *ctx, void *stream);

/*
 * Energy, forces and virial of one periodic structure (the potential of
 * Sec. II evaluated as the interface of Sec. III returns it), in an
 * orthorhombic box or in the tilted cell of aenet_set_box_tilt.
 *   n_atoms  >= 0
 *   pos      [n_atoms * 3] double, host or device; any real coordinates
 *            (wrapped internally into the cell by their fractional coordinates)
 *   types    [n_atoms] int32, host or device; 0-based species index in setup
 *            order (the species-order rule of the LAMMPS interface)
 *   box      [3] double, HOST; box edge lengths (A), each > 0
 *   energy   [1] double, host or device, or NULL: E = sum_i E_i (FP64 sum)
 *   forces   [n_atoms * 3] double, host or device, or NULL: F = -dE/dr
 *   virial   [9] double, host or device, or NULL: W_ab = -sum_d d_a dE/dd_b
 *            over all displacement vectors d = x_j + (lattice image) - x_i
 *            (row-major)
 *   e_atom   [n_atoms] double, host or device, or NULL: E_i
 * Synchronises the stream before returning.
 */
int aenet_compute(aenet_ctx *ctx, int n_atoms, const double *pos, const int32_t *types,
                  const double *box, double *energy, double *forces, double *virial,
                  double *e_atom);

/*
 * Verlet neighbour list for aenet_md_nve (the LAMMPS-style list with a skin
 * that the paper credits for ænet-LAMMPS's speed over ænet-TINKER, Sec. IV.B).
 * skin (A) >= 0; 0 (the default) bins the atoms into cells and finds their
 * neighbours anew in every step (AENET_OPT_MD_LIST says how). With
 * skin > 0 (FP32 form; the other forms ignore it) each MD step reuses a list
 * of the image-atoms within rc_max + skin of every atom and rebuilds it inside
 * the captured step only when some atom moved more than skin/2 since the last
 * build (a CUDA-graph conditional node set on the device). Energies and forces
 * are those of the cell path. The list costs (rc_max + skin)^3 / rc_max^3 more
 * candidate pairs per step and one 4-byte entry per candidate.
 * Errors: AENET_E_ARG for a negative or non-finite skin.
 */
int aenet_set_skin(aenet_ctx *ctx, double skin);

/*
 * Thermostat for aenet_md_nve (the MD cycle of Fig. 1 takes a temperature;
 * the paper names no thermostat, so this is the Berendsen weak coupling):
 * at the start of every step the velocities are scaled by
 *     lambda = sqrt(1 + (dt / tau) (T0 / T - 1)),  T = 2 E_kin / ((3N - 3) k_B),
 * E_kin being the kinetic energy of the frame the step starts from (the one
 * recorded in e_kin). T0 in K (>= 0), tau in ps; tau <= 0 (the default) turns
 * it off (NVE). The factor is computed on the device by the closing reduction
 * of each step, so steps stay asynchronous. Errors: AENET_E_ARG.
 */
int aenet_set_thermostat(aenet_ctx *ctx, double T0, double tau);

/*
 * Tilted (restricted triclinic) periodic cell for the single-structure calls
 * of this context (aenet_compute, aenet_descriptors, aenet_md_nve): their box
 * [3] = (L_x, L_y, L_z) then gives the lattice vectors
 *     a = (L_x, 0, 0),  b = (xy, L_y, 0),  c = (xz, yz, L_z),
 * the box form of the MD codes the paper's potential is used from (LAMMPS,
 * Sec. IV.B). Positions are wrapped by their fractional coordinates; the cell
 * grid has at least one cutoff between opposite cell faces along each lattice
 * direction. All zero (the default) is the orthorhombic box. Any finite tilt is
 * accepted (a very oblique cell needs a wide image window: more than 4096 image
 * cells per atom is AENET_E_ARG at the next call). Batched calls and
 * aenet_descriptors_noalloc stay orthorhombic. A change invalidates the MD
 * graph and list: the next aenet_md_nve starts from frame 0.
 * Errors: AENET_E_ARG (non-finite tilt).
 */
int aenet_set_box_tilt(aenet_ctx *ctx, double xy, double xz, double yz);

/*
 * Berendsen barostat for aenet_md_nve (the MD cycle of Fig. 1 takes T and p as
 * inputs; the paper names no barostat, so this is the isotropic weak coupling
 * of LAMMPS's press/berendsen): after every `every`-th step of a call, with the
 * pressure of that frame
 *     P = (2 E_kin + tr W) / (3 V),   V = L_x L_y L_z,  W the virial,
 * positions and the cell (edges and the tilts of aenet_set_box_tilt) are
 * scaled by
 *     mu = (1 - (every dt / tau) (P0 - P) / modulus)^(1/3),
 * and that frame is evaluated again: its e_pot / e_kin records are those of the
 * scaled state. P0 and modulus (the bulk modulus) in bar, tau in ps, every >= 1
 * steps; tau <= 0 turns it off (the default). Each coupling synchronises and
 * the next run of steps is captured again (a new cell), so AENET_MD_ASYNC is
 * refused while it is on. The cell after a call: aenet_md_box. A volume factor
 * <= 0 (a coupling too strong for the pressure) stops the call with
 * AENET_E_ARG. Errors: AENET_E_ARG.
 */
int aenet_set_barostat(aenet_ctx *ctx, double P0, double tau, double modulus, int every);

/* The cell the last aenet_md_nve call ended in (a query of the MD state with
 * no counterpart in the paper): box [3] HOST, the edges; tilt [3] HOST or NULL,
 * the tilt factors, which are also the context's tilt for later calls.
 * Errors: AENET_E_ARG (NULL box), AENET_E_STATE (no MD call yet). */
int aenet_md_box(aenet_ctx *ctx, double *box, double *tilt);

/* Number of Verlet-list builds so far on this context (a measurement with no
 * counterpart in the paper): *builds HOST. Synchronises. Errors: AENET_E_ARG. */
int aenet_md_list_builds(aenet_ctx *ctx, int64_t *builds);

/*
 * aenet_compute without synchronisation, for callers that evaluate repeatedly
 * on device data (an autograd force loop): the same evaluation enqueued on the
 * context's stream, every array a DEVICE pointer (energy, forces, virial,
 * e_atom may be NULL), box HOST. Device-side problems (neighbour-list overflow,
 * overlapping atoms, species out of range) are not read here: they stay in the
 * device error word until the next synchronising call, aenet_check for
 * instance, reports them, and the outputs of the failing evaluation are then
 * invalid. The list capacities are not regrown here: after an
 * AENET_E_CAPACITY from aenet_check, one aenet_compute (which regrows and
 * retries) restores them. Host pointers give AENET_E_ARG.
 */
int aenet_compute_async(aenet_ctx *ctx, int n_atoms, const double *pos, const int32_t *types, const double *box,
                        double *energy, double *forces, double *virial, double *e_atom);

/*
 * Energies, forces and virials of many independent periodic structures in one
 * evaluation (one binning, one potential launch over the cells of every
 * structure, one per-structure reduction). Each structure's energy is the
 * Behler-Parrinello sum E_s = sum_{i in s} E_i of Sec. II.A, its forces the
 * chain rule of Sec. II.C, exactly as aenet_compute evaluates one structure.
 *   n_struct     >= 1
 *   atom_offset  [n_struct + 1] int64, HOST: structure s holds atoms
 *                atom_offset[s] .. atom_offset[s+1]-1; atom_offset[0] = 0
 *   pos, types   [N * 3] double, [N] int32 (N = atom_offset[n_struct]), host or device
 *   boxes        [n_struct * 3] double, HOST: orthorhombic box of each structure
 *   energies     [n_struct] double, host or device, or NULL (FP64 sums of E_i)
 *   forces       [N * 3] double, host or device, or NULL
 *   virials      [n_struct * 9] double, host or device, or NULL
 * Synchronises.
 */
int aenet_compute_batch(aenet_ctx *ctx, int n_struct, const int64_t *atom_offset, const double *pos,
                        const int32_t *types, const double *boxes, double *energies, double *forces,
                        double *virials);

/*
 * Prepared batch: the batched evaluation above (the
 * energy of each structure is the Behler-Parrinello sum of Sec. II.A, its
 * forces the chain rule of Sec. II.C) made replayable for repeated
 * evaluation of one batch layout with new coordinates (an MD or screening
 * loop over many structures).
 * aenet_batch_prepare fixes the layout (atom_offset, boxes: HOST, as in
 * aenet_compute_batch) and the DEVICE buffers the evaluation reads (pos
 * [N * 3], types [N]) and writes (energies [n_struct], forces [N * 3],
 * virials [n_struct * 9]; each output may be NULL). It evaluates the batch on
 * the current contents of pos, and with flags & AENET_BATCH_AUTOTUNE times
 * candidate launches of the potential kernel on them: one CTA per cell in
 * cell order, or one resident (persistent) CTA per SM slot taking cells from
 * a global counter heaviest first, each with staging tiles of 256, 512, 1024
 * and 2048 image-atoms. It keeps the fastest and captures the whole evaluation
 * (binning, cell sort, potential, per-structure reductions, forces) in one
 * CUDA graph. Without the flag it uses the persistent form and the current
 * tile. The caller keeps the buffers alive and at the same addresses until
 * the next prepare or aenet_destroy. Synchronises.
 * Errors: AENET_E_ARG for host buffers or a bad layout, AENET_E_CAPACITY if a
 * neighbour list overflows twice, the device error codes of aenet_compute.
 */
#define AENET_BATCH_AUTOTUNE 1
int aenet_batch_prepare(aenet_ctx *ctx, int n_struct, const int64_t *atom_offset, const double *boxes,
                        const double *pos, const int32_t *types, double *energies, double *forces,
                        double *virials, int flags);

/*
 * Replays the prepared evaluation on the context's stream: reads pos/types
 * and writes the outputs given to aenet_batch_prepare. Asynchronous: device
 * errors (e.g. a neighbour list overflowing on new coordinates) are reported
 * by the next aenet_check. If the context's work buffers, stream or list
 * capacities changed since the capture (another call on the same context),
 * the graph is captured again first. AENET_E_STATE without a prepared batch.
 */
int aenet_batch_run(aenet_ctx *ctx);

/*
 * The launch aenet_batch_prepare chose: persistent (1) or one CTA per cell
 * (0), staging tile, CTAs of the potential launch, kernel nodes in the
 * captured graph, and the measured time of one evaluation (ms). Any output
 * may be NULL. AENET_E_STATE without a prepared batch.
 */
int aenet_batch_tuning(aenet_ctx *ctx, int *persistent, int *tile, int *ctas, int *kernels, float *ms);

/*
 * Descriptor only (Sec. II.B): G [n_atoms * D]
 * float32, host or device, row i = atom i in input order, layout [radial,
 * angular, radial_w, angular_w] before standardisation. Other arguments and
 * errors as aenet_compute. Synchronises.
 */
int aenet_descriptors(aenet_ctx *ctx, int n_atoms, const double *pos, const int32_t *types,
                      const double *box, float *G);

/*
 * Velocity-Verlet NVE (the propagation cycle of Fig. 1; integration in FP64):
 *   v += dt/2 F/m c;  x += dt v;  F = F(x);  v += dt/2 F/m c
 * with c = 9648.533212 (A/ps)^2 per eV/amu. Requires model masses.
 *   pos, vel [n_atoms * 3] double, host or device, updated in place
 *   types    [n_atoms] int32, host or device; box [3] HOST
 *   dt_ps    time step (ps); n_steps >= 0
 *   e_pot, e_kin  [n_steps + 1] double, host or device, or NULL: potential and
 *            kinetic energy of frames 0..n_steps
 *   flags    bitwise OR of
 *            AENET_MD_ASYNC: do not synchronise; then pos, vel, types, e_pot
 *            and e_kin must be device pointers (or NULL) and device errors are
 *            reported by the next synchronising call or aenet_check();
 *            AENET_MD_CONTINUE: see below.
 * Every step after the first is one replay of a captured CUDA graph. With the
 * barostat on (aenet_set_barostat) the cell changes during the call: read the
 * final one with aenet_md_box.
 */
#define AENET_MD_ASYNC 1
/* AENET_MD_CONTINUE: pos and vel are exactly as the previous aenet_md_nve call
 * on this context left them (same buffers, nothing else run on the context in
 * between); the forces and energy of that call's last frame are reused instead
 * of being recomputed for frame 0. */
#define AENET_MD_CONTINUE 2
/* AENET_MD_TIMING: record CUDA events between the stages of every captured MD
 * step; read them with aenet_md_stage_times(). Each event adds about 2 us of
 * device time to a step. AENET_MD_TIMING_POTENTIAL records only the events
 * around the potential (the fused kernel, or each split kernel), so that the
 * step is timed nearly as it runs untimed; the other stages then read NaN. */
#define AENET_MD_TIMING 4
#define AENET_MD_TIMING_POTENTIAL 8
int aenet_md_nve(aenet_ctx *ctx, int n_atoms, double *pos, double *vel, const int32_t *types,
                 const double *box, double dt_ps, int n_steps, double *e_pot, double *e_kin,
                 int flags);

/*
 * Neighbour statistics of the last descriptor evaluation on the context,
 * summed over atoms: out[0] = image-atoms within the largest cutoff, out[1] =
 * image-atoms within the angular cutoff, out[2] = unordered angular pairs
 * (j < k) -- the pair and triplet counts that set the cost of Eqs. radial and
 * angular. Synchronises.
 */
int aenet_neighbor_stats(aenet_ctx *ctx, int64_t out[3]);

/*
 * Device time (ms) of each stage of the last MD step run with
 * AENET_MD_TIMING (CUDA events recorded inside the captured graph, on the
 * context's stream): [kick + drift + binning, cell sort, descriptor, network,
 * forces, closing kick + FP64 reductions]; the number of kernel launches in
 * one MD step; and path flags: AENET_PATH_FUSED when descriptor, network and
 * forces run as one fused kernel (the FP32 form with hidden widths <= 32),
 * whose time is then all reported under "forces" (descriptor and network read
 * ~0), and AENET_PATH_PIPELINED when that kernel ran in its pipelined form
 * (AENET_OPT_PIPELINE), and AENET_PATH_LIST when the step built the exact
 * neighbour list in every step (AENET_OPT_MD_LIST; the list build is then
 * reported under "cell sort" and the list-driven potential kernel under
 * "forces"). Any output pointer except ms may be NULL. Returns
 * AENET_E_STATE if no timed step has run. Synchronises.
 */
#define AENET_PATH_FUSED 1
#define AENET_PATH_PIPELINED 2
#define AENET_PATH_LIST 4
int aenet_md_stage_times(aenet_ctx *ctx, float ms[6], int *kernels_per_step, int *path_flags);

/*
 * Descriptor without a context and without any device allocation.
 *
 * The paper has no counterpart: this entry point serves callers that cannot
 * call cudaMalloc when they need descriptors -- a host program whose GPU memory
 * is handed out only by its own fixed pool, code running while another
 * component owns the allocator, or a plugin that must not grow the process's
 * device footprint after start-up. It computes the same G as
 * aenet_descriptors() (same kernels) and allocates nothing: its scratch is one
 * fixed file-scope __device__ array of about 5.0 MB (cell-sorted coordinates,
 * cell table, sorted descriptor rows, error word) that every GPU which loads
 * this library holds until the process exits.
 *   n_atoms      0 .. AENET_NOALLOC_MAX_ATOMS; larger systems return
 *                AENET_E_CAPACITY (as do boxes with more than
 *                AENET_NOALLOC_MAX_CELLS cells of edge >= the largest cutoff)
 *   pos, types   DEVICE pointers of the current device (or managed memory),
 *                [n_atoms * 3] double and [n_atoms] int32; device memory of
 *                another GPU is refused with AENET_E_ARG
 *   box          [3] double, HOST: the edges of an ORTHORHOMBIC box. This entry
 *                point has no context, so a tilt set with aenet_set_box_tilt
 *                never applies to it; tilted cells go through
 *                aenet_descriptors on a context
 *   n_species, type_weight (HOST [n_species]), rc_rad, order_rad, rc_ang,
 *   order_ang    the basis, as in aenet_model_desc
 *   G            DEVICE [n_atoms * D] float32 output of the current device,
 *                input order
 *   stream       cudaStream_t (NULL = legacy default stream)
 * The first call on a device looks up the device address of the scratch
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture. Every call shares the one scratch array, so
 * calls whose GPU work overlaps (other host threads, other streams) race and
 * must be serialised by the caller. Synchronises `stream`. Messages are read
 * with aenet_last_error(NULL).
 */
#define AENET_NOALLOC_MAX_ATOMS 16384
#define AENET_NOALLOC_MAX_CELLS 16384
int aenet_descriptors_noalloc(int n_atoms, const double *pos, const int32_t *types, const double *box,
                              int n_species, const double *type_weight, double rc_rad, int order_rad,
                              double rc_ang, int order_ang, float *G, void *stream);

/*
 * Context options. AENET_OPT_KEEP_ACTIVATIONS (value 0/1): when on, every
 * aenet_compute / aenet_compute_batch keeps one activation record per atom
 * (standardised descriptor g, and x_l, delta_l of every hidden layer) so that
 * aenet_grad_weights can follow; costs (D + 2 sum H_l) floats per atom.
 */
#define AENET_OPT_KEEP_ACTIVATIONS 1
/*
 * AENET_OPT_FUSED_NETWORK (value 0/1, default 1), BF16 forms only: with 1 the
 * per-species networks run on the tensor cores inside the fused potential
 * kernel (one geometry pass; the water and solid bases, two hidden layers of
 * at most 32); with 0 they run as the three-kernel path (descriptor kernel,
 * tensor-core network kernel over species-grouped tiles, force kernel). Both
 * compute the same products; the option exists to compare the two.
 */
#define AENET_OPT_FUSED_NETWORK 2
/*
 * AENET_OPT_PIPELINE (value 0/1, default 0), FP32 fused form of a single
 * structure: with 1 the potential kernel runs pipelined (one CTA of 16 warps
 * per SM; warps prepare the next cells' neighbourhoods while others finish the
 * current cell, with no CTA-wide barrier between cells); with 0 the
 * block-synchronous form (two CTAs of 8 warps per SM, one cell at a time).
 * Same arithmetic, so the results agree to FP32 rounding order. The pipelined
 * form removes the barrier waits but runs slower on GB300 (its desynchronised
 * warps miss the instruction cache more often), so it is off by default; the
 * option exists to compare the two. It is used when its shared-memory layout
 * fits and the descriptor basis is one of the kernel's exact forms (orders
 * 17/9 or 21/7); otherwise the block-synchronous form runs.
 */
#define AENET_OPT_PIPELINE 3
/*
 * AENET_OPT_MD_LIST (value AENET_MD_LIST_AUTO, _OFF or _ON; default AUTO), MD
 * steps of the FP32 fused form without a skin (aenet_set_skin 0): the
 * neighbours of Sec. II.B (every image-atom within the largest cutoff, the
 * atom itself at zero shift excluded) are found in every step either by the
 * fused potential kernel itself from the staged cells (OFF) or by a list
 * kernel that writes each atom's exact list after the binning, which the
 * list-driven potential kernel then reads (ON; the Verlet-list machinery with
 * no skin and no rebuild test). The same pairs enter the same arithmetic, so
 * the two agree to FP32 rounding order. AUTO takes ON for every basis except
 * angular order 6 with radial order 20 (its spherical-harmonic angular sum
 * runs faster in the fused kernel). Other evaluations (aenet_compute and the
 * batch calls) always use the fused kernel. A change re-captures the MD step.
 * Other values give AENET_E_ARG.
 */
#define AENET_OPT_MD_LIST 4
#define AENET_MD_LIST_AUTO 0
#define AENET_MD_LIST_OFF 1
#define AENET_MD_LIST_ON 2
int aenet_set_option(aenet_ctx *ctx, int option, int value);

/*
 * Energy gradient with respect to the network parameters (back-propagation,
 * Sec. II.C), summed over all atoms of the last evaluation:
 *   dE/dW^l[o][k] = sum_{i of species t} delta^l_i[o] x^{l-1}_i[k],
 *   dE/db^l[o]    = sum_{i of species t} delta^l_i[o]     (delta^L = 1, x^0 = g)
 * dEdW: [n_species * n_params] double, host or device, same layout as the
 * model's params. FP64 sums of FP32 products, deterministic. Returns
 * AENET_E_STATE if the last evaluation kept no activation records.
 * Synchronises when dEdW is host memory; with a device dEdW the work is only
 * enqueued on the context's stream.
 */
int aenet_grad_weights(aenet_ctx *ctx, double *dEdW);

/*
 * Replace the network parameters ([n_species * n_params] double, same layout as
 * at set-up; Sec. II.C trains exactly these). HOST params: converted on the host,
 * copied after a synchronisation of the context's stream. DEVICE params: the
 * conversion to FP32 and, in the BF16 forms, the packing of the tensor-core
 * operands run as kernels on the context's stream, after the work already
 * enqueued there and without any host round trip; the caller keeps params
 * valid until the stream reaches them. A captured MD step picks up the new
 * parameters on its next replay.
 */
int aenet_set_params(aenet_ctx *ctx, const double *params);

/* Synchronise the context's stream and report any recorded device error. */
int aenet_check(aenet_ctx *ctx);

/* Last error message of the context (or of the last failed setup when ctx is NULL). */
const char *aenet_last_error(const aenet_ctx *ctx);

/* Free the context and all its device memory. NULL is a no-op. */
void aenet_destroy(aenet_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* AENET_GPU_H */
