// FP64 reductions of the total energy (the
// Behler-Parrinello sum E = sum_i E_i) and the virial, outputs back in input
// order, and the velocity-Verlet NVE update (the propagation step of the MD
// cycle, Fig. 1) in FP64.
//
// FP64 arithmetic has a long latency on this part, so every FP64 reduction is a
// wide tree (independent accumulators per thread, then shuffles) rather than a
// serial chain, divisions are replaced by host-computed reciprocals, and the
// MD step runs in two kernels around the potential: kick + drift + binning, and
// closing kick + all reductions (the last CTA to finish sums every partial in a
// fixed order, so results are deterministic).
#include "aenet_internal.cuh"
#include "cell_scan.cuh"

namespace aenet {

namespace {

constexpr double kEvPerAmu = 9648.533212;  // (A/ps)^2 per eV/amu
constexpr int kRedThreads = 256;
constexpr int kMdThreads = 256;

// Per-species kick factor dt/2 * c / m and kinetic factor m / (2 c).
struct KickParams {
    double k[kMaxSpecies];
    double hm[kMaxSpecies];
};

// Berendsen weak coupling: velocities are scaled by lambda at the start of each
// step, lambda = sqrt(1 + dt/tau (T0/T - 1)) with T = 2 E_kin / ((3N - 3) k_B)
// of the frame the step starts from. lambda == nullptr: NVE.
struct Thermostat {
    double *lambda;
    double T0, dt_over_tau, inv_dof_kb;
};

__device__ inline double select_species(const double (&v)[kMaxSpecies], int t) {
    double r = v[0];
#pragma unroll
    for (int s = 1; s < kMaxSpecies; ++s)
        if (t == s) r = v[s];
    return r;
}

__device__ inline double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of n values x[k * stride] (read through L2) by one warp: four independent
// accumulators per lane, then a shuffle tree. Result valid in every lane.
__device__ inline double warp_reduce_strided(const double *x, int n, int stride, int lane) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int k = lane;
    for (; k + 96 < n; k += 128) {
        a0 += __ldcg(x + (size_t)k * stride);
        a1 += __ldcg(x + (size_t)(k + 32) * stride);
        a2 += __ldcg(x + (size_t)(k + 64) * stride);
        a3 += __ldcg(x + (size_t)(k + 96) * stride);
    }
    for (; k < n; k += 32) a0 += __ldcg(x + (size_t)k * stride);
    return warp_sum_d((a0 + a1) + (a2 + a3));
}

// result[q] for q = 0 (energy, n_e partials) and 1..9 (virial, n_v x 9 partials):
// one warp per quantity.
__global__ void k_reduce(int n_e, const double *__restrict__ e_part, int n_v, const double *__restrict__ vir_part,
                         double *__restrict__ result) {
    const int lane = threadIdx.x & 31;
    const int q = blockIdx.x * (kRedThreads / 32) + (threadIdx.x >> 5);
    if (q > 9) return;
    const double v = q == 0 ? warp_reduce_strided(e_part, n_e, 1, lane)
                            : warp_reduce_strided(vir_part + (q - 1), n_v, 9, lane);
    if (lane == 0) result[q] = v;
}

__global__ void k_unsort_outputs(int n, const int *__restrict__ perm, const float4 *__restrict__ F4,
                                 const float *__restrict__ eatom, double *__restrict__ forces,
                                 double *__restrict__ e_atom_out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int i = perm[s];
    if (forces) {
        const float4 f = F4[s];
        forces[3 * i + 0] = (double)f.x;
        forces[3 * i + 1] = (double)f.y;
        forces[3 * i + 2] = (double)f.z;
    }
    if (e_atom_out) e_atom_out[i] = (double)eatom[s];
}

__global__ void k_unsort_G(int n, int D, const int *__restrict__ perm, const float *__restrict__ Gs,
                           float *__restrict__ G) {
    const size_t total = (size_t)n * D;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(k / D), c = (int)(k % D);
        G[(size_t)perm[s] * D + c] = Gs[k];
    }
}

// The per-atom part of k_md_kick_drift_bin.
__device__ inline void md_kick_drift_bin_atom(int i, int n_species, const KickParams &kp, double dt,
                                              double *__restrict__ pos, double *__restrict__ vel,
                                              const int32_t *__restrict__ types, float4 *__restrict__ F4,
                                              const Grid &g, float4 *__restrict__ tmp4, int *__restrict__ cell_of,
                                              int *__restrict__ slot, int *__restrict__ cell_count,
                                              unsigned *__restrict__ err, const double *__restrict__ lambda) {
    const double scale = lambda ? *lambda : 1.0;  // thermostat (1 for NVE)
    int t = types[i];
    if (t < 0 || t >= n_species) {
        atomicOr(err, kErrType);
        t = 0;
    }
    const int s_old = slot[i];
    const float4 f = F4[s_old];
    F4[s_old] = make_float4(0.f, 0.f, 0.f, 0.f);
    const double k = select_species(kp.k, t);
    double x[3];
    const float fa[3] = {f.x, f.y, f.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double v = fma(k, (double)fa[a], scale * vel[3 * i + a]);
        vel[3 * i + a] = v;
        x[a] = fma(dt, v, pos[3 * i + a]);
        pos[3 * i + a] = x[a];
    }
    float u[3];
    bool finite = true;
    const int cell = bin_position(x[0], x[1], x[2], g, u, finite);
    if (!finite) atomicOr(err, kErrNonfinite);
    tmp4[i] = make_float4(u[0], u[1], u[2], __int_as_float(t));
    cell_of[i] = cell;
    slot[i] = atomicAdd(&cell_count[cell], 1);
}


// v += dt/2 F/m c; x += dt v; then bin x (as k_bin_count), and the last CTA
// to finish scans the cell counts into the cell starts. F comes from the
// previous evaluation, in its cell-sorted order: slot[i] still holds atom i's
// sorted position of that evaluation (k_scatter). Each atom's force entry is
// read once here and cleared, so the potential kernel that follows finds F4
// zeroed; the cell counts were cleared by the previous scan and the neighbour
// statistics are cleared here, so the step needs no memset.
__global__ void k_md_kick_drift_bin(int n, int n_species, KickParams kp, double dt, double *__restrict__ pos,
                                    double *__restrict__ vel, const int32_t *__restrict__ types,
                                    float4 *__restrict__ F4, Grid g, float4 *__restrict__ tmp4,
                                    int *__restrict__ cell_of, int *__restrict__ slot, int *__restrict__ cell_count,
                                    int *__restrict__ cell_start, unsigned *__restrict__ done,
                                    unsigned long long *__restrict__ stats, unsigned *__restrict__ err,
                                    const double *__restrict__ lambda) {
    __shared__ bool s_last;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 4 && stats) stats[i] = 0ull;
    if (i < n) md_kick_drift_bin_atom(i, n_species, kp, dt, pos, vel, types, F4, g, tmp4, cell_of, slot, cell_count,
                                      err, lambda);
    // the last CTA to finish binning turns the counts into the cell starts
    // (done == NULL: a separate scan kernel follows; the same for every thread)
    if (!done) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    scan_cells_block(g.ncell, cell_count, cell_start);
    if (threadIdx.x == 0) *done = 0u;  // left at zero for the next user of the counter
}

// v += dt/2 F/m c with F of the current evaluation. Every CTA also sums a fixed
// slice of the potential's energy and virial partial rows and its atoms'
// kinetic energy into an 11-entry row of cta_part; the last CTA reduces those
// rows into result[0..10] (energy, virial, kinetic energy) and appends
// (E_pot, E_kin) to the records. The partition is by CTA index, so the FP64 sums
// do not depend on scheduling.
__global__ void __launch_bounds__(kMdThreads)
    k_md_kick_finish(int n, KickParams kp, double *__restrict__ vel, const int32_t *__restrict__ types,
                     const float4 *__restrict__ F4, const int *__restrict__ slot, int n_e,
                     const double *__restrict__ e_part, int n_v,
                     const double *__restrict__ vir_part, double *__restrict__ cta_part, unsigned *__restrict__ done,
                     double *__restrict__ result, int *__restrict__ step, double *__restrict__ rec_pot,
                     double *__restrict__ rec_kin, unsigned *__restrict__ vl_flag,
                     unsigned long long *__restrict__ vl_builds, Thermostat th) {
    __shared__ double s_w[kMdThreads / 32];
    __shared__ bool s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i = blockIdx.x * blockDim.x + tid;
    double ke = 0.0;
    if (i < n) {
        const int t = types[i];
        const float4 f = F4[slot[i]];  // sorted position of atom i (k_scatter)
        const double k = select_species(kp.k, t);
        const double vx = fma(k, (double)f.x, vel[3 * i + 0]);
        const double vy = fma(k, (double)f.y, vel[3 * i + 1]);
        const double vz = fma(k, (double)f.z, vel[3 * i + 2]);
        vel[3 * i + 0] = vx;
        vel[3 * i + 1] = vy;
        vel[3 * i + 2] = vz;
        ke = select_species(kp.hm, t) * fma(vx, vx, fma(vy, vy, vz * vz));
    }
    ke = warp_sum_d(ke);
    if (lane == 0) s_w[warp] = ke;
    // this CTA's slice of the energy (q = 0) and virial (q = 1..9) partial rows
    double *row = cta_part + (size_t)blockIdx.x * 11;
    for (int q = warp; q < 10; q += kMdThreads / 32) {
        const int rows = q == 0 ? n_e : n_v;
        const int per = (rows + gridDim.x - 1) / gridDim.x;
        const int r0 = min(rows, (int)blockIdx.x * per), r1 = min(rows, r0 + per);
        double a = 0.0;
        for (int r = r0 + lane; r < r1; r += 32)
            a += q == 0 ? __ldcg(e_part + r) : __ldcg(vir_part + (size_t)r * 9 + (q - 1));
        a = warp_sum_d(a);
        if (lane == 0) row[q] = a;
    }
    __syncthreads();
    if (warp == 0) {
        double v = lane < kMdThreads / 32 ? s_w[lane] : 0.0;
        v = warp_sum_d(v);
        if (lane == 0) {
            row[10] = v;
            __threadfence();
            s_last = atomicAdd(done, 1u) == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // last CTA: the 11 columns over the CTAs' rows, one warp each
    for (int q = warp; q < 11; q += kMdThreads / 32) {
        const double v = warp_reduce_strided(cta_part + q, gridDim.x, 11, lane);
        if (lane == 0) result[q] = v;
    }
    __syncthreads();
    if (tid == 0) {
        *done = 0u;
        if (vl_flag && vl_flag[0]) {  // this step rebuilt the Verlet list
            ++*vl_builds;
            vl_flag[0] = 0u;
        }
        if (rec_pot) {
            const int s = *step;
            rec_pot[s] = result[0];
            rec_kin[s] = result[10];
            *step = s + 1;
        }
        if (th.lambda) {  // Berendsen factor of the next step, from this frame's temperature
            const double T = 2.0 * result[10] * th.inv_dof_kb;
            const double l2 = T > 0.0 ? 1.0 + th.dt_over_tau * (th.T0 / T - 1.0) : 1.0;
            *th.lambda = l2 > 0.0 ? sqrt(l2) : 0.0;
        }
    }
}

// Verlet form of v += dt/2 F/m c; x += dt v (the list is kept, nothing is
// binned). The FP32 coordinate of atom i is refreshed relative to the origin of
// its cell at the last list build, u = x - origin, and written to its sorted
// slot of that build (slot[i]), so the list's image offsets stay valid; its
// force entry is cleared after it is read. An atom that moved
// more than skin/2 since the build (or is not finite) raises flag[0]; the last
// CTA to finish turns the flag into the value of the graph conditional that
// guards the rebuild.
__global__ void k_md_vl_kick_drift(int n, int n_species, KickParams kp, double dt, double half_skin2,
                                   double *__restrict__ pos, double *__restrict__ vel,
                                   const int32_t *__restrict__ types, float4 *__restrict__ F4,
                                   const int *__restrict__ slot, const double *__restrict__ origin,
                                   const double *__restrict__ ref, float4 *__restrict__ pos4,
                                   unsigned *__restrict__ flag, cudaGraphConditionalHandle cond,
                                   unsigned long long *__restrict__ stats, unsigned *__restrict__ err,
                                   const double *__restrict__ lambda) {
    __shared__ bool s_last;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 4 && stats) stats[i] = 0ull;  // neighbour statistics of the step's potential
    bool moved = false;
    if (i < n) {
        int t = types[i];
        if (t < 0 || t >= n_species) {
            atomicOr(err, kErrType);
            t = 0;
        }
        const int s = slot[i];
        const float4 f = F4[s];
        F4[s] = make_float4(0.f, 0.f, 0.f, 0.f);
        const double k = select_species(kp.k, t);
        const float fa[3] = {f.x, f.y, f.z};
        double x[3], d2 = 0.0;
        float u[3];
        const double scale = lambda ? *lambda : 1.0;  // thermostat (1 for NVE)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double v = fma(k, (double)fa[a], scale * vel[3 * i + a]);
            vel[3 * i + a] = v;
            x[a] = fma(dt, v, pos[3 * i + a]);
            pos[3 * i + a] = x[a];
            u[a] = (float)(x[a] - origin[3 * i + a]);
            const double dx = x[a] - ref[3 * i + a];
            d2 = fma(dx, dx, d2);
        }
        moved = !(d2 <= half_skin2);  // also true for a non-finite position
        pos4[s] = make_float4(u[0], u[1], u[2], __int_as_float(t));
    }
    if (__any_sync(0xffffffffu, moved) && (threadIdx.x & 31) == 0) {
        atomicOr(&flag[0], 1u);
        __threadfence();  // ordered before this CTA's arrival below
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&flag[1], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        const unsigned rebuild = atomicOr(&flag[0], 0u);
        cudaGraphSetConditional(cond, rebuild ? 1u : 0u);
        flag[1] = 0u;
    }
}

// Rebuild of the Verlet list, binning: as k_bin_count, plus the origin of each
// atom's FP32 coordinates (x - u in FP64) and its reference position x.
__global__ void k_md_vl_bin(int n, int n_species, const double *__restrict__ pos,
                            const int32_t *__restrict__ types, Grid g, float4 *__restrict__ tmp4,
                            int *__restrict__ cell_of, int *__restrict__ slot, int *__restrict__ cell_count,
                            double *__restrict__ origin, double *__restrict__ ref, unsigned *__restrict__ err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x0 = pos[3 * i], x1 = pos[3 * i + 1], x2 = pos[3 * i + 2];
    float u[3];
    double ud[3];
    bool finite = true;
    const int cell = bin_position(x0, x1, x2, g, u, finite, ud);
    if (!finite) atomicOr(err, kErrNonfinite);
    int t = types[i];
    if (t < 0 || t >= n_species) {
        atomicOr(err, kErrType);
        t = 0;
    }
    const double xs[3] = {x0, x1, x2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        origin[3 * i + a] = xs[a] - ud[a];
        ref[3 * i + a] = xs[a];
    }
    tmp4[i] = make_float4(u[0], u[1], u[2], __int_as_float(t));
    cell_of[i] = cell;
    slot[i] = atomicAdd(&cell_count[cell], 1);
}

// One warp per structure of a batch: energy = FP64 sum of its atoms' E_i (its
// atoms are contiguous in cell order), virial = FP64 sum of its cells' partials.
__global__ void k_batch_reduce(int n_struct, const StructInfo *__restrict__ sinfo, const int *__restrict__ cell_start,
                               const float *__restrict__ eatom, const double *__restrict__ vir_part,
                               double *__restrict__ out, double *__restrict__ energies,
                               double *__restrict__ virials) {
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= n_struct) return;
    const int c0 = sinfo[s].cell0, c1 = c0 + sinfo[s].ncell;
    const int a0 = cell_start[c0], a1 = cell_start[c1];
    double e0 = 0.0, e1 = 0.0;
    int k = a0 + lane;
    for (; k + 32 < a1; k += 64) {
        e0 += (double)eatom[k];
        e1 += (double)eatom[k + 32];
    }
    if (k < a1) e0 += (double)eatom[k];
    const double e = warp_sum_d(e0 + e1);
    if (lane == 0) {
        if (out) out[(size_t)s * 10] = e;
        if (energies) energies[s] = e;
    }
    for (int q = 0; q < 9; ++q) {
        const double v = warp_reduce_strided(vir_part + (size_t)c0 * 9 + q, c1 - c0, 9, lane);
        if (lane == 0) {
            if (out) out[(size_t)s * 10 + 1 + q] = v;
            if (virials) virials[(size_t)s * 9 + q] = v;
        }
    }
}

bool thermostat_on(const Context &c) { return c.thermo_tau > 0.0 && c.d_lambda; }

Thermostat thermostat(const Context &c, int n) {
    Thermostat th{};
    if (!thermostat_on(c)) return th;
    const int dof = 3 * n - 3 > 0 ? 3 * n - 3 : 1;
    th.lambda = c.d_lambda;
    th.T0 = c.thermo_T0;
    th.dt_over_tau = c.thermo_dt / c.thermo_tau;
    th.inv_dof_kb = 1.0 / (dof * 8.617333262e-5);
    return th;
}

KickParams kick_params(const Context &c, double dt) {
    KickParams kp{};
    for (int t = 0; t < kMaxSpecies; ++t) {
        const double m = t < (int)c.mass.size() ? c.mass[t] : 1.0;
        kp.k[t] = 0.5 * dt * kEvPerAmu / m;
        kp.hm[t] = 0.5 * m / kEvPerAmu;
    }
    return kp;
}

// Isotropic scaling of positions by the barostat.
__global__ void k_scale(double *__restrict__ x, long long count, double mu) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count; k += (long long)gridDim.x * blockDim.x)
        x[k] *= mu;
}

}  // namespace

cudaError_t launch_finalize(Context &c, const Grid &g, int n, int n_eparts, double *forces, double *e_atom) {
    k_reduce<<<(10 + kRedThreads / 32 - 1) / (kRedThreads / 32), kRedThreads, 0, c.stream>>>(
        n_eparts, c.d_e_part, c.last_vparts, c.d_vir_part, c.d_result);
    if ((forces || e_atom) && n > 0)
        k_unsort_outputs<<<(n + 255) / 256, 256, 0, c.stream>>>(n, c.d_perm, c.d_F4, c.d_eatom, forces, e_atom);
    return cudaGetLastError();
}

cudaError_t launch_finalize_forces(Context &c, int n, double *forces) {
    if (!forces || n <= 0) return cudaSuccess;
    k_unsort_outputs<<<(n + 255) / 256, 256, 0, c.stream>>>(n, c.d_perm, c.d_F4, c.d_eatom, forces, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_unsort_G(Context &c, int n, float *G) {
    if (n <= 0) return cudaSuccess;
    k_unsort_G<<<1024, 256, 0, c.stream>>>(n, c.basis.D, c.d_perm, c.d_G, G);
    return cudaGetLastError();
}

cudaError_t launch_batch_reduce(Context &c, double *energies, double *virials) {
    const int per = kRedThreads / 32;
    double *rows = (energies || virials) ? nullptr : c.d_bres;
    k_batch_reduce<<<(c.batch_n + per - 1) / per, kRedThreads, 0, c.stream>>>(
        c.batch_n, c.batch_sinfo, c.d_cell_start, c.d_eatom, c.d_vir_part, rows, energies, virials);
    return cudaGetLastError();
}

// Kick, drift, binning and the scan of the cell counts (the cell counts are
// zero: every binning is followed by a scan, which clears them, and a newly
// allocated count array is cleared once); k_scatter follows (launch_scatter).
// The last CTA scans when one pass of its threads covers the cells (4 per
// thread); a larger grid gets the 1,024-thread scan kernel instead (13,824
// cells: 32 us in the kick's last CTA against 8 us as a kernel).
cudaError_t launch_md_kick_drift_bin(Context &c, const Grid &g, int n, double dt, double *pos, double *vel,
                                     const int32_t *types) {
    if (n <= 0) return launch_sort(c, g, n);  // no atoms: the (all-zero) cell starts still come from a scan
    const bool fold = g.ncell <= 4 * kMdThreads;
    k_md_kick_drift_bin<<<(n + kMdThreads - 1) / kMdThreads, kMdThreads, 0, c.stream>>>(
        n, c.basis.n_species, kick_params(c, dt), dt, pos, vel, types, c.d_F4, g, c.d_tmp4, c.d_cell_of, c.d_slot,
        c.d_cell_count, c.d_cell_start, fold ? c.d_done : nullptr, c.d_stats, c.d_err,
        thermostat_on(c) ? c.d_lambda : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || fold) return e;
    return launch_scan(c, g);
}

cudaError_t launch_scale(Context &c, double *x, long long count, double mu) {
    if (count <= 0) return cudaSuccess;
    const long long blocks = std::min<long long>((count + 255) / 256, 4LL * std::max(1, c.n_sm));
    k_scale<<<(int)blocks, 256, 0, c.stream>>>(x, count, mu);
    return cudaGetLastError();
}

cudaError_t launch_md_kick_finish(Context &c, int n, double dt, double *vel, const int32_t *types,
                                  double *rec_pot, double *rec_kin, bool clear_vl) {
    const int blocks = n > 0 ? (n + kMdThreads - 1) / kMdThreads : 1;
    k_md_kick_finish<<<blocks, kMdThreads, 0, c.stream>>>(
        n, kick_params(c, dt), vel, types, c.d_F4, c.d_slot, c.last_eparts,
        c.last_epart, c.last_vparts, c.last_vpart, c.d_ke_part, c.d_done, c.d_result, c.d_step, rec_pot, rec_kin,
        clear_vl ? c.d_vl_flag : nullptr, c.d_vl_builds, thermostat(c, n));
    return cudaGetLastError();
}

cudaError_t launch_md_vl_kick_drift(Context &c, int n, double dt, double *pos, double *vel, const int32_t *types,
                                    cudaGraphConditionalHandle cond) {
    const double h = 0.5 * c.skin;
    const int blocks = n > 0 ? (n + kMdThreads - 1) / kMdThreads : 1;
    k_md_vl_kick_drift<<<blocks, kMdThreads, 0, c.stream>>>(
        n, c.basis.n_species, kick_params(c, dt), dt, h * h, pos, vel, types, c.d_F4, c.d_slot, c.d_vl_origin,
        c.d_vl_ref, c.d_pos4, c.d_vl_flag, cond, c.d_stats, c.d_err,
        thermostat_on(c) ? c.d_lambda : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_md_vl_bin(Context &c, const Grid &g, int n, const double *pos, const int32_t *types) {
    cudaError_t e = cudaMemsetAsync(c.d_cell_count, 0, sizeof(int) * g.ncell, c.stream);
    if (e != cudaSuccess || n <= 0) return e;
    k_md_vl_bin<<<(n + kMdThreads - 1) / kMdThreads, kMdThreads, 0, c.stream>>>(
        n, c.basis.n_species, pos, types, g, c.d_tmp4, c.d_cell_of, c.d_slot, c.d_cell_count, c.d_vl_origin,
        c.d_vl_ref, c.d_err);
    return cudaGetLastError();
}

}  // namespace aenet
