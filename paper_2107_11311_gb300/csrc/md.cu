// Rows a7 and a9 of the path: FP64 reductions of the total energy (the
// Behler-Parrinello sum E = sum_i E_i) and the virial, outputs back in input
// order, and the velocity-Verlet NVE update (the propagation step of the MD
// cycle, Fig. 1) in FP64. All reductions are two-level and deterministic:
// per-CTA partials are summed by one CTA in a fixed order.
#include "aenet_internal.cuh"

namespace aenet {

int ann_blocks(int n);

namespace {

constexpr double kEvPerAmu = 9648.533212;  // (A/ps)^2 per eV/amu

__device__ inline double block_sum(double v, double *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
    }
    __syncthreads();
    return s;  // valid in thread 0
}

// energy = sum of ANN-block partials; virial = sum of cell partials.
__global__ void k_reduce(int n_eblocks, const double *__restrict__ e_part, int n_vblocks,
                         const double *__restrict__ vir_part, double *__restrict__ result) {
    __shared__ double sh[32];
    double e = 0.0;
    for (int k = threadIdx.x; k < n_eblocks; k += blockDim.x) e += e_part[k];
    e = block_sum(e, sh);
    if (threadIdx.x == 0) result[0] = e;
    for (int c = 0; c < 9; ++c) {
        double v = 0.0;
        for (int k = threadIdx.x; k < n_vblocks; k += blockDim.x) v += vir_part[(size_t)k * 9 + c];
        v = block_sum(v, sh);
        if (threadIdx.x == 0) result[1 + c] = v;
    }
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

// v += dt/2 F/m c;  x += dt v
__global__ void k_vv_first(int n, double dt, double *__restrict__ pos, double *__restrict__ vel,
                           const double *__restrict__ F, const int32_t *__restrict__ types,
                           const double *__restrict__ mass) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double k = 0.5 * dt * kEvPerAmu / mass[types[i]];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double v = vel[3 * i + a] + k * F[3 * i + a];
        vel[3 * i + a] = v;
        pos[3 * i + a] += dt * v;
    }
}

// v += dt/2 F/m c, and the kinetic energy sum_i m v^2 / (2 c) as CTA partials
__global__ void k_vv_second(int n, double dt, double *__restrict__ vel, const double *__restrict__ F,
                            const int32_t *__restrict__ types, const double *__restrict__ mass,
                            double *__restrict__ ke_part) {
    __shared__ double sh[32];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0.0;
    if (i < n) {
        const double m = mass[types[i]];
        const double k = 0.5 * dt * kEvPerAmu / m;
        double v2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double v = vel[3 * i + a] + k * F[3 * i + a];
            if (dt != 0.0) vel[3 * i + a] = v;
            v2 += v * v;
        }
        ke = 0.5 * m * v2 / kEvPerAmu;
    }
    ke = block_sum(ke, sh);
    if (threadIdx.x == 0) ke_part[blockIdx.x] = ke;
}

// rec_pot[step] = E, rec_kin[step] = sum of kinetic partials; step++.
__global__ void k_record(int n_kblocks, const double *__restrict__ ke_part, const double *__restrict__ result,
                         int *__restrict__ step, double *__restrict__ rec_pot, double *__restrict__ rec_kin) {
    __shared__ double sh[32];
    double ke = 0.0;
    for (int k = threadIdx.x; k < n_kblocks; k += blockDim.x) ke += ke_part[k];
    ke = block_sum(ke, sh);
    if (threadIdx.x == 0) {
        const int s = *step;
        rec_pot[s] = result[0];
        rec_kin[s] = ke;
        *step = s + 1;
    }
}

}  // namespace

cudaError_t launch_finalize(Context &c, const Grid &g, int n, double *forces, double *e_atom) {
    k_reduce<<<1, 1024, 0, c.stream>>>(ann_blocks(n), c.d_e_part, g.ncell, c.d_vir_part, c.d_result);
    if ((forces || e_atom) && n > 0)
        k_unsort_outputs<<<(n + 255) / 256, 256, 0, c.stream>>>(n, c.d_perm, c.d_F4, c.d_eatom, forces, e_atom);
    return cudaGetLastError();
}

cudaError_t launch_unsort_G(Context &c, int n, float *G) {
    if (n <= 0) return cudaSuccess;
    k_unsort_G<<<1024, 256, 0, c.stream>>>(n, c.basis.D, c.d_perm, c.d_G, G);
    return cudaGetLastError();
}

cudaError_t launch_vv_first(Context &c, int n, double dt, double *pos, double *vel, const double *F,
                            const int32_t *types) {
    if (n <= 0) return cudaSuccess;
    k_vv_first<<<(n + 255) / 256, 256, 0, c.stream>>>(n, dt, pos, vel, F, types, c.d_mass);
    return cudaGetLastError();
}

cudaError_t launch_vv_second(Context &c, int n, double dt, double *vel, const double *F, const int32_t *types) {
    if (n <= 0) return cudaSuccess;
    k_vv_second<<<(n + 255) / 256, 256, 0, c.stream>>>(n, dt, vel, F, types, c.d_mass, c.d_ke_part);
    return cudaGetLastError();
}

cudaError_t launch_record(Context &c, int n, double *rec_pot, double *rec_kin) {
    k_record<<<1, 1024, 0, c.stream>>>((n + 255) / 256, c.d_ke_part, c.d_result, c.d_step, rec_pot, rec_kin);
    return cudaGetLastError();
}

}  // namespace aenet
