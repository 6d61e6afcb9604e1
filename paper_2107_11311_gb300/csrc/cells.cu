// The periodic cell list: wrap FP64 positions into the box, bin them into the
// cell grid (edge >= the largest cutoff) and sort them by cell.
//
// Every atom is stored as FP32 coordinates RELATIVE TO ITS CELL ORIGIN
// (u = x_wrapped - c h, computed in FP64 and then rounded), so that a
// displacement d = u_j + offset*h - u_i carries an absolute error of a few 1e-7 A
// whatever the box size; absolute FP32 coordinates in a 150 A box would carry
// ~1e-5 A.
#include "aenet_internal.cuh"
#include "cell_scan.cuh"

namespace aenet {

__global__ void k_bin_count(int n, int n_species, const double *__restrict__ pos,
                            const int32_t *__restrict__ types, Grid g,
                            float4 *__restrict__ tmp4, int *__restrict__ cell_of, int *__restrict__ slot,
                            int *__restrict__ cell_count, unsigned *__restrict__ err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float u[3];
    bool finite = true;
    const int cell = bin_position(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], g, u, finite);
    if (!finite) atomicOr(err, kErrNonfinite);
    int t = types[i];
    if (t < 0 || t >= n_species) {
        atomicOr(err, kErrType);
        t = 0;
    }
    tmp4[i] = make_float4(u[0], u[1], u[2], __int_as_float(t));
    cell_of[i] = cell;
    slot[i] = atomicAdd(&cell_count[cell], 1);
}

// Batched binning: atom i belongs to the structure with the largest atom0 <= i
// (binary search); its cell is offset into the global cell index space.
__global__ void k_bin_count_batch(int n, int n_struct, int n_species, const double *__restrict__ pos,
                                  const int32_t *__restrict__ types, const StructInfo *__restrict__ sinfo,
                                  float4 *__restrict__ tmp4, int *__restrict__ cell_of, int *__restrict__ slot,
                                  int *__restrict__ cell_count, unsigned *__restrict__ err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = n_struct - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sinfo[mid].atom0 <= i) lo = mid; else hi = mid - 1;
    }
    const StructInfo &si = sinfo[lo];
    float u[3];
    bool finite = true;
    const int cell = si.cell0 + bin_position(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], si.g, u, finite);
    if (!finite) atomicOr(err, kErrNonfinite);
    int t = types[i];
    if (t < 0 || t >= n_species) {
        atomicOr(err, kErrType);
        t = 0;
    }
    tmp4[i] = make_float4(u[0], u[1], u[2], __int_as_float(t));
    cell_of[i] = cell;
    slot[i] = atomicAdd(&cell_count[cell], 1);
}

// Exclusive scan of the cell counts by one CTA (scan_cells_block).
__global__ void k_scan_cells(int ncell, int *__restrict__ count, int *__restrict__ start) {
    scan_cells_block(ncell, count, start);
}

// Atom i to its sorted position s = cell_start[cell] + rank; slot[i] then holds
// s itself (the MD kernels read the forces of atom i at F4[slot[i]]).
__global__ void k_scatter(int n, const float4 *__restrict__ tmp4, const int *__restrict__ cell_of,
                          int *__restrict__ slot, const int *__restrict__ cell_start,
                          float4 *__restrict__ pos4, int *__restrict__ perm) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int s = cell_start[cell_of[i]] + slot[i];
    pos4[s] = tmp4[i];
    perm[s] = i;
    slot[i] = s;
}

cudaError_t launch_scan(Context &c, const Grid &g) {
    k_scan_cells<<<1, 1024, 0, c.stream>>>(g.ncell, c.d_cell_count, c.d_cell_start);
    return cudaGetLastError();
}

cudaError_t launch_scatter(Context &c, int n) {
    if (n > 0)
        k_scatter<<<(n + 255) / 256, 256, 0, c.stream>>>(n, c.d_tmp4, c.d_cell_of, c.d_slot, c.d_cell_start,
                                                         c.d_pos4, c.d_perm);
    return cudaGetLastError();
}

cudaError_t launch_sort(Context &c, const Grid &g, int n) {
    k_scan_cells<<<1, 1024, 0, c.stream>>>(g.ncell, c.d_cell_count, c.d_cell_start);
    if (n > 0) {
        k_scatter<<<(n + 255) / 256, 256, 0, c.stream>>>(n, c.d_tmp4, c.d_cell_of, c.d_slot, c.d_cell_start,
                                                         c.d_pos4, c.d_perm);
    }
    return cudaGetLastError();
}

cudaError_t launch_cells(Context &c, const Grid &g, int n, const double *pos, const int32_t *types) {
    cudaError_t e = cudaMemsetAsync(c.d_cell_count, 0, sizeof(int) * g.ncell, c.stream);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        k_bin_count<<<(n + 255) / 256, 256, 0, c.stream>>>(n, c.basis.n_species, pos, types, g, c.d_tmp4,
                                                           c.d_cell_of, c.d_slot, c.d_cell_count, c.d_err);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_sort(c, g, n);
}

cudaError_t launch_cells_batch(Context &c, int n, int total_cells, const double *pos, const int32_t *types) {
    cudaError_t e = cudaMemsetAsync(c.d_cell_count, 0, sizeof(int) * total_cells, c.stream);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        k_bin_count_batch<<<(n + 255) / 256, 256, 0, c.stream>>>(n, c.batch_n, c.basis.n_species, pos, types,
                                                                 c.batch_sinfo, c.d_tmp4, c.d_cell_of, c.d_slot,
                                                                 c.d_cell_count, c.d_err);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    Grid g{};
    g.ncell = total_cells;
    return launch_sort(c, g, n);
}

}  // namespace aenet
