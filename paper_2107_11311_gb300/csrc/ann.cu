// The per-species feed-forward networks (Sec. II.A,
// Eq. ANN-layer; tanh hidden layers, linear output) giving E_i, and their
// back-propagation to dE/dG_i for the force kernel.
//
// FP32 form: one thread per atom in cell-sorted order. A CTA loads its tile of
// descriptor rows with coalesced loads into shared memory (one padded row per
// thread, odd stride so that row-private accesses are bank-conflict free), all
// species' parameters sit in shared memory (broadcast reads), the layers run on
// the FP32 pipe and dE/dG leaves through the same coalesced tile path. The
// energy of the CTA is summed in FP64 into a per-CTA partial.
#include "aenet_internal.cuh"

namespace aenet {

namespace {

constexpr int kAnnThreads = 128;

__host__ __device__ inline int ann_row_len(const Net &net) {
    int maxw = 1;
    for (int l = 0; l <= net.n_layers; ++l) maxw = net.widths[l] > maxw ? net.widths[l] : maxw;
    int len = net.act_len + 2 * maxw;
    return len | 1;  // odd stride
}

__global__ void __launch_bounds__(kAnnThreads)
    k_ann_fp32(Net net, int n, const float4 *__restrict__ pos4, const float *__restrict__ G,
               const float *__restrict__ params, const float *__restrict__ shift, const float *__restrict__ scale,
               float *__restrict__ dEdG, float *__restrict__ eatom, double *__restrict__ e_part,
               float *__restrict__ act, int rec_len) {
    extern __shared__ __align__(16) float sm[];
    const int D = net.widths[0];
    const int L = net.n_layers;
    const int rowlen = ann_row_len(net);
    float *sP = sm;                                        // [n_species * n_params]
    float *sShift = sP + net.n_species * net.n_params;    // [n_species * D]
    float *sScale = sShift + net.n_species * D;           // [n_species * D]
    float *rows = sScale + net.n_species * D;             // [kAnnThreads * rowlen]
    __shared__ double s_e[kAnnThreads / 32];

    const int tid = threadIdx.x;
    const int s0 = blockIdx.x * kAnnThreads;
    const int nrows = min(kAnnThreads, n - s0);
    for (int k = tid; k < net.n_species * net.n_params; k += kAnnThreads) sP[k] = params[k];
    for (int k = tid; k < net.n_species * D; k += kAnnThreads) {
        sShift[k] = shift[k];
        sScale[k] = scale[k];
    }
    const float *gsrc = G + (size_t)s0 * D;
    for (int k = tid; k < nrows * D; k += kAnnThreads) rows[(k / D) * rowlen + (k % D)] = gsrc[k];
    __syncthreads();

    float E = 0.f;
    if (tid < nrows) {
        const int s = s0 + tid;
        const int t = __float_as_int(pos4[s].w);
        float *x = rows + tid * rowlen;
        const float *sh = sShift + t * D, *sc = sScale + t * D;
        for (int k = 0; k < D; ++k) x[k] = (x[k] - sh[k]) * sc[k];
        // forward
        const float *P = sP + t * net.n_params;
        int xin = 0, xout = D;
        const float *Wl = P;
        for (int l = 1; l <= L; ++l) {
            const int no = net.widths[l], ni = net.widths[l - 1];
            const float *W = Wl, *b = Wl + no * ni;
            for (int o = 0; o < no; ++o) {
                float z = b[o];
                const float *wr = W + o * ni;
                for (int k = 0; k < ni; ++k) z = fmaf(wr[k], x[xin + k], z);
                x[xout + o] = (l < L) ? tanhf(z) : z;
            }
            Wl = b + no;
            xin = xout;
            xout += no;
        }
        E = x[xin];
        eatom[s] = E;
        // optional activation record: g, then x_l and delta_l of every hidden layer
        float *rec = act ? act + (size_t)s * rec_len : nullptr;
        if (rec) {
            for (int k = 0; k < D; ++k) rec[k] = x[k];
            int r = D, a0 = D;
            for (int l = 1; l < L; ++l) {
                for (int k = 0; k < net.widths[l]; ++k) rec[r + k] = x[a0 + k];
                r += 2 * net.widths[l];
                a0 += net.widths[l];
            }
        }
        // back-propagation: delta^L = 1
        int maxw = 1;
        for (int l = 0; l <= L; ++l) maxw = net.widths[l] > maxw ? net.widths[l] : maxw;
        float *dcur = x + net.act_len, *dprev = dcur + maxw;
        dcur[0] = 1.0f;
        // offsets of layer parameters and activations
        int poff[kMaxLayers + 1], aoff[kMaxLayers + 1];
        poff[1] = 0;
        aoff[0] = 0;
        for (int l = 1; l <= L; ++l) {
            aoff[l] = aoff[l - 1] + net.widths[l - 1];
            if (l < L) poff[l + 1] = poff[l] + net.widths[l] * net.widths[l - 1] + net.widths[l];
        }
        for (int l = L; l >= 1; --l) {
            const int no = net.widths[l], ni = net.widths[l - 1];
            const float *W = P + poff[l];
            for (int k = 0; k < ni; ++k) {
                float acc = 0.f;
                for (int o = 0; o < no; ++o) acc = fmaf(W[o * ni + k], dcur[o], acc);
                if (l > 1) {
                    const float a = x[aoff[l - 1] + k];
                    acc *= (1.0f - a * a);
                }
                dprev[k] = acc;
            }
            if (rec && l > 1) {  // dprev = delta of hidden layer l - 1
                int r = D;
                for (int m = 1; m < l - 1; ++m) r += 2 * net.widths[m];
                for (int k = 0; k < ni; ++k) rec[r + net.widths[l - 1] + k] = dprev[k];
            }
            float *tmp = dcur;
            dcur = dprev;
            dprev = tmp;
        }
        for (int k = 0; k < D; ++k) x[k] = dcur[k] * sc[k];  // dE/dG = dE/dg * scale
    }
    // FP64 energy partial of the CTA
    double e = (double)E;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((tid & 31) == 0) s_e[tid >> 5] = e;
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int w = 0; w < kAnnThreads / 32; ++w) sum += s_e[w];
        e_part[blockIdx.x] = sum;
    }
    float *gdst = dEdG + (size_t)s0 * D;
    for (int k = tid; k < nrows * D; k += kAnnThreads) gdst[k] = rows[(k / D) * rowlen + (k % D)];
}

}  // namespace

size_t ann_smem_bytes(const Context &c) {
    const Net &net = c.net;
    const int D = net.widths[0];
    return sizeof(float) * ((size_t)net.n_species * net.n_params + 2 * (size_t)net.n_species * D +
                            (size_t)kAnnThreads * ann_row_len(net));
}

int ann_blocks(int n) { return (n + kAnnThreads - 1) / kAnnThreads; }

cudaError_t launch_ann(Context &c, int n) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = ann_smem_bytes(c);
    cudaError_t e = allow_max_smem(k_ann_fp32);
    if (e != cudaSuccess) return e;
    k_ann_fp32<<<ann_blocks(n), kAnnThreads, smem, c.stream>>>(c.net, n, c.d_pos4, c.d_G, c.d_params, c.d_shift,
                                                               c.d_scale, c.d_dEdG, c.d_eatom, c.d_e_part,
                                                               c.keep_act ? c.d_act : nullptr,
                                                               activation_record_len(c.net));
    return cudaGetLastError();
}

}  // namespace aenet
