// Angular fingerprint (Sec. II.B, Eq. angular) through the addition theorem of
// spherical harmonics, for angular orders up to 6 (Ka <= 7).
//
// With w_j = f_c(r_ij) and unit vectors u_j, the ordered-pair sum of the paper
//   S_a = sum_{j != k} w_j w_k T_a(u_j . u_k)
// is rewritten with T_a(x) = sum_l b_al P_l(x) (Legendre expansion of the
// Chebyshev polynomial; b_al = 0 for l > a and for l of the other parity) and
// the addition theorem P_l(u . v) = sum_m Z_lm(u) Z_lm(v), where Z_lm are the
// real spherical harmonics normalised so that the theorem has no prefactor:
//   S_a = sum_l b_al Q_l - sum_j w_j^2,   Q_l = sum_m (sum_j w_j Z_lm(u_j))^2
// (the j = k terms of the full double sum give T_a(1) = 1 times w_j^2). The
// species-weighted copy takes s_j w_j for w_j. The cost is O(neighbours x 49)
// instead of O(neighbour pairs x Ka).
//
// Components. Z_lm = N_lm Pbar_l^m(z) C_m(x, y) for m >= 0 and N_lm Pbar_l^m(z)
// S_m(x, y) for the sine part (m > 0), where Pbar_l^m = P_l^m / (1 - z^2)^{m/2}
// (associated Legendre function without the Condon-Shortley phase, divided by
// sin^m: a polynomial in z), C_m + i S_m = (x + i y)^m, and N_lm^2 = 1 (m = 0),
// 2 (l - m)! / (l + m)! (m > 0). The kernel accumulates the raw components
// v = Pbar C or Pbar S and applies N_lm^2 when it squares them. Pbar follows the
// standard recurrences Pbar_m^m = (2m - 1)!!, Pbar_{m+1}^m = (2m + 1) z Pbar_m^m,
// (l - m) Pbar_l^m = (2l - 1) z Pbar_{l-1}^m - (l + m - 1) Pbar_{l-2}^m.
//
// Gradient. With D_c = 2 N_c^2 A_c sum_a g_a b_{a l(c)} (g_a = dE/dG_a, A_c the
// component sums) and the same for the weighted copy (D'_c, s_j),
//   dE/dd_j = f_c'(r) [E_j - 2 w_j (sum_a g_a + s_j^2 sum_a g'_a)] u_j
//             + (w_j / r) (F_j - (F_j . u_j) u_j),
//   E_j = sum_c (D_c + s_j D'_c) v_c(u_j),  F_j = sum_c (D_c + s_j D'_c) grad_u v_c,
// with grad_u of Pbar C_m = (Pbar m C_{m-1}, -Pbar m S_{m-1}, Pbar' C_m) and of
// Pbar S_m = (Pbar m S_{m-1}, Pbar m C_{m-1}, Pbar' S_m) (x, y, z taken as
// independent; the projection removes the radial part).
#pragma once

#include "fp_common.cuh"

namespace aenet {
namespace detail {

constexpr int kShL = 6;        // degrees l = 0 .. 6
constexpr int kShComps = 49;   // sum of 2l + 1
constexpr int kShScratch = 128;  // floats of per-warp scratch the path needs
// shared-memory table of the path: b[a * 7 + l], then N_c^2, then l(c)
constexpr int kShTabB = 0, kShTabN = 49, kShTabL = 98, kShTab = 147;

// The bases that take the angular fingerprint through spherical harmonics:
// the exact-order forms with angular order 6 (the 4-species solid's basis).
template <int KRT, int KAT, bool EXACT>
__host__ __device__ constexpr bool sh_angular() {
    return EXACT && KAT == 7;
}

// component index of (l, m, kind): m = 0 first (c = l), then for each m > 0 the
// pairs (cos, sin) of l = m .. 6
__host__ __device__ constexpr int sh_comp(int l, int m, int kind) {
    return m == 0 ? l : kShL + 1 + (m - 1) * (2 * (kShL + 1) - m) + 2 * (l - m) + kind;
}

// (loops, not recursion: inside unrolled device loops they fold to constants)
__host__ __device__ constexpr double sh_fact(int n) {
    double f = 1.0;
    for (int k = 2; k <= n; ++k) f *= k;
    return f;
}
__host__ __device__ constexpr float sh_norm2(int l, int m) {
    return m == 0 ? 1.0f : (float)(2.0 * sh_fact(l - m) / sh_fact(l + m));
}

// Legendre coefficients b[a][l] of T_a, a, l <= 6 (host, FP64): T_a from its
// recurrence in the monomial basis, x^n to the Legendre basis by
// x P_l = ((l + 1) P_{l+1} + l P_{l-1}) / (2l + 1).
inline void sh_legendre_of_chebyshev(float (&b)[kShL + 1][kShL + 1]) {
    double t[kShL + 1][kShL + 1] = {};  // monomial coefficients of T_a
    t[0][0] = 1.0;
    t[1][1] = 1.0;
    for (int a = 2; a <= kShL; ++a)
        for (int n = 0; n <= a; ++n) t[a][n] = (n > 0 ? 2.0 * t[a - 1][n - 1] : 0.0) - t[a - 2][n];
    double xn[kShL + 1][kShL + 1] = {};  // Legendre coefficients of x^n
    xn[0][0] = 1.0;
    for (int n = 1; n <= kShL; ++n)
        for (int l = 0; l < n; ++l) {
            xn[n][l + 1] += xn[n - 1][l] * (l + 1) / (2.0 * l + 1.0);
            if (l > 0) xn[n][l - 1] += xn[n - 1][l] * l / (2.0 * l + 1.0);
        }
    for (int a = 0; a <= kShL; ++a)
        for (int l = 0; l <= kShL; ++l) {
            double s = 0.0;
            for (int n = 0; n <= kShL; ++n) s += t[a][n] * xn[n][l];
            b[a][l] = (float)s;
        }
}

// Accumulate the raw components of columns M0 .. M1 of one angular entry,
// acc[c - c0] += v_c(u) * wt (c0 the first component of column M0), and, with
// W2, acc[49 - c0] += wt^2 (the j = k term). Column by column, so only the
// current Pbar column and C_m, S_m are live; the columns are split in two
// groups (m <= 2: 29 components, m >= 3: 20 and the w^2 sum) so that one
// group's sums fit a 32-entry accumulator.
template <int M0, int M1, bool W2>
__device__ __forceinline__ void sh_accumulate(float x, float y, float z, float wt, float (&acc)[32]) {
    constexpr int c0 = sh_comp(M0, M0, 0);
    float cm = 1.f, sm = 0.f;  // C_m, S_m
    float pmm = 1.f;           // Pbar_m^m = (2m - 1)!! (a constant once the loop is unrolled)
#pragma unroll
    for (int m = 0; m <= M1; ++m) {
        if (m > 0) {
            const float c1 = x * cm - y * sm, s1 = fmaf(x, sm, y * cm);
            cm = c1;
            sm = s1;
            pmm *= (float)(2 * m - 1);
        }
        if (m < M0) continue;
        const float wc = wt * cm, ws = wt * sm;
        float p2 = 0.f, p1 = pmm;  // Pbar_{l-2}, Pbar_{l-1} (then Pbar_l)
#pragma unroll
        for (int l = m; l <= kShL; ++l) {
            float p;
            if (l == m) {
                p = p1;
            } else if (l == m + 1) {
                p = (float)(2 * m + 1) * z * p1;
            } else {
                const float a = (float)(2 * l - 1) / (float)(l - m), b = (float)(l + m - 1) / (float)(l - m);
                p = fmaf(a * z, p1, -b * p2);
            }
            if (l > m) {
                p2 = p1;
                p1 = p;
            }
            acc[sh_comp(l, m, 0) - c0] = fmaf(p, wc, acc[sh_comp(l, m, 0) - c0]);
            if (m > 0) acc[sh_comp(l, m, 1) - c0] = fmaf(p, ws, acc[sh_comp(l, m, 1) - c0]);
        }
    }
    if constexpr (W2) acc[kShComps - c0] = fmaf(wt, wt, acc[kShComps - c0]);
}

// dE/d(u) contraction of one entry: E = sum_c k_c v_c(u) and F = sum_c k_c
// grad_u v_c(u), k_c = D[2c] + s D[2c + 1] (coefficient pairs in shared memory).
// Called by all 32 lanes of the warp together (it synchronises the warp).
__device__ __forceinline__ void sh_contract(float x, float y, float z, float s, const float *D, float &E,
                                            float &Fx, float &Fy, float &Fz) {
    E = 0.f;
    Fx = 0.f;
    Fy = 0.f;
    Fz = 0.f;
    float cm = 1.f, sm = 0.f, cp = 0.f, sp = 0.f;  // C_m, S_m, C_{m-1}, S_{m-1}
    float pmm = 1.f;                                // (2m - 1)!!
#pragma unroll
    for (int m = 0; m <= kShL; ++m) {
        if (m > 0) {
            cp = cm;
            sp = sm;
            cm = x * cp - y * sp;
            sm = fmaf(x, sp, y * cp);
            pmm *= (float)(2 * m - 1);
        }
        // h = sum_l k Pbar, h' = sum_l k Pbar' for the cos and the sin parts of column m
        // (the warp sync keeps the compiler from hoisting every column's coefficient
        // loads to the top, which would hold ~100 registers)
        __syncwarp();
        float hc = 0.f, hs = 0.f, dhc = 0.f, dhs = 0.f;
        float p2 = 0.f, p1 = pmm, d2 = 0.f, d1 = 0.f;
#pragma unroll
        for (int l = m; l <= kShL; ++l) {
            float p, d;
            if (l == m) {
                p = p1;
                d = 0.f;
            } else if (l == m + 1) {
                p = (float)(2 * m + 1) * z * p1;
                d = (float)(2 * m + 1) * p1;
            } else {
                const float a = (float)(2 * l - 1) / (float)(l - m), b = (float)(l + m - 1) / (float)(l - m);
                p = fmaf(a * z, p1, -b * p2);
                d = fmaf(a, fmaf(z, d1, p1), -b * d2);
            }
            if (l > m) {
                p2 = p1;
                p1 = p;
                d2 = d1;
                d1 = d;
            }
            const float2 kc = *reinterpret_cast<const float2 *>(D + 2 * sh_comp(l, m, 0));
            const float k0 = fmaf(s, kc.y, kc.x);
            hc = fmaf(k0, p, hc);
            dhc = fmaf(k0, d, dhc);
            if (m > 0) {
                const float2 ks = *reinterpret_cast<const float2 *>(D + 2 * sh_comp(l, m, 1));
                const float k1 = fmaf(s, ks.y, ks.x);
                hs = fmaf(k1, p, hs);
                dhs = fmaf(k1, d, dhs);
            }
        }
        E = fmaf(hc, cm, fmaf(hs, sm, E));
        Fz = fmaf(dhc, cm, fmaf(dhs, sm, Fz));
        if (m > 0) {
            Fx = fmaf((float)m, fmaf(hc, cp, hs * sp), Fx);
            Fy = fmaf((float)m, fmaf(hs, cp, -hc * sp), Fy);
        }
    }
}

// The angular fingerprint S_a of one copy from its component sums A (49, and
// the sum of w^2 at [49]) in shared memory and the path's table:
// S_a = sum_c b_{a l(c)} N_c^2 A_c^2 - sum w^2. A plain loop over c with the
// table lookups keeps the register use small.
__device__ __forceinline__ float sh_fingerprint(const float *A, int alpha, const float *tab) {
    float G = -A[kShComps];
#pragma unroll 7
    for (int c = 0; c < kShComps; ++c) {
        const float ac = A[c];
        const float coef = tab[kShTabB + alpha * (kShL + 1) + (int)tab[kShTabL + c]] * tab[kShTabN + c];
        G = fmaf(coef * ac, ac, G);
    }
    return G;
}

// The path's table in shared memory (every thread of the CTA calls this).
__device__ __forceinline__ void load_sh_table(const float (&bt)[7][7], float *s_sh, int tid) {
#pragma unroll
    for (int a = 0; a <= kShL; ++a)
#pragma unroll
        for (int l = 0; l <= kShL; ++l)
            if (tid == a * (kShL + 1) + l) s_sh[kShTabB + a * (kShL + 1) + l] = bt[a][l];
    if (tid == 64) {
#pragma unroll
        for (int m = 0; m <= kShL; ++m)
#pragma unroll
            for (int l = m; l <= kShL; ++l)
#pragma unroll
                for (int kind = 0; kind < (m > 0 ? 2 : 1); ++kind) {
                    s_sh[kShTabN + sh_comp(l, m, kind)] = sh_norm2(l, m);
                    s_sh[kShTabL + sh_comp(l, m, kind)] = (float)l;
                }
    }
}

}  // namespace detail
}  // namespace aenet
