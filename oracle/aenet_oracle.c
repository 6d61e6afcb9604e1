/*
 * aenet_oracle.c -- plain FP64 CPU oracle of the ANN-potential hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library. The GPU product path never calls it
 * and shares no code, header or table with it.
 *
 * What it evaluates, written as the paper defines it and in the paper's order:
 *   - neighbours: every periodic image j+n within the cutoff of atom i,
 *     excluding only (j = i, n = 0); by brute force over all atoms and images
 *     (the definition), or through a cell list (checked against brute force);
 *   - descriptor (Sec. II.B): radial Chebyshev expansion (Eq. radial) with the
 *     recurrence for T_n and the cosine cutoff (Eq. cos-cutoff), angular
 *     expansion (Eq. angular) over ORDERED pairs (j, k) of distinct image-atoms,
 *     and the species-weighted copy of both sums (weights s_t of the neighbour
 *     species; s_j s_k for the angular sum), concatenated as
 *     G = [radial, angular, radial_w, angular_w];
 *   - standardisation g = (G - shift) * scale (a frozen input transform);
 *   - atomic energy E_i = ANN_t(g_i) (Sec. II.A, Eq. ANN-layer): tanh hidden
 *     layers, linear output; total E = sum_i E_i (Behler-Parrinello sum);
 *   - forces F = -dE/dr by back-propagation to dE/dG and the analytic
 *     derivative of every pair and triplet term; virial
 *     W_ab = -sum over displacement vectors d of d_a dE/dd_b;
 *   - dE/dW, dE/db (back-propagation, Sec. II.C) summed over atoms;
 *   - velocity-Verlet NVE integration in metal units.
 *
 * Periodic boxes: orthorhombic (edges L_x, L_y, L_z), or the restricted
 * triclinic cell of the MD codes the paper plugs into (LAMMPS): lattice vectors
 * a = (L_x, 0, 0), b = (xy, L_y, 0), c = (xz, yz, L_z). A tilted cell is handled
 * by brute force over lattice images only: x_j + n_a a + n_b b + n_c c.
 *
 * Derivative identities used (not printed in the paper, derived here):
 *   dT_n/dx = n U_{n-1}(x), U_0 = 1, U_1 = 2x, U_{n+1} = 2x U_n - U_{n-1};
 *   df_c/dr = -(pi / (2 R_c)) sin(pi r / R_c) for r <= R_c, else 0;
 *   d cos(theta)/d d_j = (u_k - cos(theta) u_j) / r_j  (u = unit vectors).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_E_ARG -1
#define ORC_E_NOMEM -7
#define ORC_E_OVERLAP -5

typedef struct {
    int n_species;
    const double *type_weight; /* [n_species] s_t of the weighted copy */
    double rc_rad;
    int order_rad;
    double rc_ang;
    int order_ang;
    int n_layers;              /* number of weight layers, e.g. 3 for D-h-h-1 */
    const int *widths;         /* [n_layers + 1]; widths[0] = D, widths[n_layers] = 1 */
    const double *params;      /* [n_species][n_params]: W^1 b^1 W^2 b^2 ... (W row-major) */
    const double *in_shift;    /* [n_species][D] or NULL */
    const double *in_scale;    /* [n_species][D] or NULL */
} orc_model;

typedef struct {
    int j;
    int img[3];
    double d[3];
    double r;
} orc_nb;

static const double ORC_PI = 3.14159265358979323846;

static int orc_D(const orc_model *m) { return 2 * (m->order_rad + 1 + m->order_ang + 1); }

static int orc_nparams(const orc_model *m) {
    int s = 0;
    for (int l = 1; l <= m->n_layers; ++l) s += m->widths[l] * m->widths[l - 1] + m->widths[l];
    return s;
}

/* ------------------------------------------------------------ basis pieces */

/* Chebyshev T_0..T_n at x by the three-term recurrence (Sec. II.B). */
static void cheb_T(int n, double x, double *T) {
    T[0] = 1.0;
    if (n >= 1) T[1] = x;
    for (int a = 1; a < n; ++a) T[a + 1] = 2.0 * x * T[a] - T[a - 1];
}

/* dT_a/dx = a U_{a-1}(x), U of the second kind by its own recurrence. */
static void cheb_dT(int n, double x, double *dT) {
    double Um1 = 0.0, U = 1.0; /* U_{-1} = 0, U_0 = 1 */
    dT[0] = 0.0;
    for (int a = 1; a <= n; ++a) {
        dT[a] = a * U; /* U holds U_{a-1} */
        double Un = 2.0 * x * U - Um1;
        Um1 = U;
        U = Un;
    }
}

/* Cosine cutoff (Eq. cos-cutoff) and its derivative. */
static double cutoff_fc(double r, double rc) {
    return (r <= rc) ? 0.5 * (cos(ORC_PI * r / rc) + 1.0) : 0.0;
}
static double cutoff_dfc(double r, double rc) {
    return (r <= rc) ? -0.5 * ORC_PI / rc * sin(ORC_PI * r / rc) : 0.0;
}

/* ------------------------------------------------------------ neighbours */

static double wrap1(double x, double L) {
    double w = x - floor(x / L) * L;
    if (w >= L) w -= L;
    if (w < 0.0) w = 0.0;
    return w;
}

/* A periodic box: edges L (the diagonal of the cell matrix) and the tilt
 * factors xy, xz, yz of the restricted triclinic form; tilted = any tilt != 0. */
typedef struct {
    double L[3];
    double xy, xz, yz;
    int tilted;
} orc_box;

static orc_box box_of(const double *box, const double *tilt) {
    orc_box B;
    for (int a = 0; a < 3; ++a) B.L[a] = box[a];
    B.xy = tilt ? tilt[0] : 0.0;
    B.xz = tilt ? tilt[1] : 0.0;
    B.yz = tilt ? tilt[2] : 0.0;
    B.tilted = B.xy != 0.0 || B.xz != 0.0 || B.yz != 0.0;
    return B;
}

/* Fractional coordinates s of x = H s, H upper triangular with columns a, b, c
 * (back substitution). */
static void to_fractional(const orc_box *B, const double *x, double *s) {
    s[2] = x[2] / B->L[2];
    s[1] = (x[1] - B->yz * s[2]) / B->L[1];
    s[0] = (x[0] - B->xy * s[1] - B->xz * s[2]) / B->L[0];
}

static void from_fractional(const orc_box *B, const double *s, double *x) {
    x[0] = B->L[0] * s[0] + B->xy * s[1] + B->xz * s[2];
    x[1] = B->L[1] * s[1] + B->yz * s[2];
    x[2] = B->L[2] * s[2];
}

/* Distance between the two lattice planes bounding the cell along each lattice
 * direction: volume / area of the face spanned by the other two vectors. */
static void plane_widths(const orc_box *B, double *w) {
    const double V = B->L[0] * B->L[1] * B->L[2];
    const double bc[3] = {B->L[1] * B->L[2], -B->xy * B->L[2], B->xy * B->yz - B->L[1] * B->xz}; /* b x c */
    const double ca[3] = {0.0, B->L[2] * B->L[0], -B->yz * B->L[0]};                           /* c x a */
    w[0] = V / sqrt(bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]);
    w[1] = V / sqrt(ca[0] * ca[0] + ca[1] * ca[1] + ca[2] * ca[2]);
    w[2] = B->L[2]; /* a x b = (0, 0, L_x L_y) */
}

typedef struct {
    int nc[3];
    double h[3];
    int m[3];
    int *start; /* [ncell + 1] */
    int *atoms; /* [n] */
} orc_cells;

static void cells_free(orc_cells *c) {
    free(c->start);
    free(c->atoms);
    c->start = c->atoms = NULL;
}

static int cells_build(orc_cells *c, int n, const double *wpos, const double *box, double rc) {
    for (int a = 0; a < 3; ++a) {
        int nc = (int)floor(box[a] / rc);
        c->nc[a] = nc < 1 ? 1 : nc;
        c->h[a] = box[a] / c->nc[a];
        c->m[a] = (int)ceil(rc / c->h[a]);
    }
    int ncell = c->nc[0] * c->nc[1] * c->nc[2];
    c->start = (int *)calloc((size_t)ncell + 1, sizeof(int));
    c->atoms = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *cid = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!c->start || !c->atoms || !cid) {
        free(cid);
        cells_free(c);
        return ORC_E_NOMEM;
    }
    for (int i = 0; i < n; ++i) {
        int ci[3];
        for (int a = 0; a < 3; ++a) {
            ci[a] = (int)floor(wpos[3 * i + a] / c->h[a]);
            if (ci[a] >= c->nc[a]) ci[a] = c->nc[a] - 1;
            if (ci[a] < 0) ci[a] = 0;
        }
        cid[i] = (ci[2] * c->nc[1] + ci[1]) * c->nc[0] + ci[0];
        c->start[cid[i] + 1]++;
    }
    for (int k = 0; k < ncell; ++k) c->start[k + 1] += c->start[k];
    int *fill = (int *)malloc(sizeof(int) * (size_t)ncell);
    if (!fill) {
        free(cid);
        cells_free(c);
        return ORC_E_NOMEM;
    }
    memcpy(fill, c->start, sizeof(int) * (size_t)ncell);
    for (int i = 0; i < n; ++i) c->atoms[fill[cid[i]]++] = i;
    free(fill);
    free(cid);
    return ORC_OK;
}

typedef struct {
    orc_nb *v;
    int n, cap;
} nb_buf;

static int nb_push(nb_buf *b, int j, const int img[3], const double d[3], double r) {
    if (b->n == b->cap) {
        int cap = b->cap ? 2 * b->cap : 256;
        orc_nb *nv = (orc_nb *)realloc(b->v, sizeof(orc_nb) * (size_t)cap);
        if (!nv) return ORC_E_NOMEM;
        b->v = nv;
        b->cap = cap;
    }
    orc_nb *e = &b->v[b->n++];
    e->j = j;
    e->r = r;
    for (int a = 0; a < 3; ++a) {
        e->img[a] = img[a];
        e->d[a] = d[a];
    }
    return ORC_OK;
}

/* Brute force: every atom j and every periodic image n with |x_j + nL - x_i| <= rc,
 * except (j = i, n = 0). x are wrapped into [0, L). */
static int neighbours_brute(int i, int n, const double *wpos, const double *box, double rc, nb_buf *out) {
    out->n = 0;
    const double rc2 = rc * rc;
    for (int j = 0; j < n; ++j) {
        double del[3];
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            del[a] = wpos[3 * j + a] - wpos[3 * i + a];
            lo[a] = (int)ceil((-rc - del[a]) / box[a]);
            hi[a] = (int)floor((rc - del[a]) / box[a]);
        }
        int img[3];
        for (img[0] = lo[0]; img[0] <= hi[0]; ++img[0])
            for (img[1] = lo[1]; img[1] <= hi[1]; ++img[1])
                for (img[2] = lo[2]; img[2] <= hi[2]; ++img[2]) {
                    if (j == i && img[0] == 0 && img[1] == 0 && img[2] == 0) continue;
                    double d[3], r2 = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        d[a] = del[a] + img[a] * box[a];
                        r2 += d[a] * d[a];
                    }
                    if (r2 > rc2) continue;
                    int e = nb_push(out, j, img, d, sqrt(r2));
                    if (e) return e;
                }
    }
    return ORC_OK;
}

/* Brute force in a tilted cell: every atom j and every lattice image
 * n = (n_a, n_b, n_c) with |x_j + n_a a + n_b b + n_c c - x_i| <= rc, except
 * (j = i, n = 0). A displacement with fractional coordinates f has length at
 * least |f_a| times the plane width along a, so |f_a| <= rc / width_a bounds
 * the images (widened by one on each side; the distance test decides). */
static int neighbours_brute_tri(int i, int n, const double *wpos, const orc_box *B, double rc, nb_buf *out) {
    out->n = 0;
    const double rc2 = rc * rc;
    double w[3];
    plane_widths(B, w);
    const double A[3][3] = {{B->L[0], 0.0, 0.0}, {B->xy, B->L[1], 0.0}, {B->xz, B->yz, B->L[2]}}; /* a, b, c */
    for (int j = 0; j < n; ++j) {
        double del[3], f[3];
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) del[a] = wpos[3 * j + a] - wpos[3 * i + a];
        to_fractional(B, del, f);
        for (int a = 0; a < 3; ++a) {
            lo[a] = (int)ceil(-rc / w[a] - f[a]) - 1;
            hi[a] = (int)floor(rc / w[a] - f[a]) + 1;
        }
        int img[3];
        for (img[0] = lo[0]; img[0] <= hi[0]; ++img[0])
            for (img[1] = lo[1]; img[1] <= hi[1]; ++img[1])
                for (img[2] = lo[2]; img[2] <= hi[2]; ++img[2]) {
                    if (j == i && img[0] == 0 && img[1] == 0 && img[2] == 0) continue;
                    double d[3], r2 = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        d[a] = del[a] + img[0] * A[0][a] + img[1] * A[1][a] + img[2] * A[2][a];
                        r2 += d[a] * d[a];
                    }
                    if (r2 > rc2) continue;
                    int e = nb_push(out, j, img, d, sqrt(r2));
                    if (e) return e;
                }
    }
    return ORC_OK;
}

/* Cell list: cells of edge h >= rc (or one cell per axis), scanned over cell
 * offsets -m..m with m = ceil(rc / h); the image index of the neighbour cell
 * follows from floor division of the unwrapped cell index. */
static int neighbours_cells(int i, const double *wpos, const double *box, double rc,
                            const orc_cells *c, nb_buf *out) {
    out->n = 0;
    const double rc2 = rc * rc;
    int ci[3];
    for (int a = 0; a < 3; ++a) {
        ci[a] = (int)floor(wpos[3 * i + a] / c->h[a]);
        if (ci[a] >= c->nc[a]) ci[a] = c->nc[a] - 1;
        if (ci[a] < 0) ci[a] = 0;
    }
    int off[3];
    for (off[2] = -c->m[2]; off[2] <= c->m[2]; ++off[2])
        for (off[1] = -c->m[1]; off[1] <= c->m[1]; ++off[1])
            for (off[0] = -c->m[0]; off[0] <= c->m[0]; ++off[0]) {
                int cc[3], img[3];
                for (int a = 0; a < 3; ++a) {
                    int u = ci[a] + off[a];
                    int q = (int)floor((double)u / c->nc[a]);
                    img[a] = q;
                    cc[a] = u - q * c->nc[a];
                }
                int cell = (cc[2] * c->nc[1] + cc[1]) * c->nc[0] + cc[0];
                for (int p = c->start[cell]; p < c->start[cell + 1]; ++p) {
                    int j = c->atoms[p];
                    if (j == i && img[0] == 0 && img[1] == 0 && img[2] == 0) continue;
                    double d[3], r2 = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        d[a] = wpos[3 * j + a] + img[a] * box[a] - wpos[3 * i + a];
                        r2 += d[a] * d[a];
                    }
                    if (r2 > rc2) continue;
                    int e = nb_push(out, j, img, d, sqrt(r2));
                    if (e) return e;
                }
            }
    return ORC_OK;
}

static double *wrapped_copy(int n, const double *pos, const double *box) {
    double *w = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!w) return NULL;
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) w[3 * i + a] = wrap1(pos[3 * i + a], box[a]);
    return w;
}

/* Positions wrapped into the cell: each fractional coordinate into [0, 1). */
static double *wrapped_copy_box(int n, const double *pos, const orc_box *B) {
    if (!B->tilted) return wrapped_copy(n, pos, B->L);
    double *w = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!w) return NULL;
    for (int i = 0; i < n; ++i) {
        double s[3];
        to_fractional(B, pos + 3 * i, s);
        for (int a = 0; a < 3; ++a) s[a] = wrap1(s[a], 1.0);
        from_fractional(B, s, w + 3 * i);
    }
    return w;
}

/* Neighbour lists for tests: counts[i] (and, when out_j != NULL, the entries at
 * offsets[i]...) with image indices relative to the WRAPPED positions. */
int orc_neighbour_lists(int mode, int n, const double *pos, const double *box, double rc,
                        int *counts, const int64_t *offsets, int *out_j, int *out_img) {
    if (n < 0 || !pos || !box || rc <= 0.0 || !counts) return ORC_E_ARG;
    double *w = wrapped_copy(n, pos, box);
    if (!w) return ORC_E_NOMEM;
    orc_cells cells = {0};
    int err = ORC_OK;
    if (mode == 1) err = cells_build(&cells, n, w, box, rc);
    nb_buf b = {0};
    for (int i = 0; i < n && !err; ++i) {
        err = (mode == 1) ? neighbours_cells(i, w, box, rc, &cells, &b)
                          : neighbours_brute(i, n, w, box, rc, &b);
        if (err) break;
        counts[i] = b.n;
        if (out_j) {
            for (int k = 0; k < b.n; ++k) {
                out_j[offsets[i] + k] = b.v[k].j;
                for (int a = 0; a < 3; ++a) out_img[3 * (offsets[i] + k) + a] = b.v[k].img[a];
            }
        }
    }
    free(b.v);
    if (mode == 1) cells_free(&cells);
    free(w);
    return err;
}

/* ------------------------------------------------------------ per-atom pass */

typedef struct {
    nb_buf nb;
    double *G, *g, *dEdG, *acts, *dE_dd, *T, *dT;
    int *ang; /* indices of angular neighbours in nb */
    int ang_cap;
} orc_work;

static void work_free(orc_work *w) {
    free(w->nb.v);
    free(w->G);
    free(w->g);
    free(w->dEdG);
    free(w->acts);
    free(w->dE_dd);
    free(w->T);
    free(w->dT);
    free(w->ang);
    memset(w, 0, sizeof(*w));
}

static int work_init(orc_work *w, const orc_model *m) {
    memset(w, 0, sizeof(*w));
    int D = orc_D(m);
    int tot = 0, nmax = 1;
    for (int l = 0; l <= m->n_layers; ++l) {
        tot += m->widths[l];
        if (m->widths[l] > nmax) nmax = m->widths[l];
    }
    int ord = m->order_rad > m->order_ang ? m->order_rad : m->order_ang;
    w->G = (double *)malloc(sizeof(double) * D);
    w->g = (double *)malloc(sizeof(double) * D);
    w->dEdG = (double *)malloc(sizeof(double) * D);
    w->acts = (double *)malloc(sizeof(double) * (size_t)(2 * tot + 2 * nmax));
    w->T = (double *)malloc(sizeof(double) * (ord + 2));
    w->dT = (double *)malloc(sizeof(double) * (ord + 2));
    if (!w->G || !w->g || !w->dEdG || !w->acts || !w->T || !w->dT) {
        work_free(w);
        return ORC_E_NOMEM;
    }
    return ORC_OK;
}

/* Descriptor of atom i from its neighbour list (Eqs. radial, angular, the
 * weighted copy); fills w->G and the list of angular neighbours. */
static int descriptor(const orc_model *m, const int *types, orc_work *w) {
    const int Kr = m->order_rad + 1, Ka = m->order_ang + 1;
    double *rad = w->G, *ang = w->G + Kr, *radw = w->G + Kr + Ka, *angw = w->G + 2 * Kr + Ka;
    memset(w->G, 0, sizeof(double) * orc_D(m));
    if (w->ang_cap < w->nb.n) {
        int *na = (int *)realloc(w->ang, sizeof(int) * (size_t)w->nb.n);
        if (!na) return ORC_E_NOMEM;
        w->ang = na;
        w->ang_cap = w->nb.n;
    }
    int n_ang = 0;
    for (int p = 0; p < w->nb.n; ++p) {
        const orc_nb *e = &w->nb.v[p];
        if (e->r < 1e-8) return ORC_E_OVERLAP;
        double s = m->type_weight[types[e->j]];
        if (e->r <= m->rc_rad) {
            double fc = cutoff_fc(e->r, m->rc_rad);
            cheb_T(m->order_rad, 2.0 * e->r / m->rc_rad - 1.0, w->T);
            for (int a = 0; a < Kr; ++a) {
                rad[a] += w->T[a] * fc;
                radw[a] += s * w->T[a] * fc;
            }
        }
        if (e->r <= m->rc_ang) w->ang[n_ang++] = p;
    }
    for (int pa = 0; pa < n_ang; ++pa) {
        const orc_nb *ej = &w->nb.v[w->ang[pa]];
        double fj = cutoff_fc(ej->r, m->rc_ang), sj = m->type_weight[types[ej->j]];
        for (int pb = 0; pb < n_ang; ++pb) {
            if (pb == pa) continue; /* k != j as image-atoms; ordered pairs */
            const orc_nb *ek = &w->nb.v[w->ang[pb]];
            double fk = cutoff_fc(ek->r, m->rc_ang), sk = m->type_weight[types[ek->j]];
            double cth = (ej->d[0] * ek->d[0] + ej->d[1] * ek->d[1] + ej->d[2] * ek->d[2]) / (ej->r * ek->r);
            cheb_T(m->order_ang, cth, w->T);
            for (int a = 0; a < Ka; ++a) {
                ang[a] += w->T[a] * fj * fk;
                angw[a] += sj * sk * w->T[a] * fj * fk;
            }
        }
    }
    return n_ang;
}

/* Network of species t: forward (Eq. ANN-layer, tanh hidden, linear output),
 * then back-propagation of dE_i/dg; optional accumulation of dE/dW, dE/db. */
static double network(const orc_model *m, int t, orc_work *w, double *dEdW_t) {
    const int L = m->n_layers, D = orc_D(m);
    const double *P = m->params + (size_t)t * orc_nparams(m);
    const double *sh = m->in_shift ? m->in_shift + (size_t)t * D : NULL;
    const double *sc = m->in_scale ? m->in_scale + (size_t)t * D : NULL;
    /* activations x^0..x^L stored back to back */
    int off[64];
    off[0] = 0;
    for (int l = 1; l <= L; ++l) off[l] = off[l - 1] + m->widths[l - 1];
    double *x = w->acts;
    for (int k = 0; k < D; ++k) x[k] = (w->G[k] - (sh ? sh[k] : 0.0)) * (sc ? sc[k] : 1.0);
    const double *Wl = P;
    const double *Wptr[64];
    for (int l = 1; l <= L; ++l) {
        int no = m->widths[l], ni = m->widths[l - 1];
        const double *W = Wl, *b = Wl + (size_t)no * ni;
        Wptr[l] = W;
        for (int o = 0; o < no; ++o) {
            double z = b[o];
            for (int k = 0; k < ni; ++k) z += W[(size_t)o * ni + k] * x[off[l - 1] + k];
            x[off[l] + o] = (l < L) ? tanh(z) : z;
        }
        Wl = b + no;
    }
    double E = x[off[L]];
    /* back-propagation: delta^L = dE/dz^L = 1; two scratch vectors after x^L */
    int nmax = 1;
    for (int l = 0; l <= L; ++l)
        if (m->widths[l] > nmax) nmax = m->widths[l];
    double *dcur = w->acts + off[L] + m->widths[L], *dprev = dcur + nmax;
    dcur[0] = 1.0;
    size_t poff = 0;
    size_t lay_off[64];
    for (int l = 1; l <= L; ++l) {
        lay_off[l] = poff;
        poff += (size_t)m->widths[l] * m->widths[l - 1] + m->widths[l];
    }
    for (int l = L; l >= 1; --l) {
        int no = m->widths[l], ni = m->widths[l - 1];
        const double *W = Wptr[l];
        if (dEdW_t) {
            double *gW = dEdW_t + lay_off[l], *gb = gW + (size_t)no * ni;
            for (int o = 0; o < no; ++o) {
                gb[o] += dcur[o];
                for (int k = 0; k < ni; ++k) gW[(size_t)o * ni + k] += dcur[o] * x[off[l - 1] + k];
            }
        }
        for (int k = 0; k < ni; ++k) {
            double s = 0.0;
            for (int o = 0; o < no; ++o) s += W[(size_t)o * ni + k] * dcur[o];
            if (l - 1 >= 1) {
                double a = x[off[l - 1] + k];
                s *= (1.0 - a * a);
            }
            dprev[k] = s;
        }
        double *tmp = dcur;
        dcur = dprev;
        dprev = tmp;
    }
    /* dcur now holds dE/dg; dE/dG = dE/dg * scale */
    for (int k = 0; k < D; ++k) w->dEdG[k] = dcur[k] * (sc ? sc[k] : 1.0);
    return E;
}

/* dE_i/dd for every neighbour entry of atom i, from dE_i/dG. */
static void descriptor_grad(const orc_model *m, const int *types, orc_work *w, int n_ang) {
    const int Kr = m->order_rad + 1, Ka = m->order_ang + 1;
    const double *gr = w->dEdG, *ga = w->dEdG + Kr, *grw = w->dEdG + Kr + Ka, *gaw = w->dEdG + 2 * Kr + Ka;
    double *G3 = w->dE_dd;
    memset(G3, 0, sizeof(double) * 3 * (size_t)w->nb.n);
    for (int p = 0; p < w->nb.n; ++p) {
        const orc_nb *e = &w->nb.v[p];
        if (e->r > m->rc_rad) continue;
        double s = m->type_weight[types[e->j]];
        double x = 2.0 * e->r / m->rc_rad - 1.0;
        double fc = cutoff_fc(e->r, m->rc_rad), dfc = cutoff_dfc(e->r, m->rc_rad);
        cheb_T(m->order_rad, x, w->T);
        cheb_dT(m->order_rad, x, w->dT);
        double dEdr = 0.0;
        for (int a = 0; a < Kr; ++a) {
            double coef = gr[a] + s * grw[a];
            dEdr += coef * (w->dT[a] * (2.0 / m->rc_rad) * fc + w->T[a] * dfc);
        }
        for (int a = 0; a < 3; ++a) G3[3 * p + a] += dEdr * e->d[a] / e->r;
    }
    for (int pa = 0; pa < n_ang; ++pa) {
        int ij = w->ang[pa];
        const orc_nb *ej = &w->nb.v[ij];
        double fj = cutoff_fc(ej->r, m->rc_ang), dfj = cutoff_dfc(ej->r, m->rc_ang);
        double sj = m->type_weight[types[ej->j]];
        double uj[3] = {ej->d[0] / ej->r, ej->d[1] / ej->r, ej->d[2] / ej->r};
        for (int pb = 0; pb < n_ang; ++pb) {
            if (pb == pa) continue;
            int ik = w->ang[pb];
            const orc_nb *ek = &w->nb.v[ik];
            double fk = cutoff_fc(ek->r, m->rc_ang), dfk = cutoff_dfc(ek->r, m->rc_ang);
            double sk = m->type_weight[types[ek->j]];
            double uk[3] = {ek->d[0] / ek->r, ek->d[1] / ek->r, ek->d[2] / ek->r};
            double cth = uj[0] * uk[0] + uj[1] * uk[1] + uj[2] * uk[2];
            cheb_T(m->order_ang, cth, w->T);
            cheb_dT(m->order_ang, cth, w->dT);
            double S = 0.0, dS = 0.0;
            for (int a = 0; a < Ka; ++a) {
                double coef = ga[a] + sj * sk * gaw[a];
                S += coef * w->T[a];
                dS += coef * w->dT[a];
            }
            for (int a = 0; a < 3; ++a) {
                double dcos_dj = (uk[a] - cth * uj[a]) / ej->r;
                double dcos_dk = (uj[a] - cth * uk[a]) / ek->r;
                G3[3 * ij + a] += dS * fj * fk * dcos_dj + S * dfj * fk * uj[a];
                G3[3 * ik + a] += dS * fj * fk * dcos_dk + S * fj * dfk * uk[a];
            }
        }
    }
}

static int check_model(const orc_model *m) {
    if (!m || m->n_species < 1 || !m->type_weight || m->rc_rad <= 0.0 || m->rc_ang <= 0.0 ||
        m->order_rad < 0 || m->order_ang < 0 || m->n_layers < 1 || m->n_layers > 60 || !m->widths ||
        !m->params)
        return ORC_E_ARG;
    if (m->widths[0] != orc_D(m) || m->widths[m->n_layers] != 1) return ORC_E_ARG;
    return ORC_OK;
}

/*
 * Energy, forces, virial (and optionally per-atom energies, G, dE/dG, dE/dW)
 * of one periodic structure (orthorhombic, or a tilted restricted triclinic cell).
 *   mode        0 = brute-force neighbours, 1 = cell list
 *   center_mask NULL = every atom is a centre; else only atoms with mask != 0
 *               contribute E_i (and their force / virial terms)
 *   outputs     any may be NULL; forces [n*3], virial [9] row-major,
 *               e_atom [n], G and dEdG [n*D], dEdW [n_species*n_params]
 */
static int compute_box(const orc_model *m, int n, const double *pos, const int *types, const orc_box *B,
                       int mode, int n_threads, const unsigned char *center_mask, double *energy, double *e_atom,
                       double *forces, double *virial, double *G_out, double *dEdG_out, double *dEdW) {
    if (check_model(m) || n < 0 || (n > 0 && (!pos || !types))) return ORC_E_ARG;
    for (int a = 0; a < 3; ++a)
        if (!(B->L[a] > 0.0)) return ORC_E_ARG;
    if (!isfinite(B->xy) || !isfinite(B->xz) || !isfinite(B->yz)) return ORC_E_ARG;
    for (int i = 0; i < n; ++i)
        if (types[i] < 0 || types[i] >= m->n_species) return ORC_E_ARG;
    if (B->tilted) mode = 0; /* tilted cells: brute force only */
    const double *box = B->L;
    const int D = orc_D(m), NP = orc_nparams(m);
    const double rc = m->rc_rad > m->rc_ang ? m->rc_rad : m->rc_ang;
    double *w = wrapped_copy_box(n, pos, B);
    if (!w) return ORC_E_NOMEM;
    orc_cells cells = {0};
    if (mode == 1 && cells_build(&cells, n, w, box, rc)) {
        free(w);
        return ORC_E_NOMEM;
    }
    int nt = 1;
#ifdef _OPENMP
    nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#endif
    double *Fth = (double *)calloc((size_t)nt * 3 * (size_t)(n > 0 ? n : 1), sizeof(double));
    double *Wth = (double *)calloc((size_t)nt * 9, sizeof(double));
    double *Eth = (double *)calloc((size_t)nt, sizeof(double));
    double *gWth = dEdW ? (double *)calloc((size_t)nt * m->n_species * NP, sizeof(double)) : NULL;
    int err = ORC_OK;
    if (!Fth || !Wth || !Eth || (dEdW && !gWth)) err = ORC_E_NOMEM;

#pragma omp parallel num_threads(nt) if (nt > 1)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        orc_work wk;
        memset(&wk, 0, sizeof(wk));
        int lerr = err ? err : work_init(&wk, m);
        double *F = Fth ? Fth + (size_t)tid * 3 * n : NULL;
        double *V = Wth ? Wth + 9 * tid : NULL;
#pragma omp for schedule(dynamic, 16)
        for (int i = 0; i < n; ++i) {
            if (lerr) continue;
            if (center_mask && !center_mask[i]) {
                if (e_atom) e_atom[i] = 0.0;
                continue;
            }
            int e = (mode == 1)  ? neighbours_cells(i, w, box, rc, &cells, &wk.nb)
                    : B->tilted ? neighbours_brute_tri(i, n, w, B, rc, &wk.nb)
                                : neighbours_brute(i, n, w, box, rc, &wk.nb);
            if (e) {
                lerr = e;
                continue;
            }
            int n_ang = descriptor(m, types, &wk);
            if (n_ang < 0) {
                lerr = n_ang;
                continue;
            }
            double Ei = network(m, types[i], &wk, gWth ? gWth + ((size_t)tid * m->n_species + types[i]) * NP : NULL);
            Eth[tid] += Ei;
            if (e_atom) e_atom[i] = Ei;
            if (G_out) memcpy(G_out + (size_t)i * D, wk.G, sizeof(double) * D);
            if (dEdG_out) memcpy(dEdG_out + (size_t)i * D, wk.dEdG, sizeof(double) * D);
            if (forces || virial) {
                double *nd = (double *)realloc(wk.dE_dd, sizeof(double) * 3 * (size_t)(wk.nb.n > 0 ? wk.nb.n : 1));
                if (!nd) {
                    lerr = ORC_E_NOMEM;
                    continue;
                }
                wk.dE_dd = nd;
                descriptor_grad(m, types, &wk, n_ang);
                for (int p = 0; p < wk.nb.n; ++p) {
                    const orc_nb *q = &wk.nb.v[p];
                    const double *g3 = wk.dE_dd + 3 * p;
                    for (int a = 0; a < 3; ++a) {
                        /* d = x_j + nL - x_i: dE/dx_j = +g, dE/dx_i = -g; F = -dE/dx */
                        F[3 * q->j + a] -= g3[a];
                        F[3 * i + a] += g3[a];
                        for (int b = 0; b < 3; ++b) V[3 * a + b] -= q->d[a] * g3[b];
                    }
                }
            }
        }
#pragma omp critical
        {
            if (lerr && !err) err = lerr;
        }
        work_free(&wk);
    }
    if (!err) {
        double E = 0.0;
        for (int t = 0; t < nt; ++t) E += Eth[t];
        if (energy) *energy = E;
        if (forces) {
            for (size_t k = 0; k < 3 * (size_t)n; ++k) {
                double s = 0.0;
                for (int t = 0; t < nt; ++t) s += Fth[(size_t)t * 3 * n + k];
                forces[k] = s;
            }
        }
        if (virial) {
            for (int k = 0; k < 9; ++k) {
                double s = 0.0;
                for (int t = 0; t < nt; ++t) s += Wth[9 * t + k];
                virial[k] = s;
            }
        }
        if (dEdW) {
            for (size_t k = 0; k < (size_t)m->n_species * NP; ++k) {
                double s = 0.0;
                for (int t = 0; t < nt; ++t) s += gWth[(size_t)t * m->n_species * NP + k];
                dEdW[k] = s;
            }
        }
    }
    free(Fth);
    free(Wth);
    free(Eth);
    free(gWth);
    if (mode == 1) cells_free(&cells);
    free(w);
    return err;
}

int orc_compute(const orc_model *m, int n, const double *pos, const int *types, const double *box,
                int mode, int n_threads, const unsigned char *center_mask, double *energy, double *e_atom,
                double *forces, double *virial, double *G_out, double *dEdG_out, double *dEdW) {
    if (!box) return ORC_E_ARG;
    const orc_box B = box_of(box, NULL);
    return compute_box(m, n, pos, types, &B, mode, n_threads, center_mask, energy, e_atom, forces, virial, G_out,
                       dEdG_out, dEdW);
}

/* The same in a restricted triclinic cell: box = (L_x, L_y, L_z), tilt =
 * (xy, xz, yz); a tilted cell is evaluated by brute force whatever the mode. */
int orc_compute_tri(const orc_model *m, int n, const double *pos, const int *types, const double *box,
                    const double *tilt, int mode, int n_threads, double *energy, double *e_atom, double *forces,
                    double *virial, double *G_out) {
    if (!box || !tilt) return ORC_E_ARG;
    const orc_box B = box_of(box, tilt);
    return compute_box(m, n, pos, types, &B, mode, n_threads, NULL, energy, e_atom, forces, virial, G_out, NULL,
                       NULL);
}

/* Forces on a few target atoms only: every atom within the largest cutoff of a
 * target (any image) is a centre; the rest are skipped. */
int orc_forces_subset(const orc_model *m, int n, const double *pos, const int *types, const double *box,
                      int mode, int n_threads, int n_targets, const int *targets, double *forces_out,
                      double *e_atom_out) {
    if (check_model(m) || n <= 0 || n_targets < 0 || (n_targets > 0 && !targets) || !forces_out) return ORC_E_ARG;
    const double rc = m->rc_rad > m->rc_ang ? m->rc_rad : m->rc_ang;
    double *w = wrapped_copy(n, pos, box);
    unsigned char *mask = (unsigned char *)calloc((size_t)n, 1);
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *Ea = (double *)malloc(sizeof(double) * (size_t)n);
    if (!w || !mask || !F || !Ea) {
        free(w);
        free(mask);
        free(F);
        free(Ea);
        return ORC_E_NOMEM;
    }
    orc_cells cells = {0};
    int err = (mode == 1) ? cells_build(&cells, n, w, box, rc) : ORC_OK;
    nb_buf b = {0};
    for (int t = 0; t < n_targets && !err; ++t) {
        int i = targets[t];
        if (i < 0 || i >= n) {
            err = ORC_E_ARG;
            break;
        }
        mask[i] = 1;
        err = (mode == 1) ? neighbours_cells(i, w, box, rc, &cells, &b) : neighbours_brute(i, n, w, box, rc, &b);
        for (int k = 0; k < b.n && !err; ++k) mask[b.v[k].j] = 1;
    }
    free(b.v);
    if (mode == 1) cells_free(&cells);
    free(w);
    if (!err) err = orc_compute(m, n, pos, types, box, mode, n_threads, mask, NULL, Ea, F, NULL, NULL, NULL, NULL);
    if (!err) {
        for (int t = 0; t < n_targets; ++t) {
            for (int a = 0; a < 3; ++a) forces_out[3 * t + a] = F[3 * targets[t] + a];
            if (e_atom_out) e_atom_out[t] = Ea[targets[t]];
        }
    }
    free(mask);
    free(F);
    free(Ea);
    return err;
}

/*
 * Velocity-Verlet NVE (metal units): v += dt/2 F/m c; x += dt v; F(x);
 * v += dt/2 F/m c, with c = 9648.533212 (A/ps)^2 per eV/amu.
 * pos, vel updated in place; e_pot, e_kin [n_steps + 1] (frame 0 first).
 */
/* Velocity Verlet; with tau > 0 the Berendsen weak-coupling thermostat: at the
 * start of every step the velocities are scaled by
 *     lambda = sqrt(1 + (dt / tau) (T0 / T - 1)),   T = 2 E_kin / ((3N - 3) k_B),
 * E_kin being the kinetic energy recorded for the frame the step starts from
 * (the paper's MD cycle takes T as an input, Fig. 1; it names no thermostat). */
/* Berendsen barostat (isotropic; not in the paper, which runs its potential
 * inside LAMMPS): after every `every`-th step of a run, with the pressure of
 * that frame
 *     P = (2 E_kin + tr W) / (3 V)   (W the virial above, V = L_x L_y L_z),
 * positions and cell (edges and tilts) are scaled by
 *     mu = (1 - (every dt / tau) (P0 - P) / B)^(1/3),
 * B the bulk modulus, and the forces re-evaluated; the record of that frame is
 * the scaled state. Pressures in bar: 1 eV/A^3 = 1.602176634e6 bar. */
typedef struct {
    double P0, tau, modulus; /* bar, ps, bar */
    int every;
} orc_baro;

#define ORC_EV_A3_BAR 1.602176634e6

static int md_run(const orc_model *m, int n, double *pos, double *vel, const int *types,
                  const double *mass_of_type, orc_box *box, double dt, int n_steps, int mode,
                  int n_threads, double *e_pot, double *e_kin, double T0, double tau, const orc_baro *baro) {
    const double c = 9648.533212;
    const double kB = 8.617333262e-5;
    if (check_model(m) || n <= 0 || !pos || !vel || !mass_of_type || n_steps < 0) return ORC_E_ARG;
    if (baro && (baro->every < 1 || !(baro->tau > 0.0) || !(baro->modulus > 0.0))) return ORC_E_ARG;
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    if (!F) return ORC_E_NOMEM;
    double E = 0.0, W[9];
    int err = compute_box(m, n, pos, types, box, mode, n_threads, NULL, &E, NULL, F, W, NULL, NULL, NULL);
    for (int s = 0; s <= n_steps && !err; ++s) {
        double K = 0.0;
        for (int i = 0; i < n; ++i) {
            double mi = mass_of_type[types[i]];
            for (int a = 0; a < 3; ++a) K += 0.5 * mi * vel[3 * i + a] * vel[3 * i + a] / c;
        }
        if (e_pot) e_pot[s] = E;
        if (e_kin) e_kin[s] = K;
        if (s == n_steps) break;
        if (tau > 0.0) {
            const int dof = 3 * n - 3 > 0 ? 3 * n - 3 : 1;
            const double T = 2.0 * K / (dof * kB);
            const double l2 = T > 0.0 ? 1.0 + (dt / tau) * (T0 / T - 1.0) : 1.0;
            const double lambda = l2 > 0.0 ? sqrt(l2) : 0.0;
            for (int q = 0; q < 3 * n; ++q) vel[q] *= lambda;
        }
        for (int i = 0; i < n; ++i) {
            double k = 0.5 * dt * c / mass_of_type[types[i]];
            for (int a = 0; a < 3; ++a) {
                vel[3 * i + a] += k * F[3 * i + a];
                pos[3 * i + a] += dt * vel[3 * i + a];
            }
        }
        err = compute_box(m, n, pos, types, box, mode, n_threads, NULL, &E, NULL, F, W, NULL, NULL, NULL);
        if (err) break;
        for (int i = 0; i < n; ++i) {
            double k = 0.5 * dt * c / mass_of_type[types[i]];
            for (int a = 0; a < 3; ++a) vel[3 * i + a] += k * F[3 * i + a];
        }
        if (baro && (s + 1) % baro->every == 0) {
            double K1 = 0.0;
            for (int i = 0; i < n; ++i) {
                double mi = mass_of_type[types[i]];
                for (int a = 0; a < 3; ++a) K1 += 0.5 * mi * vel[3 * i + a] * vel[3 * i + a] / c;
            }
            const double V = box->L[0] * box->L[1] * box->L[2];
            const double P = (2.0 * K1 + W[0] + W[4] + W[8]) / (3.0 * V) * ORC_EV_A3_BAR;
            const double arg = 1.0 - (baro->every * dt / baro->tau) * (baro->P0 - P) / baro->modulus;
            if (!(arg > 0.0)) {
                err = ORC_E_ARG;
                break;
            }
            const double mu = cbrt(arg);
            for (int q = 0; q < 3 * n; ++q) pos[q] *= mu;
            for (int a = 0; a < 3; ++a) box->L[a] *= mu;
            box->xy *= mu;
            box->xz *= mu;
            box->yz *= mu;
            err = compute_box(m, n, pos, types, box, mode, n_threads, NULL, &E, NULL, F, W, NULL, NULL, NULL);
        }
    }
    free(F);
    return err;
}

int orc_md_nve(const orc_model *m, int n, double *pos, double *vel, const int *types,
               const double *mass_of_type, const double *box, double dt, int n_steps, int mode,
               int n_threads, double *e_pot, double *e_kin) {
    if (!box) return ORC_E_ARG;
    orc_box B = box_of(box, NULL);
    return md_run(m, n, pos, vel, types, mass_of_type, &B, dt, n_steps, mode, n_threads, e_pot, e_kin, 0.0, 0.0,
                  NULL);
}

int orc_md_nvt(const orc_model *m, int n, double *pos, double *vel, const int *types,
               const double *mass_of_type, const double *box, double dt, int n_steps, int mode,
               int n_threads, double *e_pot, double *e_kin, double T0, double tau) {
    if (!box) return ORC_E_ARG;
    orc_box B = box_of(box, NULL);
    return md_run(m, n, pos, vel, types, mass_of_type, &B, dt, n_steps, mode, n_threads, e_pot, e_kin, T0, tau,
                  NULL);
}

/* Velocity Verlet (tau > 0: with the Berendsen thermostat) in a restricted
 * triclinic cell: box = (L_x, L_y, L_z), tilt = (xy, xz, yz). */
int orc_md_tri(const orc_model *m, int n, double *pos, double *vel, const int *types, const double *mass_of_type,
               const double *box, const double *tilt, double dt, int n_steps, int n_threads, double *e_pot,
               double *e_kin, double T0, double tau) {
    if (!box || !tilt) return ORC_E_ARG;
    orc_box B = box_of(box, tilt);
    return md_run(m, n, pos, vel, types, mass_of_type, &B, dt, n_steps, 0, n_threads, e_pot, e_kin, T0, tau, NULL);
}

/* Velocity Verlet with the Berendsen barostat (and, tau_T > 0, the Berendsen
 * thermostat) in an orthorhombic or restricted triclinic cell; box [3] and
 * tilt [3] are updated in place to the final cell. */
int orc_md_npt(const orc_model *m, int n, double *pos, double *vel, const int *types, const double *mass_of_type,
               double *box, double *tilt, double dt, int n_steps, int n_threads, double *e_pot, double *e_kin,
               double T0, double tau_T, double P0, double tau_P, double modulus, int every) {
    if (!box || !tilt) return ORC_E_ARG;
    orc_box B = box_of(box, tilt);
    const orc_baro baro = {P0, tau_P, modulus, every};
    /* the cell list needs a fixed orthorhombic cell: brute force throughout */
    int err = md_run(m, n, pos, vel, types, mass_of_type, &B, dt, n_steps, 0, n_threads, e_pot, e_kin, T0, tau_T,
                     &baro);
    for (int a = 0; a < 3; ++a) box[a] = B.L[a];
    tilt[0] = B.xy;
    tilt[1] = B.xz;
    tilt[2] = B.yz;
    return err;
}

/* Test hooks: the basis pieces on their own. */
void orc_chebyshev(int n, double x, double *T, double *dT) {
    cheb_T(n, x, T);
    cheb_dT(n, x, dT);
}

void orc_cutoff(double r, double rc, double *fc_dfc) {
    fc_dfc[0] = cutoff_fc(r, rc);
    fc_dfc[1] = cutoff_dfc(r, rc);
}
