/*
 * CPU oracle for the short-range particle-particle force path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header or constant with the CUDA path.
 *
 * Everything here is the plain definition, written to be checked by eye:
 *
 *   a_i = sum_{j != i, s_ij < r_c^2} m_j f_SR(s_ij) d_ij,
 *   f_SR(s) = (s + eps)^(-3/2) - poly(s),  poly(s) = sum_k c_k s^k,
 *
 * (Eq. 7 of the paper, the short-range kernel; s = r.r; the cutoff test is
 * folded into the pair loop as in the paper's discussion of the select
 * instruction, Sec. III), with d_ij = x_j - x_i taken as the minimum periodic
 * image, evaluated in float64 by brute force over all j.  Positions and masses
 * are float64 arrays (float32 inputs widened, or a float64 trajectory).
 *
 * The chaining-mesh binning reference follows the float32 expression sequence
 * that defines a particle's cell (the build's reading of the paper's spatial
 * partition, Sec. III: a mesh replaces the RCB tree): wrap into [0, L), cell
 * index per axis, offset from the cell's centre (c + 1/2) w.  Each step is a
 * single IEEE float32
 * operation with round-to-nearest; this file must be compiled with
 * -ffp-contract=off so that no step is fused.
 *
 * Compile: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int ora_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Chaining mesh geometry                                                    */
/* ------------------------------------------------------------------------ */

/* n = floor(L / cell_min) cells per side (float64 quotient); w = L / n and
 * inv_w = n / L, each one float32 division. */
void ora_mesh(float L, float cell_min, int32_t *n_out, float *w_out, float *inv_w_out)
{
    int32_t n = (int32_t)floor((double)L / (double)cell_min);
    float nf = (float)n;
    *n_out = n;
    *w_out = L / nf;
    *inv_w_out = nf / L;
}

/* Wrap one float32 coordinate into [0, L): q = floor(x / L); x - q L; then one
 * correction step for the two rounding edge cases. */
static float wrap32(float x, float L)
{
    float q = floorf(x / L);
    float ql = q * L;
    float xw = x - ql;
    if (xw < 0.0f) xw = xw + L;
    if (xw >= L) xw = xw - L;
    return xw;
}

static int32_t cell1(float xw, float inv_w, int32_t n);

/* The same wrap of a float64 position x + d (displacement mode). */
static double wrap64(double p, double L)
{
    double q = floor(p / L);
    double ql = q * L;
    double pw = p - ql;
    if (pw < 0.0) pw = pw + L;
    if (pw >= L) pw = pw - L;
    return pw;
}

static int32_t cell64(double pw, float inv_w, int32_t n)
{
    double t = pw * (double)inv_w;
    int32_t c = (int32_t)floor(t);
    if (c > n - 1) c = n - 1;
    if (c < 0) c = 0;
    return c;
}

/* Cell coordinate and offset from the cell centre ctr = fl32((c + 1/2) w) of
 * one coordinate: float32 steps for an absolute position; with a
 * displacement d (non-NULL), the position x + d is formed and wrapped in
 * float64 and only the offset is rounded. */
static int32_t axis_cell(float x, const float *d, int64_t i, float L, int32_t n, float w, float inv_w,
                         float *o)
{
    if (!d) {
        float xw = wrap32(x, L);
        int32_t c = cell1(xw, inv_w, n);
        float ctr = ((float)c + 0.5f) * w;
        *o = xw - ctr;
        return c;
    }
    double pw = wrap64((double)x + (double)d[i], (double)L);
    int32_t c = cell64(pw, inv_w, n);
    float ctr = ((float)c + 0.5f) * w;
    *o = (float)(pw - (double)ctr);
    return c;
}

static int32_t cell1(float xw, float inv_w, int32_t n)
{
    float t = xw * inv_w;
    int32_t c = (int32_t)floorf(t);
    if (c > n - 1) c = n - 1;
    if (c < 0) c = 0;
    return c;
}

/* Binning of one volume.  Outputs: cell_of[i] (cell of particle i), counts per
 * cell, and the stable order: perm[k] = original index of the particle in
 * sorted slot k, particles ordered by cell and, within a cell, by original
 * index.  sorted4[4k..4k+3] = (ox, oy, oz, m) with o the offset from the
 * cell centre (float32).  dx, dy, dz: optional displacements (all NULL for absolute
 * positions).  cell_start has n^3 + 1 entries.  Returns 0. */
int ora_bin(const float *x, const float *y, const float *z, const float *dx, const float *dy,
            const float *dz, const float *m, int64_t N, float L, int32_t n, float w, float inv_w,
            int32_t *cell_of, int32_t *cell_start, int32_t *perm, float *sorted4)
{
    int64_t nc = (int64_t)n * n * n;
    int64_t *cnt = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    float *off = (float *)malloc((size_t)(N > 0 ? N : 1) * 3 * sizeof(float));
    if (!cnt || !off) {
        free(cnt);
        free(off);
        return -1;
    }
    for (int64_t i = 0; i < N; ++i) {
        int32_t cx = axis_cell(x[i], dx, i, L, n, w, inv_w, &off[3 * i + 0]);
        int32_t cy = axis_cell(y[i], dy, i, L, n, w, inv_w, &off[3 * i + 1]);
        int32_t cz = axis_cell(z[i], dz, i, L, n, w, inv_w, &off[3 * i + 2]);
        int32_t c = (cz * n + cy) * n + cx;
        cell_of[i] = c;
        cnt[c] += 1;
    }
    int64_t run = 0;
    for (int64_t c = 0; c < nc; ++c) {
        cell_start[c] = (int32_t)run;
        run += cnt[c];
        cnt[c] = cell_start[c]; /* becomes the fill cursor */
    }
    cell_start[nc] = (int32_t)run;
    /* visiting particles in index order makes the placement stable */
    for (int64_t i = 0; i < N; ++i) {
        int64_t k = cnt[cell_of[i]]++;
        perm[k] = (int32_t)i;
        sorted4[4 * k + 0] = off[3 * i + 0];
        sorted4[4 * k + 1] = off[3 * i + 1];
        sorted4[4 * k + 2] = off[3 * i + 2];
        sorted4[4 * k + 3] = m[i];
    }
    free(cnt);
    free(off);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Cell-pair interaction lists                                              */
/* ------------------------------------------------------------------------ */

/* Stencil reach: offsets with |delta_a| <= R, R = ceil(r_c / w). */
int32_t ora_reach(float w, float rcut)
{
    return (int32_t)ceil((double)rcut / (double)w);
}

/* Two cells whose integer offsets are delta can hold a pair closer than r_c
 * iff the minimum distance between the boxes is below r_c:
 * sum_a max(0, |delta_a| - 1)^2 w^2 < r_c^2, in float64. */
static int cells_within(int dx, int dy, int dz, double w, double rc)
{
    double gx = abs(dx) > 1 ? (double)(abs(dx) - 1) : 0.0;
    double gy = abs(dy) > 1 ? (double)(abs(dy) - 1) : 0.0;
    double gz = abs(dz) > 1 ? (double)(abs(dz) - 1) : 0.0;
    return (gx * gx + gy * gy + gz * gz) * w * w < rc * rc;
}

/* Per-cell neighbour lists of one volume, canonical order: for cell c
 * (ascending), offsets (dz, dy, dx) ascending lexicographically over
 * [-R, R]^3 restricted to cells_within.  Each entry: neighbour cell id and a
 * periodic shift code (sz+1)*9 + (sy+1)*3 + (sx+1), s_a in {-1, 0, 1} the
 * image of the neighbour along axis a.  nbr_off has n^3 + 1 entries.  When
 * nbr_cell is NULL only the counts are produced.  Returns the entry count,
 * or -1 if the mesh is too coarse for a unique image (n < 2R + 1). */
int64_t ora_lists(int32_t n, float w, float rcut, int64_t *nbr_off, int32_t *nbr_cell,
                  int8_t *nbr_shift)
{
    int32_t R = ora_reach(w, rcut);
    if (n < 2 * R + 1) return -1;
    int64_t nc = (int64_t)n * n * n;
    int64_t e = 0;
    for (int64_t c = 0; c < nc; ++c) {
        int32_t cx = (int32_t)(c % n), cy = (int32_t)((c / n) % n), cz = (int32_t)(c / ((int64_t)n * n));
        if (nbr_off) nbr_off[c] = e;
        for (int dz = -R; dz <= R; ++dz)
            for (int dy = -R; dy <= R; ++dy)
                for (int dx = -R; dx <= R; ++dx) {
                    if (!cells_within(dx, dy, dz, (double)w, (double)rcut)) continue;
                    int32_t px = cx + dx, py = cy + dy, pz = cz + dz;
                    int sx = 0, sy = 0, sz = 0;
                    if (px < 0) { px += n; sx = -1; } else if (px >= n) { px -= n; sx = 1; }
                    if (py < 0) { py += n; sy = -1; } else if (py >= n) { py -= n; sy = 1; }
                    if (pz < 0) { pz += n; sz = -1; } else if (pz >= n) { pz -= n; sz = 1; }
                    if (nbr_cell) {
                        nbr_cell[e] = (pz * n + py) * n + px;
                        nbr_shift[e] = (int8_t)((sz + 1) * 9 + (sy + 1) * 3 + (sx + 1));
                    }
                    ++e;
                }
    }
    if (nbr_off) nbr_off[nc] = e;
    return e;
}

/* Work items: each cell's particle range cut into consecutive chunks of at
 * most T particles, cells ascending.  Each task: (cell, begin, end) in sorted
 * slots.  Returns the task count (tasks may be NULL to count). */
int64_t ora_tasks(const int32_t *cell_start, int64_t ncells, int32_t T, int32_t *tasks3)
{
    int64_t t = 0;
    for (int64_t c = 0; c < ncells; ++c) {
        int32_t b = cell_start[c], e = cell_start[c + 1];
        for (int32_t i = b; i < e; i += T) {
            if (tasks3) {
                tasks3[3 * t + 0] = (int32_t)c;
                tasks3[3 * t + 1] = i;
                tasks3[3 * t + 2] = (i + T < e) ? i + T : e;
            }
            ++t;
        }
    }
    return t;
}

/* ------------------------------------------------------------------------ */
/* Recursive coordinate bisection (RCB) tree with fat leaves                 */
/* ------------------------------------------------------------------------ */

/* The paper's short-range tree (Sec. III, spatial locality): divide a group
 * of particles in two at the centre of mass along the longest side of its
 * box, keep each half in its own contiguous range, recurse until a leaf holds
 * at most leaf_max particles.  Exact integer version of that rule, so the
 * tree is reproducible bit for bit: per axis q = floor(xw 2^21 / L) in
 * [0, 2^21) (xw the float32-wrapped coordinate, the product in float64); the
 * box is the integer min/max of q; the split axis is the longest side (lowest
 * axis on ties); the split value is the floor of the integer mean of q (the
 * centre of mass of equal-mass particles); a particle goes left iff
 * q <= split; the partition is stable.  If every side has length 0 the first
 * half (cnt / 2 particles, by position) goes left.  A group becomes a leaf
 * when it holds at most leaf_max particles or sits at depth max_depth (the
 * roots have depth 0).  Leaves come out in depth-first, left-first order,
 * which is the order of their first slots. */
#define ORA_QBITS 21

static int32_t quant21(float xw, float L)
{
    double t = (double)xw * ((double)(1 << ORA_QBITS) / (double)L);
    int64_t q = (int64_t)floor(t);
    if (q > (1 << ORA_QBITS) - 1) q = (1 << ORA_QBITS) - 1;
    if (q < 0) q = 0;
    return (int32_t)q;
}

typedef struct {
    int32_t *q;    /* [3 N] quantised coordinates in current order */
    int32_t *idx;  /* [N] original index in current order */
    int32_t *tmp;  /* [4 N] scratch */
    int32_t leaf_max;
    int32_t max_depth;
    int64_t n_leaves;
    int32_t *leaf_start; /* appended */
    int32_t *leaf_qbox;  /* appended: 6 per leaf (lo xyz, hi xyz) */
} ora_rcb_state;

static void rcb_split(ora_rcb_state *S, int64_t b, int64_t e, int32_t depth)
{
    int64_t cnt = e - b;
    if (cnt <= 0) return; /* never reached by the rule above (both halves are non-empty) */
    int32_t lo[3], hi[3];
    int64_t sum[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) {
        lo[a] = S->q[3 * b + a];
        hi[a] = S->q[3 * b + a];
    }
    for (int64_t i = b; i < e; ++i)
        for (int a = 0; a < 3; ++a) {
            int32_t v = S->q[3 * i + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
            sum[a] += v;
        }
    if (cnt <= S->leaf_max || depth >= S->max_depth) {
        int64_t l = S->n_leaves++;
        S->leaf_start[l] = (int32_t)b;
        for (int a = 0; a < 3; ++a) {
            S->leaf_qbox[6 * l + a] = lo[a];
            S->leaf_qbox[6 * l + 3 + a] = hi[a];
        }
        return;
    }
    int axis = 0;
    for (int a = 1; a < 3; ++a)
        if (hi[a] - lo[a] > hi[axis] - lo[axis]) axis = a;
    int64_t nl = 0;
    if (hi[axis] == lo[axis]) {
        nl = cnt / 2; /* coincident: split by position */
    } else {
        int64_t split = sum[axis] / cnt; /* floor of the mean (non-negative) */
        /* stable partition through the scratch array */
        int64_t w = 0;
        for (int64_t pass = 0; pass < 2; ++pass)
            for (int64_t i = b; i < e; ++i) {
                int left = S->q[3 * i + axis] <= split;
                if ((pass == 0) == (left != 0)) {
                    for (int a = 0; a < 3; ++a) S->tmp[4 * w + a] = S->q[3 * i + a];
                    S->tmp[4 * w + 3] = S->idx[i];
                    ++w;
                    if (pass == 0) ++nl;
                }
            }
        for (int64_t k = 0; k < cnt; ++k) {
            for (int a = 0; a < 3; ++a) S->q[3 * (b + k) + a] = S->tmp[4 * k + a];
            S->idx[b + k] = S->tmp[4 * k + 3];
        }
    }
    rcb_split(S, b, b + nl, depth + 1);
    rcb_split(S, b + nl, e, depth + 1);
}

/* RCB of one volume.  Outputs (capacity N + 1 leaves): perm[k] = original
 * index at tree slot k; leaf_start[0..n_leaves] (leaf_start[n_leaves] = N);
 * leaf_qbox[6 l..6 l + 5] the leaf's integer box; sorted4 = (o, m) with
 * o = xw - origin rounded once to float32 (float64 difference), origin =
 * float32 of qlo L / 2^21 (the leaf's conservative lower corner).  Returns the
 * number of leaves, or -1 on allocation failure. */
int64_t ora_rcb_build(const float *x, const float *y, const float *z, const float *m, int64_t N, float L,
                      int32_t leaf_max, int32_t max_depth, int32_t *perm, int32_t *leaf_start, int32_t *leaf_qbox, float *sorted4)
{
    ora_rcb_state S;
    S.q = (int32_t *)malloc((size_t)(N > 0 ? N : 1) * 3 * sizeof(int32_t));
    S.idx = (int32_t *)malloc((size_t)(N > 0 ? N : 1) * sizeof(int32_t));
    S.tmp = (int32_t *)malloc((size_t)(N > 0 ? N : 1) * 4 * sizeof(int32_t));
    if (!S.q || !S.idx || !S.tmp) {
        free(S.q);
        free(S.idx);
        free(S.tmp);
        return -1;
    }
    for (int64_t i = 0; i < N; ++i) {
        S.q[3 * i + 0] = quant21(wrap32(x[i], L), L);
        S.q[3 * i + 1] = quant21(wrap32(y[i], L), L);
        S.q[3 * i + 2] = quant21(wrap32(z[i], L), L);
        S.idx[i] = (int32_t)i;
    }
    S.leaf_max = leaf_max;
    S.max_depth = max_depth;
    S.n_leaves = 0;
    S.leaf_start = leaf_start;
    S.leaf_qbox = leaf_qbox;
    if (N > 0) rcb_split(&S, 0, N, 0);
    leaf_start[S.n_leaves] = (int32_t)N;
    double scale = (double)L / (double)(1 << ORA_QBITS);
    for (int64_t l = 0; l < S.n_leaves; ++l) {
        float org[3];
        for (int a = 0; a < 3; ++a) org[a] = (float)((double)leaf_qbox[6 * l + a] * scale);
        for (int64_t k = leaf_start[l]; k < leaf_start[l + 1]; ++k) {
            int32_t i = S.idx[k];
            perm[k] = i;
            sorted4[4 * k + 0] = (float)((double)wrap32(x[i], L) - (double)org[0]);
            sorted4[4 * k + 1] = (float)((double)wrap32(y[i], L) - (double)org[1]);
            sorted4[4 * k + 2] = (float)((double)wrap32(z[i], L) - (double)org[2]);
            sorted4[4 * k + 3] = m[i];
        }
    }
    free(S.q);
    free(S.idx);
    free(S.tmp);
    return S.n_leaves;
}

/* Leaf interaction lists of one volume (the tree walk's result, by brute
 * force over leaf pairs): leaf j with image shift s is listed for leaf i iff
 * their boxes come closer than r_c:
 *   sum_a max(0, lo_j,a + s_a L - hi_i,a, lo_i,a - hi_j,a - s_a L)^2 < r_c^2
 * in float64, each leaf box widened by one grid quantum q_L = L / 2^21 on
 * every side, [(qlo - 1) q_L, (qhi + 2) q_L], so that it holds its particles
 * whatever the rounding of the quantisation.  Canonical order per i:
 * ascending shift code (sz+1)*9 + (sy+1)*3 + (sx+1), then ascending j.
 * For the leaves `targets` (NULL: every leaf), nbr_off[count + 1]; entries
 * (j, code) when nbr_leaf != NULL.  Returns the entry count. */
int64_t ora_rcb_lists(int64_t n_leaves, const int32_t *leaf_qbox, float L, float rcut, const int64_t *targets,
                      int64_t n_targets, int64_t *nbr_off, int32_t *nbr_leaf, int8_t *nbr_shift)
{
    double scale = (double)L / (double)(1 << ORA_QBITS);
    double rc2 = (double)rcut * (double)rcut;
    int64_t e = 0;
    int64_t n_i = targets ? n_targets : n_leaves;
    for (int64_t t = 0; t < n_i; ++t) {
        int64_t i = targets ? targets[t] : t;
        if (nbr_off) nbr_off[t] = e;
        for (int code = 0; code < 27; ++code) {
            int sx = code % 3 - 1, sy = (code / 3) % 3 - 1, sz = code / 9 - 1;
            int sh[3] = {sx, sy, sz};
            for (int64_t j = 0; j < n_leaves; ++j) {
                double d2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    double ilo = (double)(leaf_qbox[6 * i + a] - 1) * scale;
                    double ihi = (double)(leaf_qbox[6 * i + 3 + a] + 2) * scale;
                    double jlo = (double)(leaf_qbox[6 * j + a] - 1) * scale + (double)sh[a] * (double)L;
                    double jhi = (double)(leaf_qbox[6 * j + 3 + a] + 2) * scale + (double)sh[a] * (double)L;
                    double g = 0.0;
                    if (jlo - ihi > g) g = jlo - ihi;
                    if (ilo - jhi > g) g = ilo - jhi;
                    d2 += g * g;
                }
                if (d2 < rc2) {
                    if (nbr_leaf) {
                        nbr_leaf[e] = (int32_t)j;
                        nbr_shift[e] = (int8_t)code;
                    }
                    ++e;
                }
            }
        }
    }
    if (nbr_off) nbr_off[n_i] = e;
    return e;
}

/* ------------------------------------------------------------------------ */
/* Short-range force (Eq. 7), brute force in float64                         */
/* ------------------------------------------------------------------------ */

static double min_image(double d, double L)
{
    return d - L * nearbyint(d / L);
}

static double poly5(const double *c, double s)
{
    return c[0] + s * (c[1] + s * (c[2] + s * (c[3] + s * (c[4] + s * c[5]))));
}

static double dpoly5(const double *c, double s)
{
    return c[1] + s * (2.0 * c[2] + s * (3.0 * c[3] + s * (4.0 * c[4] + s * 5.0 * c[5])));
}

/* f_SR(s) = (s + eps)^-3/2 - poly(s) */
double ora_fsr(double s, double eps, const double *c)
{
    return pow(s + eps, -1.5) - poly5(c, s);
}

/* f_SR'(s) = -3/2 (s + eps)^-5/2 - poly'(s) */
double ora_dfsr(double s, double eps, const double *c)
{
    return -1.5 * pow(s + eps, -2.5) - dpoly5(c, s);
}

/* Accelerations of the S target particles targets[0..S-1] from all N
 * particles of one periodic box of side L. */
void ora_sr_force(const double *x, const double *y, const double *z, const double *m, int64_t N,
                  double L, double eps, double rcut, const double *c,
                  const int64_t *targets, int64_t S, double *ax, double *ay, double *az)
{
    double rc2 = rcut * rcut;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < S; ++t) {
        int64_t i = targets[t];
        double xi = x[i], yi = y[i], zi = z[i];
        double sx = 0.0, sy = 0.0, sz = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double dx = min_image(x[j] - xi, L);
            double dy = min_image(y[j] - yi, L);
            double dz = min_image(z[j] - zi, L);
            double s = dx * dx + dy * dy + dz * dz;
            if (!(s < rc2)) continue;
            double g = m[j] * ora_fsr(s, eps, c);
            sx += g * dx;
            sy += g * dy;
            sz += g * dz;
        }
        ax[t] = sx;
        ay[t] = sy;
        az[t] = sz;
    }
}

/* Short-range pair potential: the integral of the force law that vanishes at
 * the cutoff.  With P(s) = sum_k c_k s^(k+1) / (k+1) (so P' = poly):
 *   V(s) = [(r_c^2 + eps)^-1/2 + P(r_c^2)/2] - [(s + eps)^-1/2 + P(s)/2],
 * dV/ds = f_SR(s)/2, hence -grad_i of sum_{pairs} m_i m_j V = m_i a_i. */
static double P6(const double *c, double s)
{
    return s * (c[0] + s * (c[1] / 2.0 + s * (c[2] / 3.0 + s * (c[3] / 4.0 + s * (c[4] / 5.0 + s * c[5] / 6.0)))));
}

double ora_pair_potential(double s, double eps, double rcut, const double *c)
{
    double rc2 = rcut * rcut;
    return (1.0 / sqrt(rc2 + eps) + 0.5 * P6(c, rc2)) - (1.0 / sqrt(s + eps) + 0.5 * P6(c, s));
}

/* phi_i = sum_{j != i, s_ij < r_c^2} m_j V(s_ij) for the S targets. */
void ora_sr_potential(const double *x, const double *y, const double *z, const double *m, int64_t N,
                      double L, double eps, double rcut, const double *c, const int64_t *targets,
                      int64_t S, double *phi)
{
    double rc2 = rcut * rcut;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < S; ++t) {
        int64_t i = targets[t];
        double acc = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double dx = min_image(x[j] - x[i], L);
            double dy = min_image(y[j] - y[i], L);
            double dz = min_image(z[j] - z[i], L);
            double s = dx * dx + dy * dy + dz * dz;
            if (!(s < rc2)) continue;
            acc += m[j] * ora_pair_potential(s, eps, rcut, c);
        }
        phi[t] = acc;
    }
}

/* Number of ordered pairs (i, j), j != i, with s_ij < r_c^2. */
int64_t ora_pair_count(const double *x, const double *y, const double *z, int64_t N,
                       double L, double rcut, const int64_t *targets, int64_t S)
{
    double rc2 = rcut * rcut;
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
    for (int64_t t = 0; t < S; ++t) {
        int64_t i = targets[t];
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double dx = min_image(x[j] - x[i], L);
            double dy = min_image(y[j] - y[i], L);
            double dz = min_image(z[j] - z[i], L);
            if (dx * dx + dy * dy + dz * dz < rc2) total += 1;
        }
    }
    return total;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the force (vector-Jacobian product), float64                   */
/* ------------------------------------------------------------------------ */

/* Given the cotangent lam_k = dL/da_k of every particle's acceleration,
 * returns for each target i:
 *   dL/dx_i = sum_j [ m_i J(d_ij) lam_j - m_j J(d_ij) lam_i ],
 *   J(d) = f(s) I + 2 f'(s) d d^T   (the Jacobian of f(d.d) d),
 * because x_i enters a_i through every d_ij = x_j - x_i (sign -) and every a_j
 * through d_ji = x_i - x_j (sign +, J even in d).  And
 *   dL/dm_i = sum_j lam_j . f(s_ij) d_ji,
 * because m_i multiplies its pair term in every a_j.  Pairs beyond the cutoff
 * contribute nothing (the step at r_c is not differentiated). */
void ora_sr_force_adjoint(const double *x, const double *y, const double *z, const double *m,
                          int64_t N, double L, double eps, double rcut, const double *c,
                          const double *lx, const double *ly, const double *lz,
                          const int64_t *targets, int64_t S,
                          double *gx, double *gy, double *gz, double *gm)
{
    double rc2 = rcut * rcut;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < S; ++t) {
        int64_t i = targets[t];
        double xi = x[i], yi = y[i], zi = z[i], mi = m[i];
        double li[3] = {lx[i], ly[i], lz[i]};
        double g[3] = {0.0, 0.0, 0.0}, gmi = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double d[3];
            d[0] = min_image(x[j] - xi, L);
            d[1] = min_image(y[j] - yi, L);
            d[2] = min_image(z[j] - zi, L);
            double s = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(s < rc2)) continue;
            double f = ora_fsr(s, eps, c);
            double fp = ora_dfsr(s, eps, c);
            double mj = m[j];
            double lj[3] = {lx[j], ly[j], lz[j]};
            double dlj = d[0] * lj[0] + d[1] * lj[1] + d[2] * lj[2];
            double dli = d[0] * li[0] + d[1] * li[1] + d[2] * li[2];
            for (int a = 0; a < 3; ++a) {
                double Jlj = f * lj[a] + 2.0 * fp * d[a] * dlj; /* J(d) lam_j */
                double Jli = f * li[a] + 2.0 * fp * d[a] * dli; /* J(d) lam_i */
                g[a] += mi * Jlj - mj * Jli;
            }
            /* d_ji = -d_ij */
            gmi += -f * dlj;
        }
        gx[t] = g[0];
        gy[t] = g[1];
        gz[t] = g[2];
        if (gm) gm[t] = gmi;
    }
}

/* ------------------------------------------------------------------------ */
/* Kick and drift (the kick/stream maps of Eq. 6's symplectic step)           */
/* ------------------------------------------------------------------------ */

/* v <- v + dt_k a ; then, if x != NULL, x <- x + dt_d v (with the new v),
 * all in float64 on float64 arrays; no wrapping. */
void ora_kick_drift(int64_t N, double *vx, double *vy, double *vz,
                    const double *ax, const double *ay, const double *az, double dt_k,
                    double *x, double *y, double *z, double dt_d)
{
    for (int64_t i = 0; i < N; ++i) {
        vx[i] += dt_k * ax[i];
        vy[i] += dt_k * ay[i];
        vz[i] += dt_k * az[i];
        if (x) {
            x[i] += dt_d * vx[i];
            y[i] += dt_d * vy[i];
            z[i] += dt_d * vz[i];
        }
    }
}
