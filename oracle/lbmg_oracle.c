/*
 * lbmg_oracle.c -- plain, slow, FP64 CPU oracle for the connectivity-aware
 * multi-level finite-element system of Chuang & Kazhdan,
 * "A Connectivity-Aware Multi-level Finite-Element System for Solving
 * Laplace-Beltrami Equations" (arXiv 1505.03615).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or helper with the GPU library; it is written to be checked against
 * the paper by eye, not to be fast.
 *
 * What it computes, in the paper's order:
 *   - the restricted trilinear B-spline space on a regular grid of depth d
 *     (Section 3.2, Definitions 1-2): hat functions b_k at grid corners k whose
 *     support (the 2x2x2 voxels around k) meets the mesh;
 *   - the connectivity-aware split (Section 4.1 Definition 3, Section 4.2):
 *     one function b_k^i per connected component C_k^i of supp(b_k) /\ M;
 *   - the prolongation between successive grids (Section 4.3, Eq. 4) with the
 *     indicator chi(C_k^i, C_k'^i') and the trilinear refinement stencil;
 *   - the Galerkin matrices M_ij = int b_i b_j and
 *     L_ij = int <grad_M b_i, grad_M b_j> (Eq. 2 and Section 5.1), by exact
 *     quadrature over the pieces of each triangle cut by the voxel grid;
 *   - the right-hand side int f b_i for f linear on each triangle (Section 5.2);
 *   - a multigrid V-cycle with lexicographic Gauss-Seidel smoothing
 *     (Sections 4.3 and 5.2) and a dense Cholesky solve on the coarsest grid
 *     with the eps*Id regularisation of the Discussion in Section 5;
 *   - general cycles (orc_cycles): V or W (two coarse visits per level, the
 *     cycle of the convergence experiment of Section 5.2), Gauss-Seidel by
 *     corner-parity colour or lexicographic, the coarsest grid solved or
 *     relaxed like the others (the minimum-depth sweep of Section 5.2).
 *
 * Readings where the paper is silent or inconsistent (each also listed in
 * the design notes):
 *   - sign of L: the positive semi-definite form +int <grad b_i, grad b_j>
 *     is used, so that M + t L is symmetric positive definite (Eq. 2 prints
 *     the negative form; the systems of Sections 5.2-5.3 need the positive one);
 *   - refinement stencil: the trilinear hat refines with the 1D stencil
 *     1/2 (1 2 1) (Section 3.2 prints 1/4 (1 3 3 1), the quadratic B-spline's);
 *   - connectivity: two triangles of supp(b_k) /\ M are joined when they share
 *     a mesh edge whose segment meets the open support cube, or a mesh vertex
 *     strictly inside it (Section 4.2 leaves "connected component" to the
 *     reader);
 *   - embedding: the bounding box is centred in a cube of side 1.1 times its
 *     largest extent; computations use finest-grid units (voxel side 1 at the
 *     finest depth) and M and the right-hand side are scaled back to physical
 *     area;
 *   - fragments of area at most 1e-12 finest voxel faces are ignored;
 *   - dof order: lexicographic corner index, then the smallest triangle id of
 *     the component;
 *   - smoothing order (left open by the paper): lexicographic by default; the
 *     coloured order of orc_cycles (colours 0..7 on the way down, 7..0 on the
 *     way up) relaxes no row whose diagonal is not above 1e-20 of the level's
 *     mean diagonal, as the GPU smoother does.
 */
#define _DEFAULT_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXD 12
#define ORC_MAXP 12          /* a triangle clipped by 6 planes has <= 9 vertices */
#define ORC_TAU 1e-12        /* fragment area threshold in finest-voxel units */
#define ORC_NQ 4             /* Gauss-Legendre points per direction (exact to degree 6 on a triangle) */

/* ------------------------------------------------------------------------ */
/* small utilities                                                          */
/* ------------------------------------------------------------------------ */

static void *xmalloc(size_t n) {
    void *p = malloc(n ? n : 1);
    if (!p) { fprintf(stderr, "oracle: out of memory (%zu bytes)\n", n); abort(); }
    return p;
}
static void *xcalloc(size_t n, size_t s) {
    void *p = calloc(n ? n : 1, s ? s : 1);
    if (!p) { fprintf(stderr, "oracle: out of memory\n"); abort(); }
    return p;
}
static void *xrealloc(void *p, size_t n) {
    p = realloc(p, n ? n : 1);
    if (!p) { fprintf(stderr, "oracle: out of memory\n"); abort(); }
    return p;
}

static void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre rule on [0,1] by Newton iteration on P_n                   */
/* ------------------------------------------------------------------------ */

static double gl_x[ORC_NQ], gl_w[ORC_NQ];
static int gl_ready = 0;

static void legendre(int n, double x, double *p, double *dp) {
    double p0 = 1.0, p1 = x;
    for (int k = 1; k < n; k++) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1; p1 = p2;
    }
    *p = p1;
    *dp = n * (x * p1 - p0) / (x * x - 1.0);
}

static void gl_init(void) {
    if (gl_ready) return;
    const int n = ORC_NQ;
    for (int i = 0; i < n; i++) {
        double x = cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; it++) {
            double p, dp;
            legendre(n, x, &p, &dp);
            double dx = p / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        double p, dp;
        legendre(n, x, &p, &dp);
        gl_x[i] = 0.5 * (x + 1.0);
        gl_w[i] = 0.5 * 2.0 / ((1.0 - x * x) * dp * dp);
    }
    gl_ready = 1;
}

/* ------------------------------------------------------------------------ */
/* data structures                                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    int tri;
    int vox[3];
    int np;
    double p[ORC_MAXP][3];
    double area;
} Frag;

typedef struct { long long key; int tri; } CornerTri;

typedef struct {
    int d, s, N;                 /* depth, voxel side in finest units, voxels per axis */
    int nfrag; Frag *frag;
    int nct; long long *ctkey; int *cttri; int *ctdof;  /* (corner, triangle) -> dof, sorted */
    int ndof; int *dcorner; int *dmintri;               /* dof -> corner index triple, min triangle */
    int *fdof;                                          /* fragment -> dof of each of its 8 corners */
    long nnz; int *rp; int *ci; double *M; double *L;    /* Galerkin matrices, CSR */
    long pnnz; int *prp; int *pci; double *pv;          /* prolongation from depth d-1, n_d x n_{d-1} */
} Level;

typedef struct orc_hier {
    int D, d0, split, nv, nt;
    double *V;                   /* vertices in finest-grid units */
    int *F;
    double S, c[3], sigma;       /* cube side, centre, physical length per grid unit */
    double *tn;                  /* unit triangle normals */
    int ne; long long *ekey; int *etri;   /* sorted (edge key, triangle) */
    int *vtp, *vt;               /* vertex -> incident triangles */
    Level lev[ORC_MAXD + 1];
} orc_hier;

/* ------------------------------------------------------------------------ */
/* clipping a triangle by a voxel (Sutherland-Hodgman against 6 planes)      */
/* ------------------------------------------------------------------------ */

/* keep the part of polygon `in` (n vertices) with sign*(p[axis]-c) >= 0 */
static int clip_plane(double in[][3], int n, double out[][3], int axis, double c, double sign) {
    int m = 0;
    for (int i = 0; i < n; i++) {
        const double *a = in[i], *b = in[(i + 1) % n];
        double da = sign * (a[axis] - c), db = sign * (b[axis] - c);
        if (da >= 0) {
            if (m == ORC_MAXP) { fprintf(stderr, "oracle: clipped polygon too large\n"); abort(); }
            memcpy(out[m++], a, sizeof(double) * 3);
        }
        if ((da >= 0) != (db >= 0)) {
            if (m == ORC_MAXP) { fprintf(stderr, "oracle: clipped polygon too large\n"); abort(); }
            double t = (c - a[axis]) / (b[axis] - a[axis]);
            for (int k = 0; k < 3; k++) out[m][k] = a[k] + t * (b[k] - a[k]);
            out[m][axis] = c;
            m++;
        }
    }
    return m;
}

static double polygon_area(double p[][3], int n) {
    double s[3] = {0, 0, 0};
    for (int i = 1; i + 1 < n; i++) {
        double e1[3], e2[3], c[3];
        for (int k = 0; k < 3; k++) { e1[k] = p[i][k] - p[0][k]; e2[k] = p[i + 1][k] - p[0][k]; }
        cross3(e1, e2, c);
        for (int k = 0; k < 3; k++) s[k] += c[k];
    }
    return 0.5 * sqrt(dot3(s, s));
}

/* polygon of triangle t inside voxel (i,j,l) of side s; returns vertex count */
static int clip_triangle(const orc_hier *h, int t, const int *vox, int s, double out[][3]) {
    double a[ORC_MAXP][3], b[ORC_MAXP][3];
    for (int k = 0; k < 3; k++) memcpy(a[k], h->V + 3 * (size_t)h->F[3 * t + k], sizeof(double) * 3);
    int n = 3;
    for (int ax = 0; ax < 3 && n > 0; ax++) {
        double lo = (double)vox[ax] * s, hi = (double)(vox[ax] + 1) * s;
        n = clip_plane(a, n, b, ax, lo, +1.0);
        if (n == 0) break;
        n = clip_plane(b, n, a, ax, hi, -1.0);
    }
    for (int k = 0; k < n; k++) memcpy(out[k], a[k], sizeof(double) * 3);
    return n;
}

/* ------------------------------------------------------------------------ */
/* geometric predicates on the open support cube of a corner                */
/* ------------------------------------------------------------------------ */

/* does the closed segment [a,b] meet the open box (lo,hi)^3 ? */
static int segment_meets_open_box(const double *a, const double *b, const double *lo, const double *hi) {
    double L = -INFINITY, U = INFINITY;
    for (int k = 0; k < 3; k++) {
        double d = b[k] - a[k];
        if (d == 0.0) {
            if (!(a[k] > lo[k] && a[k] < hi[k])) return 0;
        } else {
            double t1 = (lo[k] - a[k]) / d, t2 = (hi[k] - a[k]) / d;
            if (t1 > t2) { double tmp = t1; t1 = t2; t2 = tmp; }
            if (t1 > L) L = t1;
            if (t2 < U) U = t2;
        }
    }
    return (L < U) && (L < 1.0) && (U > 0.0);
}

static int point_in_open_box(const double *p, const double *lo, const double *hi) {
    for (int k = 0; k < 3; k++) if (!(p[k] > lo[k] && p[k] < hi[k])) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* union-find                                                               */
/* ------------------------------------------------------------------------ */

static int uf_find(int *par, int a) {
    while (par[a] != a) { par[a] = par[par[a]]; a = par[a]; }
    return a;
}
static void uf_union(int *par, int a, int b) {
    a = uf_find(par, a); b = uf_find(par, b);
    if (a == b) return;
    if (a < b) par[b] = a; else par[a] = b;
}

/* ------------------------------------------------------------------------ */
/* sorting helpers                                                          */
/* ------------------------------------------------------------------------ */

static int cmp_corner_tri(const void *x, const void *y) {
    const CornerTri *a = x, *b = y;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return (a->tri > b->tri) - (a->tri < b->tri);
}

typedef struct { long long key; int tri; } EdgeTri;
static int cmp_edge_tri(const void *x, const void *y) {
    const EdgeTri *a = x, *b = y;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return (a->tri > b->tri) - (a->tri < b->tri);
}

static long long corner_key(const int *c, int N) {
    return ((long long)c[0] * (N + 1) + c[1]) * (long long)(N + 1) + c[2];
}
static void corner_decode(long long key, int N, int *c) {
    c[2] = (int)(key % (N + 1)); key /= (N + 1);
    c[1] = (int)(key % (N + 1)); key /= (N + 1);
    c[0] = (int)key;
}

/* first index in sorted (ctkey, cttri) equal to (key, tri), or -1 */
static int ct_lookup(const Level *lv, long long key, int tri) {
    int lo = 0, hi = lv->nct;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (lv->ctkey[mid] < key || (lv->ctkey[mid] == key && lv->cttri[mid] < tri)) lo = mid + 1;
        else hi = mid;
    }
    if (lo < lv->nct && lv->ctkey[lo] == key && lv->cttri[lo] == tri) return lo;
    return -1;
}

/* ------------------------------------------------------------------------ */
/* building one level: fragments, split basis                                */
/* ------------------------------------------------------------------------ */

static void build_fragments(orc_hier *h, Level *lv) {
    int cap = h->nt * 2 + 16, n = 0;
    Frag *fr = xmalloc(sizeof(Frag) * (size_t)cap);
    const int s = lv->s, N = lv->N;
    for (int t = 0; t < h->nt; t++) {
        double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int k = 0; k < 3; k++) {
            const double *p = h->V + 3 * (size_t)h->F[3 * t + k];
            for (int a = 0; a < 3; a++) { if (p[a] < mn[a]) mn[a] = p[a]; if (p[a] > mx[a]) mx[a] = p[a]; }
        }
        int lo[3], hi[3];
        for (int a = 0; a < 3; a++) {
            lo[a] = (int)floor(mn[a] / s); hi[a] = (int)floor(mx[a] / s);
            if (lo[a] < 0) lo[a] = 0;
            if (hi[a] > N - 1) hi[a] = N - 1;
        }
        int vox[3];
        for (vox[0] = lo[0]; vox[0] <= hi[0]; vox[0]++)
            for (vox[1] = lo[1]; vox[1] <= hi[1]; vox[1]++)
                for (vox[2] = lo[2]; vox[2] <= hi[2]; vox[2]++) {
                    double poly[ORC_MAXP][3];
                    int np = clip_triangle(h, t, vox, s, poly);
                    if (np < 3) continue;
                    double area = polygon_area(poly, np);
                    if (!(area > ORC_TAU)) continue;
                    if (n == cap) { cap *= 2; fr = xrealloc(fr, sizeof(Frag) * (size_t)cap); }
                    Frag *f = &fr[n++];
                    f->tri = t;
                    memcpy(f->vox, vox, sizeof vox);
                    f->np = np;
                    memcpy(f->p, poly, sizeof(double) * 3 * (size_t)np);
                    f->area = area;
                }
    }
    lv->nfrag = n;
    lv->frag = fr;
}

/* Section 4.2: one function per connected component of supp(b_k) /\ M */
static void build_split_basis(orc_hier *h, Level *lv) {
    const int N = lv->N, s = lv->s;
    /* (corner, triangle) pairs of every fragment */
    size_t np = (size_t)lv->nfrag * 8;
    CornerTri *ct = xmalloc(sizeof(CornerTri) * np);
    size_t m = 0;
    for (int f = 0; f < lv->nfrag; f++) {
        const Frag *fr = &lv->frag[f];
        for (int a = 0; a < 8; a++) {
            int c[3] = {fr->vox[0] + (a & 1), fr->vox[1] + ((a >> 1) & 1), fr->vox[2] + ((a >> 2) & 1)};
            ct[m].key = corner_key(c, N);
            ct[m].tri = fr->tri;
            m++;
        }
    }
    qsort(ct, m, sizeof(CornerTri), cmp_corner_tri);
    size_t u = 0;
    for (size_t i = 0; i < m; i++)
        if (u == 0 || ct[i].key != ct[u - 1].key || ct[i].tri != ct[u - 1].tri) ct[u++] = ct[i];
    lv->nct = (int)u;
    lv->ctkey = xmalloc(sizeof(long long) * u);
    lv->cttri = xmalloc(sizeof(int) * u);
    lv->ctdof = xmalloc(sizeof(int) * u);
    for (size_t i = 0; i < u; i++) { lv->ctkey[i] = ct[i].key; lv->cttri[i] = ct[i].tri; }
    free(ct);

    int dcap = 1024, ndof = 0;
    int *dcorner = xmalloc(sizeof(int) * 3 * dcap), *dmintri = xmalloc(sizeof(int) * dcap);
    int *par = xmalloc(sizeof(int) * (u + 1)), *lab = xmalloc(sizeof(int) * (u + 1));

    size_t g0 = 0;
    while (g0 < u) {
        size_t g1 = g0;
        while (g1 < u && lv->ctkey[g1] == lv->ctkey[g0]) g1++;
        int msz = (int)(g1 - g0);
        const int *T = lv->cttri + g0;   /* triangles of supp(b_k), ascending */
        int c[3];
        corner_decode(lv->ctkey[g0], N, c);
        double lo[3], hi[3];
        for (int a = 0; a < 3; a++) { lo[a] = (double)(c[a] - 1) * s; hi[a] = (double)(c[a] + 1) * s; }
        for (int i = 0; i < msz; i++) par[i] = i;
        if (h->split) {
            for (int i = 0; i < msz; i++) {
                int t = T[i];
                for (int e = 0; e < 3; e++) {
                    int va = h->F[3 * t + e], vb = h->F[3 * t + (e + 1) % 3];
                    if (!segment_meets_open_box(h->V + 3 * (size_t)va, h->V + 3 * (size_t)vb, lo, hi)) continue;
                    int x = va < vb ? va : vb, y = va < vb ? vb : va;
                    long long key = (long long)x * h->nv + y;
                    /* all triangles sharing this edge */
                    int l = 0, r = h->ne;
                    while (l < r) { int mid = (l + r) / 2; if (h->ekey[mid] < key) l = mid + 1; else r = mid; }
                    for (int q = l; q < h->ne && h->ekey[q] == key; q++) {
                        int t2 = h->etri[q];
                        if (t2 == t) continue;
                        /* is t2 in T ? */
                        int a = 0, b = msz;
                        while (a < b) { int mid = (a + b) / 2; if (T[mid] < t2) a = mid + 1; else b = mid; }
                        if (a < msz && T[a] == t2) uf_union(par, i, a);
                    }
                }
                for (int e = 0; e < 3; e++) {
                    int v = h->F[3 * t + e];
                    if (!point_in_open_box(h->V + 3 * (size_t)v, lo, hi)) continue;
                    for (int q = h->vtp[v]; q < h->vtp[v + 1]; q++) {
                        int t2 = h->vt[q];
                        int a = 0, b = msz;
                        while (a < b) { int mid = (a + b) / 2; if (T[mid] < t2) a = mid + 1; else b = mid; }
                        if (a < msz && T[a] == t2) uf_union(par, i, a);
                    }
                }
            }
        } else {
            for (int i = 0; i < msz; i++) par[i] = 0;
        }
        /* label components in order of their smallest triangle */
        for (int i = 0; i < msz; i++) lab[i] = -1;
        for (int i = 0; i < msz; i++) {
            int r = uf_find(par, i);
            if (lab[r] < 0) {
                if (ndof == dcap) {
                    dcap *= 2;
                    dcorner = xrealloc(dcorner, sizeof(int) * 3 * dcap);
                    dmintri = xrealloc(dmintri, sizeof(int) * dcap);
                }
                lab[r] = ndof;
                memcpy(dcorner + 3 * ndof, c, sizeof c);
                dmintri[ndof] = T[i];
                ndof++;
            }
            lv->ctdof[g0 + i] = lab[r];
        }
        g0 = g1;
    }
    free(par); free(lab);
    lv->ndof = ndof;
    lv->dcorner = dcorner;
    lv->dmintri = dmintri;

    /* dof of each corner of each fragment: the component holding its triangle */
    lv->fdof = xmalloc(sizeof(int) * 8 * (size_t)lv->nfrag);
    for (int f = 0; f < lv->nfrag; f++) {
        const Frag *fr = &lv->frag[f];
        for (int a = 0; a < 8; a++) {
            int cc[3] = {fr->vox[0] + (a & 1), fr->vox[1] + ((a >> 1) & 1), fr->vox[2] + ((a >> 2) & 1)};
            int idx = ct_lookup(lv, corner_key(cc, N), fr->tri);
            if (idx < 0) { fprintf(stderr, "oracle: missing corner/triangle pair\n"); abort(); }
            lv->fdof[8 * f + a] = lv->ctdof[idx];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Galerkin matrices by quadrature (Eq. 2, Section 5.1)                      */
/* ------------------------------------------------------------------------ */

typedef struct { int n, cap; int *c; double *m, *l; } Row;

static void row_add(Row *r, int col, double m, double l) {
    for (int i = 0; i < r->n; i++)
        if (r->c[i] == col) { r->m[i] += m; r->l[i] += l; return; }
    if (r->n == r->cap) {
        r->cap = r->cap ? 2 * r->cap : 32;
        r->c = xrealloc(r->c, sizeof(int) * r->cap);
        r->m = xrealloc(r->m, sizeof(double) * r->cap);
        r->l = xrealloc(r->l, sizeof(double) * r->cap);
    }
    r->c[r->n] = col; r->m[r->n] = m; r->l[r->n] = l; r->n++;
}

/* hat function of the corner at position cpos (finest units), support half-width s,
   its gradient; `upper` says on which side of the voxel the corner sits per axis */
static void hat_eval(const double *p, const double *cpos, double s, const int *upper, double *val, double *grad) {
    double f[3], df[3];
    for (int a = 0; a < 3; a++) {
        f[a] = 1.0 - fabs(p[a] - cpos[a]) / s;
        df[a] = (upper[a] ? 1.0 : -1.0) / s;
    }
    *val = f[0] * f[1] * f[2];
    grad[0] = df[0] * f[1] * f[2];
    grad[1] = f[0] * df[1] * f[2];
    grad[2] = f[0] * f[1] * df[2];
}

/* int b_a b_c and int <grad_M b_a, grad_M b_c> over fragment fi of a level, for its 8 voxel
   corners a, c (finest-grid units) */
static void fragment_local(const orc_hier *h, const Level *lv, int fi, double Mloc[8][8], double Lloc[8][8]) {
    const double s = lv->s;
    const Frag *fr = &lv->frag[fi];
    const double *n = h->tn + 3 * (size_t)fr->tri;
    double cpos[8][3];
    int upper[8][3];
    for (int a = 0; a < 8; a++) {
        upper[a][0] = a & 1; upper[a][1] = (a >> 1) & 1; upper[a][2] = (a >> 2) & 1;
        for (int k = 0; k < 3; k++) cpos[a][k] = (fr->vox[k] + upper[a][k]) * s;
    }
    for (int a = 0; a < 8; a++)
        for (int c = 0; c < 8; c++) { Mloc[a][c] = 0.0; Lloc[a][c] = 0.0; }
    for (int st = 1; st + 1 < fr->np; st++) {
        const double *P0 = fr->p[0], *P1 = fr->p[st], *P2 = fr->p[st + 1];
        double e1[3], e2[3], cr[3];
        for (int k = 0; k < 3; k++) { e1[k] = P1[k] - P0[k]; e2[k] = P2[k] - P0[k]; }
        cross3(e1, e2, cr);
        double jac = sqrt(dot3(cr, cr));    /* twice the sub-triangle area */
        for (int qa = 0; qa < ORC_NQ; qa++)
            for (int qb = 0; qb < ORC_NQ; qb++) {
                double xi = gl_x[qa], eta = gl_x[qb] * (1.0 - gl_x[qa]);
                double w = gl_w[qa] * gl_w[qb] * (1.0 - gl_x[qa]) * jac;
                double p[3];
                for (int k = 0; k < 3; k++) p[k] = P0[k] + xi * e1[k] + eta * e2[k];
                double b[8], g[8][3];
                for (int a = 0; a < 8; a++) {
                    double grad[3];
                    hat_eval(p, cpos[a], s, upper[a], &b[a], grad);
                    double gn = dot3(grad, n);
                    for (int k = 0; k < 3; k++) g[a][k] = grad[k] - gn * n[k];   /* tangential gradient */
                }
                for (int a = 0; a < 8; a++)
                    for (int c = 0; c < 8; c++) {
                        Mloc[a][c] += w * b[a] * b[c];
                        Lloc[a][c] += w * dot3(g[a], g[c]);
                    }
            }
    }
}

static void assemble_level(orc_hier *h, Level *lv) {
    gl_init();
    Row *rows = xcalloc((size_t)lv->ndof, sizeof(Row));
    for (int fi = 0; fi < lv->nfrag; fi++) {
        double Mloc[8][8], Lloc[8][8];
        fragment_local(h, lv, fi, Mloc, Lloc);
        for (int a = 0; a < 8; a++)
            for (int c = 0; c < 8; c++)
                row_add(&rows[lv->fdof[8 * fi + a]], lv->fdof[8 * fi + c], Mloc[a][c], Lloc[a][c]);
    }
    /* CSR with sorted columns; M scaled to physical area */
    long nnz = 0;
    for (int i = 0; i < lv->ndof; i++) nnz += rows[i].n;
    lv->nnz = nnz;
    lv->rp = xmalloc(sizeof(int) * (lv->ndof + 1));
    lv->ci = xmalloc(sizeof(int) * (size_t)nnz);
    lv->M = xmalloc(sizeof(double) * (size_t)nnz);
    lv->L = xmalloc(sizeof(double) * (size_t)nnz);
    const double area_scale = h->sigma * h->sigma;
    long pos = 0;
    for (int i = 0; i < lv->ndof; i++) {
        Row *r = &rows[i];
        for (int a = 1; a < r->n; a++) {      /* insertion sort by column */
            int c = r->c[a]; double m = r->m[a], l = r->l[a];
            int b = a - 1;
            while (b >= 0 && r->c[b] > c) { r->c[b + 1] = r->c[b]; r->m[b + 1] = r->m[b]; r->l[b + 1] = r->l[b]; b--; }
            r->c[b + 1] = c; r->m[b + 1] = m; r->l[b + 1] = l;
        }
        lv->rp[i] = (int)pos;
        for (int a = 0; a < r->n; a++) {
            lv->ci[pos] = r->c[a];
            lv->M[pos] = r->m[a] * area_scale;
            lv->L[pos] = r->l[a];
            pos++;
        }
        free(r->c); free(r->m); free(r->l);
    }
    lv->rp[lv->ndof] = (int)pos;
    free(rows);
}

/* ------------------------------------------------------------------------ */
/* prolongation (Section 4.3, Eq. 4)                                         */
/* ------------------------------------------------------------------------ */

/* P maps depth d-1 coefficients to depth d: row = fine dof, column = coarse dof.
   A fine dof at corner k' has, per axis, the coarse corner k'/2 with weight 1
   when k' is even, and (k'-1)/2, (k'+1)/2 with weight 1/2 each when odd; the
   coarse function is the component of that coarse corner that contains the
   fine component (chi = 1), found through any of its triangles. */
static void build_prolongation(Level *fine, const Level *coarse) {
    fine->prp = xmalloc(sizeof(int) * (fine->ndof + 1));
    fine->pci = xmalloc(sizeof(int) * 8 * (size_t)fine->ndof);
    fine->pv = xmalloc(sizeof(double) * 8 * (size_t)fine->ndof);
    long pos = 0;
    for (int j = 0; j < fine->ndof; j++) {
        const int *kf = fine->dcorner + 3 * j;
        int cand[3][2], wn[3];
        double wv[3];
        for (int a = 0; a < 3; a++) {
            if (kf[a] % 2 == 0) { cand[a][0] = kf[a] / 2; wn[a] = 1; wv[a] = 1.0; }
            else { cand[a][0] = (kf[a] - 1) / 2; cand[a][1] = (kf[a] + 1) / 2; wn[a] = 2; wv[a] = 0.5; }
        }
        fine->prp[j] = (int)pos;
        int tri = fine->dmintri[j];
        /* collect (coarse dof, weight), then sort by coarse dof */
        int cols[8]; double vals[8]; int m = 0;
        for (int x = 0; x < wn[0]; x++)
            for (int y = 0; y < wn[1]; y++)
                for (int z = 0; z < wn[2]; z++) {
                    int kc[3] = {cand[0][x], cand[1][y], cand[2][z]};
                    int idx = ct_lookup(coarse, corner_key(kc, coarse->N), tri);
                    if (idx < 0) { fprintf(stderr, "oracle: fine component has no parent component\n"); abort(); }
                    cols[m] = coarse->ctdof[idx];
                    vals[m] = wv[0] * wv[1] * wv[2];
                    m++;
                }
        for (int a = 1; a < m; a++) {
            int c = cols[a]; double v = vals[a]; int b = a - 1;
            while (b >= 0 && cols[b] > c) { cols[b + 1] = cols[b]; vals[b + 1] = vals[b]; b--; }
            cols[b + 1] = c; vals[b + 1] = v;
        }
        for (int a = 0; a < m; a++) { fine->pci[pos] = cols[a]; fine->pv[pos] = vals[a]; pos++; }
    }
    fine->prp[fine->ndof] = (int)pos;
    fine->pnnz = pos;
}

/* ------------------------------------------------------------------------ */
/* public: build                                                             */
/* ------------------------------------------------------------------------ */

static void build_level(orc_hier *h, int d) {
    Level *lv = &h->lev[d];
    memset(lv, 0, sizeof *lv);
    lv->d = d;
    lv->s = 1 << (h->D - d);
    lv->N = 1 << d;
    build_fragments(h, lv);
    build_split_basis(h, lv);
    assemble_level(h, lv);
}

/* The embedding (reading of Section 3.2, which leaves it open): by default the
   bounding box is centred in a cube of side 1.1 x its largest extent.  A caller
   may instead fix the cube (side S > 0, centre c), e.g. to put a piece of a
   mesh on exactly the grid of the whole mesh; every vertex must then lie inside
   the cube. */
static orc_hier *build_hier(const double *V, int nv, const int *F, int nt, int depth, int min_depth,
                            int coarse_max, int split, double S_fixed, const double *c_fixed) {
    if (depth < 1 || depth > ORC_MAXD || nv < 3 || nt < 1) return NULL;
    for (int i = 0; i < 3 * nt; i++) if (F[i] < 0 || F[i] >= nv) return NULL;
    for (int i = 0; i < 3 * nv; i++) if (!isfinite(V[i])) return NULL;
    orc_hier *h = xcalloc(1, sizeof(orc_hier));
    h->D = depth; h->nv = nv; h->nt = nt; h->split = split;
    if (S_fixed > 0) {
        h->S = S_fixed;
        for (int a = 0; a < 3; a++) h->c[a] = c_fixed[a];
        for (int i = 0; i < nv; i++)
            for (int a = 0; a < 3; a++)
                if (!(fabs(V[3 * i + a] - h->c[a]) < 0.5 * h->S)) { free(h); return NULL; }
    } else {
        /* centre the bounding box in a cube of side 1.1 x largest extent */
        double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int i = 0; i < nv; i++)
            for (int a = 0; a < 3; a++) {
                if (V[3 * i + a] < mn[a]) mn[a] = V[3 * i + a];
                if (V[3 * i + a] > mx[a]) mx[a] = V[3 * i + a];
            }
        double ext = 0;
        for (int a = 0; a < 3; a++) { h->c[a] = 0.5 * (mn[a] + mx[a]); if (mx[a] - mn[a] > ext) ext = mx[a] - mn[a]; }
        h->S = 1.1 * ext;
    }
    const double G = (double)(1 << depth);
    h->sigma = h->S / G;
    h->V = xmalloc(sizeof(double) * 3 * (size_t)nv);
    for (int i = 0; i < nv; i++)
        for (int a = 0; a < 3; a++) h->V[3 * i + a] = (V[3 * i + a] - h->c[a]) / h->S * G + 0.5 * G;
    h->F = xmalloc(sizeof(int) * 3 * (size_t)nt);
    memcpy(h->F, F, sizeof(int) * 3 * (size_t)nt);
    /* unit normals */
    h->tn = xmalloc(sizeof(double) * 3 * (size_t)nt);
    for (int t = 0; t < nt; t++) {
        const double *A = h->V + 3 * (size_t)F[3 * t], *B = h->V + 3 * (size_t)F[3 * t + 1], *C = h->V + 3 * (size_t)F[3 * t + 2];
        double e1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]}, e2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]}, n[3];
        cross3(e1, e2, n);
        double ln = sqrt(dot3(n, n));
        for (int a = 0; a < 3; a++) h->tn[3 * t + a] = ln > 0 ? n[a] / ln : 0.0;
    }
    /* edge -> triangles, vertex -> triangles */
    EdgeTri *et = xmalloc(sizeof(EdgeTri) * 3 * (size_t)nt);
    for (int t = 0; t < nt; t++)
        for (int e = 0; e < 3; e++) {
            int a = F[3 * t + e], b = F[3 * t + (e + 1) % 3];
            int x = a < b ? a : b, y = a < b ? b : a;
            et[3 * t + e].key = (long long)x * nv + y;
            et[3 * t + e].tri = t;
        }
    qsort(et, 3 * (size_t)nt, sizeof(EdgeTri), cmp_edge_tri);
    h->ne = 3 * nt;
    h->ekey = xmalloc(sizeof(long long) * h->ne);
    h->etri = xmalloc(sizeof(int) * h->ne);
    for (int i = 0; i < h->ne; i++) { h->ekey[i] = et[i].key; h->etri[i] = et[i].tri; }
    free(et);
    h->vtp = xcalloc((size_t)nv + 1, sizeof(int));
    for (int i = 0; i < 3 * nt; i++) h->vtp[F[i] + 1]++;
    for (int i = 0; i < nv; i++) h->vtp[i + 1] += h->vtp[i];
    h->vt = xmalloc(sizeof(int) * 3 * (size_t)nt);
    int *fill = xcalloc((size_t)nv, sizeof(int));
    for (int t = 0; t < nt; t++)
        for (int e = 0; e < 3; e++) { int v = F[3 * t + e]; h->vt[h->vtp[v] + fill[v]++] = t; }
    free(fill);
    /* levels from the finest down; stop at min_depth, or (min_depth < 0) at the
       first level with at most coarse_max functions */
    int d = depth;
    for (;;) {
        build_level(h, d);
        if (min_depth >= 0) { if (d <= min_depth) break; }
        else if (h->lev[d].ndof <= coarse_max) break;
        if (d == 0) break;
        d--;
    }
    h->d0 = d;
    for (int k = h->d0 + 1; k <= depth; k++) build_prolongation(&h->lev[k], &h->lev[k - 1]);
    return h;
}

orc_hier *orc_build(const double *V, int nv, const int *F, int nt, int depth, int min_depth,
                    int coarse_max, int split) {
    return build_hier(V, nv, F, nt, depth, min_depth, coarse_max, split, 0.0, NULL);
}

orc_hier *orc_build_embedded(const double *V, int nv, const int *F, int nt, int depth, int min_depth,
                             int coarse_max, int split, double S, const double *center) {
    if (!(S > 0) || !isfinite(S) || !center) return NULL;
    return build_hier(V, nv, F, nt, depth, min_depth, coarse_max, split, S, center);
}

void orc_free(orc_hier *h) {
    if (!h) return;
    for (int d = 0; d <= ORC_MAXD; d++) {
        Level *lv = &h->lev[d];
        free(lv->frag); free(lv->ctkey); free(lv->cttri); free(lv->ctdof);
        free(lv->dcorner); free(lv->dmintri); free(lv->fdof);
        free(lv->rp); free(lv->ci); free(lv->M); free(lv->L);
        free(lv->prp); free(lv->pci); free(lv->pv);
    }
    free(h->V); free(h->F); free(h->tn); free(h->ekey); free(h->etri); free(h->vtp); free(h->vt);
    free(h);
}

/* ------------------------------------------------------------------------ */
/* public: queries                                                           */
/* ------------------------------------------------------------------------ */

int orc_depth(const orc_hier *h) { return h->D; }
int orc_min_depth(const orc_hier *h) { return h->d0; }
double orc_cube_side(const orc_hier *h) { return h->S; }
void orc_center(const orc_hier *h, double *c) { memcpy(c, h->c, sizeof(double) * 3); }
int orc_ndof(const orc_hier *h, int d) { return h->lev[d].ndof; }
int orc_nfrag(const orc_hier *h, int d) { return h->lev[d].nfrag; }
long orc_nnz(const orc_hier *h, int d) { return h->lev[d].nnz; }
long orc_prolong_nnz(const orc_hier *h, int d) { return h->lev[d].pnnz; }

void orc_dofs(const orc_hier *h, int d, int *corner, int *mintri) {
    const Level *lv = &h->lev[d];
    memcpy(corner, lv->dcorner, sizeof(int) * 3 * (size_t)lv->ndof);
    memcpy(mintri, lv->dmintri, sizeof(int) * (size_t)lv->ndof);
}

/* (corner key, triangle, dof) membership table of a level: nct entries */
int orc_ncorner_tri(const orc_hier *h, int d) { return h->lev[d].nct; }
void orc_corner_tri(const orc_hier *h, int d, long long *key, int *tri, int *dof) {
    const Level *lv = &h->lev[d];
    memcpy(key, lv->ctkey, sizeof(long long) * (size_t)lv->nct);
    memcpy(tri, lv->cttri, sizeof(int) * (size_t)lv->nct);
    memcpy(dof, lv->ctdof, sizeof(int) * (size_t)lv->nct);
}

void orc_fragments(const orc_hier *h, int d, int *tri, int *vox, double *area) {
    const Level *lv = &h->lev[d];
    for (int f = 0; f < lv->nfrag; f++) {
        tri[f] = lv->frag[f].tri;
        memcpy(vox + 3 * f, lv->frag[f].vox, sizeof(int) * 3);
        area[f] = lv->frag[f].area * h->sigma * h->sigma;
    }
}

void orc_matrices(const orc_hier *h, int d, int *rp, int *ci, double *M, double *L) {
    const Level *lv = &h->lev[d];
    memcpy(rp, lv->rp, sizeof(int) * (lv->ndof + 1));
    memcpy(ci, lv->ci, sizeof(int) * (size_t)lv->nnz);
    if (M) memcpy(M, lv->M, sizeof(double) * (size_t)lv->nnz);
    if (L) memcpy(L, lv->L, sizeof(double) * (size_t)lv->nnz);
}

/* Mass matrix of level d with one weight per triangle, M_ij = sum_T w[T] int_T b_i b_j, in
   the CSR pattern of orc_matrices.  When the surface moves by an affine map per triangle,
   as in the time steps of the conformalized mean-curvature flow of Section 5.3, the area
   element of triangle T is its build-time one times A_t(T) / A_0(T), so with those ratios as
   w this is the mass matrix M_t of the moved surface on the build-time function space. */
void orc_mass_weighted(const orc_hier *h, int d, const double *w, double *M) {
    const Level *lv = &h->lev[d];
    gl_init();
    for (long k = 0; k < lv->nnz; k++) M[k] = 0.0;
    for (int fi = 0; fi < lv->nfrag; fi++) {
        double Mloc[8][8], Lloc[8][8];
        fragment_local(h, lv, fi, Mloc, Lloc);
        const double wt = w[lv->frag[fi].tri];
        for (int a = 0; a < 8; a++) {
            const int i = lv->fdof[8 * fi + a];
            for (int c = 0; c < 8; c++) {
                const int j = lv->fdof[8 * fi + c];
                int lo = lv->rp[i], hi = lv->rp[i + 1];
                while (lo < hi) {      /* column j in row i */
                    const int mid = (lo + hi) / 2;
                    if (lv->ci[mid] < j) lo = mid + 1; else hi = mid;
                }
                M[lo] += wt * Mloc[a][c];
            }
        }
    }
    const double area_scale = h->sigma * h->sigma;
    for (long k = 0; k < lv->nnz; k++) M[k] *= area_scale;
}

void orc_prolongation(const orc_hier *h, int d, int *rp, int *ci, double *v) {
    const Level *lv = &h->lev[d];
    memcpy(rp, lv->prp, sizeof(int) * (lv->ndof + 1));
    memcpy(ci, lv->pci, sizeof(int) * (size_t)lv->pnnz);
    memcpy(v, lv->pv, sizeof(double) * (size_t)lv->pnnz);
}

/* Observation of Section 4.1: every triangle of a fine component maps to the
   same component of each parent corner.  Returns the number of violations. */
long orc_check_nesting(const orc_hier *h) {
    long bad = 0;
    for (int d = h->d0 + 1; d <= h->D; d++) {
        const Level *f = &h->lev[d], *c = &h->lev[d - 1];
        for (int i = 0; i < f->nct; i++) {
            int kf[3];
            corner_decode(f->ctkey[i], f->N, kf);
            int j = f->ctdof[i];
            int tri = f->cttri[i];
            int cand[3][2], wn[3];
            for (int a = 0; a < 3; a++) {
                if (kf[a] % 2 == 0) { cand[a][0] = kf[a] / 2; wn[a] = 1; }
                else { cand[a][0] = (kf[a] - 1) / 2; cand[a][1] = (kf[a] + 1) / 2; wn[a] = 2; }
            }
            for (int x = 0; x < wn[0]; x++)
                for (int y = 0; y < wn[1]; y++)
                    for (int z = 0; z < wn[2]; z++) {
                        int kc[3] = {cand[0][x], cand[1][y], cand[2][z]};
                        long long key = corner_key(kc, c->N);
                        int a = ct_lookup(c, key, tri), b = ct_lookup(c, key, f->dmintri[j]);
                        if (a < 0 || b < 0 || c->ctdof[a] != c->ctdof[b]) bad++;
                    }
        }
    }
    return bad;
}

/* ------------------------------------------------------------------------ */
/* right-hand side int f b_i, f linear on each triangle (Section 5.2)         */
/* ------------------------------------------------------------------------ */

/* rhs_i = sum_T wt[T] int_T f b_i, f linear on each triangle; wt = NULL: all weights 1 */
static void project_rhs(const orc_hier *h, const double *fv, int nrhs, const double *wt, double *rhs) {
    gl_init();
    const Level *lv = &h->lev[h->D];
    const double s = lv->s;
    memset(rhs, 0, sizeof(double) * (size_t)lv->ndof * nrhs);
    for (int fi = 0; fi < lv->nfrag; fi++) {
        const Frag *fr = &lv->frag[fi];
        const int t = fr->tri;
        const double *A = h->V + 3 * (size_t)h->F[3 * t], *B = h->V + 3 * (size_t)h->F[3 * t + 1], *C = h->V + 3 * (size_t)h->F[3 * t + 2];
        double u1[3], u2[3];
        for (int k = 0; k < 3; k++) { u1[k] = B[k] - A[k]; u2[k] = C[k] - A[k]; }
        double g11 = dot3(u1, u1), g12 = dot3(u1, u2), g22 = dot3(u2, u2), det = g11 * g22 - g12 * g12;
        double cpos[8][3];
        int upper[8][3];
        for (int a = 0; a < 8; a++) {
            upper[a][0] = a & 1; upper[a][1] = (a >> 1) & 1; upper[a][2] = (a >> 2) & 1;
            for (int k = 0; k < 3; k++) cpos[a][k] = (fr->vox[k] + upper[a][k]) * s;
        }
        for (int st = 1; st + 1 < fr->np; st++) {
            const double *P0 = fr->p[0], *P1 = fr->p[st], *P2 = fr->p[st + 1];
            double e1[3], e2[3], cr[3];
            for (int k = 0; k < 3; k++) { e1[k] = P1[k] - P0[k]; e2[k] = P2[k] - P0[k]; }
            cross3(e1, e2, cr);
            double jac = sqrt(dot3(cr, cr));
            for (int qa = 0; qa < ORC_NQ; qa++)
                for (int qb = 0; qb < ORC_NQ; qb++) {
                    double xi = gl_x[qa], eta = gl_x[qb] * (1.0 - gl_x[qa]);
                    double w = gl_w[qa] * gl_w[qb] * (1.0 - gl_x[qa]) * jac * h->sigma * h->sigma;
                    if (wt) w *= wt[t];
                    double p[3], q[3];
                    for (int k = 0; k < 3; k++) { p[k] = P0[k] + xi * e1[k] + eta * e2[k]; q[k] = p[k] - A[k]; }
                    /* barycentric coordinates of p in triangle (A,B,C) */
                    double r1 = dot3(u1, q), r2 = dot3(u2, q);
                    double beta = (g22 * r1 - g12 * r2) / det, gamma = (g11 * r2 - g12 * r1) / det;
                    double lam[3] = {1.0 - beta - gamma, beta, gamma};
                    for (int a = 0; a < 8; a++) {
                        double b, grad[3];
                        hat_eval(p, cpos[a], s, upper[a], &b, grad);
                        int dof = lv->fdof[8 * fi + a];
                        for (int r = 0; r < nrhs; r++) {
                            double f = 0;
                            for (int k = 0; k < 3; k++) f += lam[k] * fv[(size_t)h->F[3 * t + k] * nrhs + r];
                            rhs[(size_t)dof * nrhs + r] += w * f * b;
                        }
                    }
                }
        }
    }
}

void orc_project_rhs(const orc_hier *h, const double *fv, int nrhs, double *rhs) {
    project_rhs(h, fv, nrhs, NULL, rhs);
}

/* int f b_i with the area element of triangle T scaled by w[T]: the right-hand side M_t u_t of
   a cMCF step (Section 5.3) on the build-time space */
void orc_project_rhs_weighted(const orc_hier *h, const double *fv, int nrhs, const double *w, double *rhs) {
    project_rhs(h, fv, nrhs, w, rhs);
}

/* ------------------------------------------------------------------------ */
/* evaluation at mesh vertices: u(v) = sum_i x_i b_i(v)                     */
/* ------------------------------------------------------------------------ */

void orc_eval_vertices(const orc_hier *h, const double *x, int nrhs, double *u) {
    const Level *lv = &h->lev[h->D];
    const double s = lv->s;
    for (int v = 0; v < h->nv; v++) {
        for (int r = 0; r < nrhs; r++) u[(size_t)v * nrhs + r] = 0.0;
        if (h->vtp[v] == h->vtp[v + 1]) continue;
        int t = h->vt[h->vtp[v]];
        const double *p = h->V + 3 * (size_t)v;
        int vox[3];
        for (int a = 0; a < 3; a++) {
            vox[a] = (int)floor(p[a] / s);
            if (vox[a] < 0) vox[a] = 0;
            if (vox[a] > lv->N - 1) vox[a] = lv->N - 1;
        }
        for (int a = 0; a < 8; a++) {
            int up[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
            int c[3];
            double cp[3], b, grad[3];
            for (int k = 0; k < 3; k++) { c[k] = vox[k] + up[k]; cp[k] = (double)c[k] * s; }
            hat_eval(p, cp, s, up, &b, grad);
            if (!(b > 0.0)) continue;
            int idx = ct_lookup(lv, corner_key(c, lv->N), t);
            if (idx < 0) continue;
            int dof = lv->ctdof[idx];
            for (int r = 0; r < nrhs; r++) u[(size_t)v * nrhs + r] += b * x[(size_t)dof * nrhs + r];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* multigrid: lexicographic Gauss-Seidel V-cycle, dense Cholesky at the bottom */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n; const int *rp, *ci; double *a;   /* A = M + t L in CSR */
    double *chol;                           /* dense factor at the coarsest level */
} SysLevel;

static void gs_sweep(const SysLevel *A, const double *b, double *x, int backward) {
    for (int q = 0; q < A->n; q++) {
        int i = backward ? A->n - 1 - q : q;
        double s = b[i], diag = 0.0;
        for (int k = A->rp[i]; k < A->rp[i + 1]; k++) {
            int j = A->ci[k];
            if (j == i) diag = A->a[k]; else s -= A->a[k] * x[j];
        }
        x[i] = s / diag;
    }
}

static void residual(const SysLevel *A, const double *b, const double *x, double *r) {
    for (int i = 0; i < A->n; i++) {
        double s = b[i];
        for (int k = A->rp[i]; k < A->rp[i + 1]; k++) s -= A->a[k] * x[A->ci[k]];
        r[i] = s;
    }
}

/* dense Cholesky of A + eps*Id, eps = 1e-12 * mean(diag A) (Discussion of Section 5) */
static int dense_cholesky(SysLevel *A) {
    int n = A->n;
    double *G = xcalloc((size_t)n * n, sizeof(double));
    double tr = 0;
    for (int i = 0; i < n; i++)
        for (int k = A->rp[i]; k < A->rp[i + 1]; k++) {
            G[(size_t)i * n + A->ci[k]] = A->a[k];
            if (A->ci[k] == i) tr += A->a[k];
        }
    double eps = 1e-12 * tr / (n > 0 ? n : 1);
    for (int i = 0; i < n; i++) G[(size_t)i * n + i] += eps;
    for (int j = 0; j < n; j++) {
        double s = G[(size_t)j * n + j];
        for (int k = 0; k < j; k++) s -= G[(size_t)j * n + k] * G[(size_t)j * n + k];
        if (!(s > 0)) { free(G); return -1; }
        double l = sqrt(s);
        G[(size_t)j * n + j] = l;
        for (int i = j + 1; i < n; i++) {
            double t = G[(size_t)i * n + j];
            for (int k = 0; k < j; k++) t -= G[(size_t)i * n + k] * G[(size_t)j * n + k];
            G[(size_t)i * n + j] = t / l;
        }
    }
    A->chol = G;
    return 0;
}

static void cholesky_solve(const SysLevel *A, const double *b, double *x) {
    int n = A->n;
    const double *G = A->chol;
    for (int i = 0; i < n; i++) {
        double s = b[i];
        for (int k = 0; k < i; k++) s -= G[(size_t)i * n + k] * x[k];
        x[i] = s / G[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = x[i];
        for (int k = i + 1; k < n; k++) s -= G[(size_t)k * n + i] * x[k];
        x[i] = s / G[(size_t)i * n + i];
    }
}

typedef struct {
    const orc_hier *h;
    SysLevel sys[ORC_MAXD + 1];
    double *r[ORC_MAXD + 1], *bc[ORC_MAXD + 1], *xc[ORC_MAXD + 1];
    int nu1, nu2;
    /* options of orc_cycles: coarse-grid visits per level (1 V-cycle, 2 W-cycle), colour-ordered
       smoothing, and relaxation instead of the direct solve at the coarsest level */
    int gamma, coloured, coarse_smooth;
    int *order[ORC_MAXD + 1];       /* rows by corner-parity colour (coloured smoothing) */
    double floor_d[ORC_MAXD + 1];   /* diagonals at or below this are not relaxed (coloured smoothing) */
} MG;

/* Gauss-Seidel over the rows in the order given by `order` (reversed when backward).
   Rows whose diagonal is not above `floor` are left unchanged. */
static void gs_sweep_ordered(const SysLevel *A, const int *order, double floor, const double *b, double *x,
                             int backward) {
    for (int q = 0; q < A->n; q++) {
        int i = order[backward ? A->n - 1 - q : q];
        double s = b[i], diag = 0.0;
        for (int k = A->rp[i]; k < A->rp[i + 1]; k++) {
            int j = A->ci[k];
            if (j == i) diag = A->a[k]; else s -= A->a[k] * x[j];
        }
        if (diag > floor) x[i] = s / diag;
    }
}

/* the order of coloured smoothing: rows by the parity class (k mod 2)^3 of their corner, colour
   c = kx%2 + 2 (ky%2) + 4 (kz%2), within a class by index (rows of one class never couple, so
   any order inside a class gives the same sweep); and the diagonal floor of reading A17 */
static void colour_order(const orc_hier *h, int d, const SysLevel *A, int **out, double *floor_out) {
    const Level *lv = &h->lev[d];
    int *ord = xmalloc(sizeof(int) * (size_t)(lv->ndof + 1));
    int pos = 0;
    for (int c = 0; c < 8; c++)
        for (int i = 0; i < lv->ndof; i++) {
            const int *k = lv->dcorner + 3 * (size_t)i;
            if ((k[0] & 1) + 2 * (k[1] & 1) + 4 * (k[2] & 1) == c) ord[pos++] = i;
        }
    double tr = 0.0;
    for (int i = 0; i < A->n; i++)
        for (int k = A->rp[i]; k < A->rp[i + 1]; k++)
            if (A->ci[k] == i) tr += A->a[k];
    /* a diagonal not above 1e-20 of the level's mean (or not positive) is not relaxed (A17) */
    double fl = 1e-20 * tr / (A->n > 0 ? A->n : 1);
    *out = ord;
    *floor_out = fl > 0.0 ? fl : 0.0;
}

static void smooth(MG *mg, int d, const double *b, double *x, int sweeps, int backward) {
    SysLevel *A = &mg->sys[d];
    for (int s = 0; s < sweeps; s++) {
        if (mg->coloured) gs_sweep_ordered(A, mg->order[d], mg->floor_d[d], b, x, backward);
        else gs_sweep(A, b, x, backward);
    }
}

/* One multigrid cycle on A_d x = b (Section 4.3): nu1 sweeps, the residual restricted by P^T,
   gamma visits of the next coarser level on the correction (gamma = 1: V-cycle, 2: W-cycle),
   the correction prolonged by P and added, nu2 sweeps in the reverse order.  The coarsest level
   is solved directly, or (coarse_smooth) relaxed by nu1 forward and nu2 backward sweeps. */
static void mg_cycle(MG *mg, int d, const double *b, double *x) {
    const orc_hier *h = mg->h;
    SysLevel *A = &mg->sys[d];
    if (d == h->d0) {
        if (mg->coarse_smooth) {
            smooth(mg, d, b, x, mg->nu1, 0);
            smooth(mg, d, b, x, mg->nu2, 1);
        } else {
            cholesky_solve(A, b, x);
        }
        return;
    }
    smooth(mg, d, b, x, mg->nu1, 0);
    residual(A, b, x, mg->r[d]);
    const Level *lv = &h->lev[d];
    int nc = h->lev[d - 1].ndof;
    double *bc = mg->bc[d - 1], *xc = mg->xc[d - 1];
    memset(bc, 0, sizeof(double) * (size_t)nc);
    memset(xc, 0, sizeof(double) * (size_t)nc);
    for (int i = 0; i < lv->ndof; i++)                    /* restriction: P^T r */
        for (int k = lv->prp[i]; k < lv->prp[i + 1]; k++) bc[lv->pci[k]] += lv->pv[k] * mg->r[d][i];
    for (int g = 0; g < mg->gamma; g++) mg_cycle(mg, d - 1, bc, xc);
    for (int i = 0; i < lv->ndof; i++)                    /* prolongation: x += P xc */
        for (int k = lv->prp[i]; k < lv->prp[i + 1]; k++) x[i] += lv->pv[k] * xc[lv->pci[k]];
    smooth(mg, d, b, x, mg->nu2, 1);
}

static void vcycle(MG *mg, int d, const double *b, double *x) {
    const orc_hier *h = mg->h;
    SysLevel *A = &mg->sys[d];
    if (d == h->d0) { cholesky_solve(A, b, x); return; }
    for (int s = 0; s < mg->nu1; s++) gs_sweep(A, b, x, 0);
    residual(A, b, x, mg->r[d]);
    const Level *lv = &h->lev[d];
    int nc = h->lev[d - 1].ndof;
    double *bc = mg->bc[d - 1], *xc = mg->xc[d - 1];
    memset(bc, 0, sizeof(double) * (size_t)nc);
    memset(xc, 0, sizeof(double) * (size_t)nc);
    for (int i = 0; i < lv->ndof; i++)                    /* restriction: P^T r */
        for (int k = lv->prp[i]; k < lv->prp[i + 1]; k++) bc[lv->pci[k]] += lv->pv[k] * mg->r[d][i];
    vcycle(mg, d - 1, bc, xc);
    for (int i = 0; i < lv->ndof; i++)                    /* prolongation: x += P xc */
        for (int k = lv->prp[i]; k < lv->prp[i + 1]; k++) x[i] += lv->pv[k] * xc[lv->pci[k]];
    for (int s = 0; s < mg->nu2; s++) gs_sweep(A, b, x, 1);
}

static double norm2(const double *v, int n) {
    double s = 0;
    for (int i = 0; i < n; i++) s += v[i] * v[i];
    return sqrt(s);
}

/* Solve (M + t L) x = rhs by V-cycles until ||rhs - A x|| <= tol ||rhs|| for
   every right-hand side, starting from the given x.  rhs and x are [n_D][nrhs].
   res_hist (optional, [(max_cycles+1) * nrhs]) receives relative residuals.
   Returns the number of cycles taken, or -1 if the coarse factor failed. */
int orc_solve(const orc_hier *h, double t, const double *rhs, double *x, int nrhs, double tol,
              int max_cycles, int nu1, int nu2, double *res_hist) {
    MG mg;
    memset(&mg, 0, sizeof mg);
    mg.h = h; mg.nu1 = nu1; mg.nu2 = nu2;
    int rc = 0;
    for (int d = h->d0; d <= h->D; d++) {
        const Level *lv = &h->lev[d];
        SysLevel *S = &mg.sys[d];
        S->n = lv->ndof; S->rp = lv->rp; S->ci = lv->ci;
        S->a = xmalloc(sizeof(double) * (size_t)(lv->nnz ? lv->nnz : 1));
        for (long k = 0; k < lv->nnz; k++) S->a[k] = lv->M[k] + t * lv->L[k];
        mg.r[d] = xmalloc(sizeof(double) * (size_t)(lv->ndof + 1));
        mg.bc[d] = xmalloc(sizeof(double) * (size_t)(lv->ndof + 1));
        mg.xc[d] = xmalloc(sizeof(double) * (size_t)(lv->ndof + 1));
    }
    if (dense_cholesky(&mg.sys[h->d0]) != 0) rc = -1;
    int n = h->lev[h->D].ndof, cycles = 0;
    double *b = xmalloc(sizeof(double) * (size_t)n), *xx = xmalloc(sizeof(double) * (size_t)n), *r = xmalloc(sizeof(double) * (size_t)n);
    for (int q = 0; q < nrhs && rc == 0; q++) {
        for (int i = 0; i < n; i++) { b[i] = rhs[(size_t)i * nrhs + q]; xx[i] = x[(size_t)i * nrhs + q]; }
        double nb = norm2(b, n);
        int c = 0;
        for (;;) {
            residual(&mg.sys[h->D], b, xx, r);
            double rel = nb > 0 ? norm2(r, n) / nb : 0.0;
            if (res_hist) res_hist[(size_t)c * nrhs + q] = rel;
            if (rel <= tol || c >= max_cycles) break;
            vcycle(&mg, h->D, b, xx);
            c++;
        }
        if (res_hist) for (int k = c + 1; k <= max_cycles; k++) res_hist[(size_t)k * nrhs + q] = NAN;
        if (c > cycles) cycles = c;
        for (int i = 0; i < n; i++) x[(size_t)i * nrhs + q] = xx[i];
    }
    free(b); free(xx); free(r);
    for (int d = h->d0; d <= h->D; d++) {
        free(mg.sys[d].a); free(mg.sys[d].chol); free(mg.r[d]); free(mg.bc[d]); free(mg.xc[d]);
    }
    return rc == 0 ? cycles : -1;
}

/* exactly `cycles` V-cycles per right-hand side, no residual checks (for timing) */
int orc_vcycles(const orc_hier *h, double t, const double *rhs, double *x, int nrhs, int cycles, int nu1, int nu2) {
    MG mg;
    memset(&mg, 0, sizeof mg);
    mg.h = h; mg.nu1 = nu1; mg.nu2 = nu2;
    for (int d = h->d0; d <= h->D; d++) {
        const Level *lv = &h->lev[d];
        SysLevel *S = &mg.sys[d];
        S->n = lv->ndof; S->rp = lv->rp; S->ci = lv->ci;
        S->a = xmalloc(sizeof(double) * (size_t)(lv->nnz ? lv->nnz : 1));
        for (long k = 0; k < lv->nnz; k++) S->a[k] = lv->M[k] + t * lv->L[k];
        mg.r[d] = xmalloc(sizeof(double) * (size_t)(lv->ndof + 1));
        mg.bc[d] = xmalloc(sizeof(double) * (size_t)(lv->ndof + 1));
        mg.xc[d] = xmalloc(sizeof(double) * (size_t)(lv->ndof + 1));
    }
    int rc = dense_cholesky(&mg.sys[h->d0]);
    int n = h->lev[h->D].ndof;
    double *b = xmalloc(sizeof(double) * (size_t)n), *xx = xmalloc(sizeof(double) * (size_t)n);
    for (int q = 0; q < nrhs && rc == 0; q++) {
        for (int i = 0; i < n; i++) { b[i] = rhs[(size_t)i * nrhs + q]; xx[i] = x[(size_t)i * nrhs + q]; }
        for (int c = 0; c < cycles; c++) vcycle(&mg, h->D, b, xx);
        for (int i = 0; i < n; i++) x[(size_t)i * nrhs + q] = xx[i];
    }
    free(b); free(xx);
    for (int d = h->d0; d <= h->D; d++) {
        free(mg.sys[d].a); free(mg.sys[d].chol); free(mg.r[d]); free(mg.bc[d]); free(mg.xc[d]);
    }
    return rc;
}

/* Exactly `cycles` multigrid cycles per right-hand side from the given x (no stopping test):
   gamma = 1 V-cycles, 2 W-cycles; coloured = 1 smooths colour by colour (colours 0..7 forward,
   7..0 backward) with the diagonal floor of reading A17, 0 lexicographically; coarse_smooth = 1
   relaxes the coarsest level instead of solving it.  Returns 0, or -1 if the coarse factor
   failed or an option is out of range. */
int orc_cycles(const orc_hier *h, double t, const double *rhs, double *x, int nrhs, int cycles, int nu1, int nu2,
               int gamma, int coloured, int coarse_smooth) {
    if (gamma < 1 || gamma > 2 || nu1 < 0 || nu2 < 0 || cycles < 0) return -1;
    MG mg;
    memset(&mg, 0, sizeof mg);
    mg.h = h; mg.nu1 = nu1; mg.nu2 = nu2;
    mg.gamma = gamma; mg.coloured = coloured != 0; mg.coarse_smooth = coarse_smooth != 0;
    for (int d = h->d0; d <= h->D; d++) {
        const Level *lv = &h->lev[d];
        SysLevel *S = &mg.sys[d];
        S->n = lv->ndof; S->rp = lv->rp; S->ci = lv->ci;
        S->a = xmalloc(sizeof(double) * (size_t)(lv->nnz ? lv->nnz : 1));
        for (long k = 0; k < lv->nnz; k++) S->a[k] = lv->M[k] + t * lv->L[k];
        mg.r[d] = xmalloc(sizeof(double) * (size_t)(lv->ndof + 1));
        mg.bc[d] = xmalloc(sizeof(double) * (size_t)(lv->ndof + 1));
        mg.xc[d] = xmalloc(sizeof(double) * (size_t)(lv->ndof + 1));
        if (mg.coloured) colour_order(h, d, S, &mg.order[d], &mg.floor_d[d]);
    }
    int rc = mg.coarse_smooth ? 0 : dense_cholesky(&mg.sys[h->d0]);
    int n = h->lev[h->D].ndof;
    double *b = xmalloc(sizeof(double) * (size_t)(n + 1)), *xx = xmalloc(sizeof(double) * (size_t)(n + 1));
    for (int q = 0; q < nrhs && rc == 0; q++) {
        for (int i = 0; i < n; i++) { b[i] = rhs[(size_t)i * nrhs + q]; xx[i] = x[(size_t)i * nrhs + q]; }
        for (int c = 0; c < cycles; c++) mg_cycle(&mg, h->D, b, xx);
        for (int i = 0; i < n; i++) x[(size_t)i * nrhs + q] = xx[i];
    }
    free(b); free(xx);
    for (int d = h->d0; d <= h->D; d++) {
        free(mg.sys[d].a); free(mg.sys[d].chol); free(mg.r[d]); free(mg.bc[d]); free(mg.xc[d]); free(mg.order[d]);
    }
    return rc == 0 ? 0 : -1;
}
