/*
 * vt_oracle.c -- plain FP64 CPU oracle for the per-particle Voronoi path.
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU
 * baseline leg of the benchmark call this file; the GPU library never does,
 * and this file shares no code, header or table with the GPU path.
 *
 * What it computes (PARAVT, arXiv:1601.06429):
 *   - Introduction: the Voronoi cell of particle i is the region of points
 *     nearer to x_i than to any other particle; the box may be periodic
 *     (Abstract, Discussion: "periodic conditions").
 *   - Implementation section: the cell volume from the cell facets, the
 *     density m_i / V_i, and the neighbour list read off shared facets.
 *
 * Method, written from the definition, no blocking or fusion:
 *   The cell is the intersection of the half-spaces
 *        H_p = { y : (y - x_i) . d <= |d|^2 / 2 },   d = p - x_i,
 *   over every other point p (every periodic image x_j + s L, s in {-1,0,1}^3,
 *   which suffices because the cell lies inside the cube of half-side L/2
 *   around x_i, the half-spaces of i's own six images).  The polytope is kept
 *   as a list of vertices, each tagged with the three planes that meet there;
 *   clipping by a plane removes the vertices strictly on the far side and
 *   adds one vertex on every edge (pair of vertices sharing two planes) that
 *   joins a removed and a kept vertex.
 *
 *   Side predicate.  For a vertex v = (a,b,c) and a plane j the question
 *   "is v strictly on the far side of plane j" equals "does x_j lie strictly
 *   inside the circumsphere of x_i, x_a, x_b, x_c".  It is decided first in
 *   interval arithmetic (every operation rounded outward by one ulp), and
 *   when the interval contains zero, exactly, with floating-point expansion
 *   arithmetic (the method of J. R. Shewchuk, "Adaptive precision
 *   floating-point arithmetic and fast robust geometric predicates", 1997:
 *   two-sum, two-product and grow-expansion), on the exact input doubles.
 *
 *   Candidate planes are taken in increasing order of a rigorous lower bound
 *   of |d|; a plane with |d| >= 2 R (R = an upper bound of the largest vertex
 *   distance from x_i) cannot cut, because every vertex y has
 *   y.d <= R |d| <= |d|^2/2.  Brute mode therefore still examines all
 *   27N-1 images (sorted); certified mode enumerates them from a k-d tree in
 *   radius passes and stops with the same lemma.
 *
 * Precision: FP64 geometry, exact predicates; no fused multiply-add except
 * where written explicitly (compile with -ffp-contract=off).
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* interval arithmetic, outward rounding by one ulp per operation       */
/* ------------------------------------------------------------------ */
typedef struct { double lo, hi; } ivl;

static inline double rdn(double x) { return nextafter(x, -INFINITY); }
static inline double rup(double x) { return nextafter(x, INFINITY); }
static inline ivl iv_pt(double x) { ivl r = {x, x}; return r; }
static inline ivl iv_add(ivl a, ivl b) { ivl r = {rdn(a.lo + b.lo), rup(a.hi + b.hi)}; return r; }
static inline ivl iv_sub(ivl a, ivl b) { ivl r = {rdn(a.lo - b.hi), rup(a.hi - b.lo)}; return r; }
static inline ivl iv_mul(ivl a, ivl b) {
    double p1 = a.lo * b.lo, p2 = a.lo * b.hi, p3 = a.hi * b.lo, p4 = a.hi * b.hi;
    double lo = fmin(fmin(p1, p2), fmin(p3, p4));
    double hi = fmax(fmax(p1, p2), fmax(p3, p4));
    ivl r = {rdn(lo), rup(hi)};
    return r;
}
static inline ivl iv_sq(ivl a) {
    double l2 = a.lo * a.lo, h2 = a.hi * a.hi;
    ivl r;
    if (a.lo >= 0) { r.lo = rdn(l2); r.hi = rup(h2); }
    else if (a.hi <= 0) { r.lo = rdn(h2); r.hi = rup(l2); }
    else { r.lo = 0.0; r.hi = rup(fmax(l2, h2)); }
    if (r.lo < 0) r.lo = 0.0;
    return r;
}
/* a / b for b not containing zero */
static inline ivl iv_div(ivl a, ivl b) {
    double q1 = a.lo / b.lo, q2 = a.lo / b.hi, q3 = a.hi / b.lo, q4 = a.hi / b.hi;
    double lo = fmin(fmin(q1, q2), fmin(q3, q4));
    double hi = fmax(fmax(q1, q2), fmax(q3, q4));
    ivl r = {rdn(lo), rup(hi)};
    return r;
}
static inline ivl iv_scale_exact(ivl a, double s) { /* s a power of two or +-1 */
    ivl r;
    if (s >= 0) { r.lo = a.lo * s; r.hi = a.hi * s; }
    else { r.lo = a.hi * s; r.hi = a.lo * s; }
    return r;
}
static inline int iv_has_zero(ivl a) { return a.lo <= 0.0 && a.hi >= 0.0; }

/* ------------------------------------------------------------------ */
/* exact expansion arithmetic (Shewchuk 1997)                           */
/* ------------------------------------------------------------------ */
#define XCAP 1024
typedef struct { int n; double c[XCAP]; } xpn; /* nonoverlapping, increasing magnitude */

static __thread int g_xp_overflow = 0;

static inline void two_sum(double a, double b, double *x, double *y) {
    double s = a + b;
    double bv = s - a;
    double av = s - bv;
    double br = b - bv;
    double ar = a - av;
    *x = s;
    *y = ar + br;
}
static inline void two_prod(double a, double b, double *x, double *y) {
    double p = a * b;
    *x = p;
    *y = fma(a, b, -p);
}
/* e += b, exactly (Grow-Expansion with zero elimination), in place */
static void xp_add_d(xpn *e, double b) {
    double q = b;
    int m = 0;
    for (int i = 0; i < e->n; i++) {
        double s, t;
        two_sum(q, e->c[i], &s, &t);
        if (t != 0.0) e->c[m++] = t;
        q = s;
    }
    if (q != 0.0) {
        if (m >= XCAP) { g_xp_overflow = 1; return; }
        e->c[m++] = q;
    }
    e->n = m;
}
static void xp_zero(xpn *e) { e->n = 0; }
static void xp_set_d(xpn *e, double a) { e->n = 0; xp_add_d(e, a); }
/* out += sign * a * b */
static void xp_addmul(xpn *out, const xpn *a, const xpn *b, int sign) {
    for (int i = 0; i < a->n; i++)
        for (int k = 0; k < b->n; k++) {
            double p, e;
            two_prod(a->c[i], b->c[k], &p, &e);
            if (sign < 0) { p = -p; e = -e; }
            xp_add_d(out, e);
            xp_add_d(out, p);
        }
}
static void xp_mul(xpn *out, const xpn *a, const xpn *b) {
    xp_zero(out);
    xp_addmul(out, a, b, +1);
}
static int xp_sign(const xpn *e) {
    if (e->n == 0) return 0;
    double top = e->c[e->n - 1];
    return (top > 0) - (top < 0);
}

/* ------------------------------------------------------------------ */
/* problem description                                                  */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t N;
    const double *x; /* [N][3] */
    double lo[3], hi[3], L[3];
    int periodic;
} problem;

/* A plane  n . y <= h  in the frame centred on x_i.
 * kind 0: bisector with point j under image shift s:  n = d, h = |d|^2/2.
 * kind 1: wall (bounded box), wall index w = 2*axis + (0: upper, 1: lower).
 * kind 2: voxel wall at the absolute coordinate bnd + sl along the axis of w
 *         (bnd a grid coordinate, sl a periodic shift), same orientation as a wall. */
typedef struct {
    double n[3], h;
    ivl ni[3], hi;
    int kind;
    int64_t j;
    int s[3];
    int w;
    double key_lo; /* rigorous lower bound of |d|^2 (bisectors) */
    double bnd, sl; /* voxel walls */
} plane_t;

typedef struct {
    int p[3];   /* plane ids */
    double y[3]; /* FP64 position, frame of x_i */
    ivl yi[3];   /* enclosure of the exact position */
} vert_t;

#define MAXV 2048
#define MAXP 4096

typedef struct {
    const problem *pb;
    int64_t i;
    plane_t *pl;
    int np;
    vert_t *v, *tmp;
    int nv;
    int8_t *side;
    /* counters */
    int64_t n_pred, n_exact, n_zero, n_tested, n_cut;
    int err;
} cellwork;

enum { OE_OK = 0, OE_CAP = -1, OE_DUP = -2, OE_NUM = -3, OE_XP = -4 };

/* exact displacement component: x_j[c] + s L[c] - x_i[c] */
static void exact_disp(const problem *pb, int64_t i, int64_t j, const int s[3], int c, xpn *out) {
    xp_zero(out);
    xp_add_d(out, pb->x[3 * j + c]);
    if (s[c] != 0) xp_add_d(out, s[c] * pb->L[c]);
    xp_add_d(out, -pb->x[3 * i + c]);
}

/* exact row (n_x, n_y, n_z, w) of plane p, scaled by a positive factor */
static void exact_row(const cellwork *cw, const plane_t *p, xpn row[4]) {
    const problem *pb = cw->pb;
    if (p->kind == 0) {
        xpn d[3];
        for (int c = 0; c < 3; c++) exact_disp(pb, cw->i, p->j, p->s, c, &d[c]);
        /* row = (2d, |d|^2) */
        xp_zero(&row[3]);
        for (int c = 0; c < 3; c++) {
            xp_zero(&row[c]);
            for (int k = 0; k < d[c].n; k++) xp_add_d(&row[c], 2.0 * d[c].c[k]);
            xp_addmul(&row[3], &d[c], &d[c], +1);
        }
    } else if (p->kind == 1) {
        int axis = p->w / 2, upper = (p->w % 2) == 0;
        for (int c = 0; c < 3; c++) xp_set_d(&row[c], c == axis ? (upper ? 1.0 : -1.0) : 0.0);
        xp_zero(&row[3]);
        if (upper) { xp_add_d(&row[3], pb->hi[axis]); xp_add_d(&row[3], -pb->x[3 * cw->i + axis]); }
        else { xp_add_d(&row[3], pb->x[3 * cw->i + axis]); xp_add_d(&row[3], -pb->lo[axis]); }
    } else {
        int axis = p->w / 2, upper = (p->w % 2) == 0;
        double sg = upper ? 1.0 : -1.0;
        for (int c = 0; c < 3; c++) xp_set_d(&row[c], c == axis ? sg : 0.0);
        /* h = sg (bnd + sl - x_i), exactly */
        xp_zero(&row[3]);
        xp_add_d(&row[3], sg * p->bnd);
        if (p->sl != 0.0) xp_add_d(&row[3], sg * p->sl);
        xp_add_d(&row[3], -sg * pb->x[3 * cw->i + axis]);
    }
}

/* exact 3x3 determinant of the n-parts of rows r0, r1, r2 */
static void exact_det3(xpn *out, xpn r0[4], xpn r1[4], xpn r2[4]) {
    xpn t1, t2;
    xp_zero(out);
    /* r0x (r1y r2z - r1z r2y) */
    xp_mul(&t1, &r1[1], &r2[2]); xp_addmul(&t1, &r1[2], &r2[1], -1);
    xp_addmul(out, &r0[0], &t1, +1);
    /* - r0y (r1x r2z - r1z r2x) */
    xp_mul(&t2, &r1[0], &r2[2]); xp_addmul(&t2, &r1[2], &r2[0], -1);
    xp_addmul(out, &r0[1], &t2, -1);
    /* + r0z (r1x r2y - r1y r2x) */
    xp_mul(&t1, &r1[0], &r2[1]); xp_addmul(&t1, &r1[1], &r2[0], -1);
    xp_addmul(out, &r0[2], &t1, +1);
}

/* exact side of vertex (a,b,c) w.r.t. plane j: +1 strictly outside (cut),
 * 0 on the plane, -1 strictly inside.  With N = rows a,b,c and
 * D4 = det[[n_a,h_a],[n_b,h_b],[n_c,h_c],[n_j,h_j]] one has
 * n_j.v - h_j = -D4 / det N. */
static int exact_side(cellwork *cw, const vert_t *v, const plane_t *pj) {
    static __thread xpn *buf = NULL;
    if (!buf) buf = (xpn *)malloc(sizeof(xpn) * 24);
    xpn *ra = buf, *rb = buf + 4, *rc = buf + 8, *rj = buf + 12;
    xpn *M = buf + 16, *D = buf + 17, *detN = buf + 18;
    g_xp_overflow = 0;
    exact_row(cw, &cw->pl[v->p[0]], ra);
    exact_row(cw, &cw->pl[v->p[1]], rb);
    exact_row(cw, &cw->pl[v->p[2]], rc);
    exact_row(cw, pj, rj);
    xp_zero(D);
    exact_det3(M, rb, rc, rj); xp_addmul(D, &ra[3], M, -1);
    exact_det3(M, ra, rc, rj); xp_addmul(D, &rb[3], M, +1);
    exact_det3(M, ra, rb, rj); xp_addmul(D, &rc[3], M, -1);
    exact_det3(detN, ra, rb, rc); xp_addmul(D, &rj[3], detN, +1);
    if (g_xp_overflow) { cw->err = OE_XP; return 0; }
    int sd = xp_sign(D), sn = xp_sign(detN);
    if (sn == 0) { cw->err = OE_NUM; return 0; }
    return -sd * sn;
}

static int side_of(cellwork *cw, const vert_t *v, const plane_t *pj) {
    cw->n_pred++;
    ivl s = iv_sub(iv_add(iv_add(iv_mul(pj->ni[0], v->yi[0]), iv_mul(pj->ni[1], v->yi[1])),
                          iv_mul(pj->ni[2], v->yi[2])),
                   pj->hi);
    if (s.lo > 0) return 1;
    if (s.hi < 0) return -1;
    cw->n_exact++;
    int r = exact_side(cw, v, pj);
    if (r == 0) cw->n_zero++;
    return r;
}

/* build a bisector plane for point j under image shift s */
static void make_bisector(const problem *pb, int64_t i, int64_t j, const int s[3], plane_t *p) {
    p->kind = 0; p->j = j; p->w = -1;
    ivl key = iv_pt(0.0);
    for (int c = 0; c < 3; c++) {
        p->s[c] = s[c];
        double xj = pb->x[3 * j + c], xi = pb->x[3 * i + c], sl = s[c] * pb->L[c];
        double t = xj - xi;
        p->n[c] = t + sl;
        ivl ti = iv_sub(iv_pt(xj), iv_pt(xi));
        p->ni[c] = s[c] ? iv_add(ti, iv_pt(sl)) : ti;
        key = iv_add(key, iv_sq(p->ni[c]));
    }
    p->h = 0.5 * (p->n[0] * p->n[0] + p->n[1] * p->n[1] + p->n[2] * p->n[2]);
    p->hi = iv_scale_exact(key, 0.5);
    p->key_lo = key.lo;
}

static void make_wall(const problem *pb, int64_t i, int w, plane_t *p) {
    int axis = w / 2, upper = (w % 2) == 0;
    p->kind = 1; p->j = -1; p->w = w; p->s[0] = p->s[1] = p->s[2] = 0;
    for (int c = 0; c < 3; c++) {
        double val = (c == axis) ? (upper ? 1.0 : -1.0) : 0.0;
        p->n[c] = val; p->ni[c] = iv_pt(val);
    }
    double xi = pb->x[3 * i + axis];
    if (upper) { p->h = pb->hi[axis] - xi; p->hi = iv_sub(iv_pt(pb->hi[axis]), iv_pt(xi)); }
    else { p->h = xi - pb->lo[axis]; p->hi = iv_sub(iv_pt(xi), iv_pt(pb->lo[axis])); }
    p->key_lo = 0.0;
}

/* voxel wall w (2*axis + 0 upper / 1 lower) at absolute coordinate bnd + sl */
static void make_voxel_wall(const problem *pb, int64_t i, int w, double bnd, double sl, plane_t *p) {
    int axis = w / 2, upper = (w % 2) == 0;
    p->kind = 2; p->j = -1; p->w = w; p->s[0] = p->s[1] = p->s[2] = 0;
    p->bnd = bnd; p->sl = sl;
    for (int c = 0; c < 3; c++) {
        double val = (c == axis) ? (upper ? 1.0 : -1.0) : 0.0;
        p->n[c] = val; p->ni[c] = iv_pt(val);
    }
    double xi = pb->x[3 * i + axis];
    ivl b = iv_add(iv_pt(bnd), iv_pt(sl));
    if (upper) { p->h = (bnd + sl) - xi; p->hi = iv_sub(b, iv_pt(xi)); }
    else { p->h = xi - (bnd + sl); p->hi = iv_sub(iv_pt(xi), b); }
    p->key_lo = 0.0;
}

/* vertex of planes a,b,c by Cramer's rule, FP64 and interval enclosure */
static int make_vertex(cellwork *cw, int a, int b, int c, vert_t *v) {
    const plane_t *A = &cw->pl[a], *B = &cw->pl[b], *C = &cw->pl[c];
    v->p[0] = a; v->p[1] = b; v->p[2] = c;
    /* plain FP64 */
    double bc[3] = {B->n[1] * C->n[2] - B->n[2] * C->n[1], B->n[2] * C->n[0] - B->n[0] * C->n[2],
                    B->n[0] * C->n[1] - B->n[1] * C->n[0]};
    double ca[3] = {C->n[1] * A->n[2] - C->n[2] * A->n[1], C->n[2] * A->n[0] - C->n[0] * A->n[2],
                    C->n[0] * A->n[1] - C->n[1] * A->n[0]};
    double ab[3] = {A->n[1] * B->n[2] - A->n[2] * B->n[1], A->n[2] * B->n[0] - A->n[0] * B->n[2],
                    A->n[0] * B->n[1] - A->n[1] * B->n[0]};
    double det = A->n[0] * bc[0] + A->n[1] * bc[1] + A->n[2] * bc[2];
    for (int k = 0; k < 3; k++) v->y[k] = (A->h * bc[k] + B->h * ca[k] + C->h * ab[k]) / det;
    /* interval */
    ivl ibc[3], ica[3], iab[3];
    for (int k = 0; k < 3; k++) {
        int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        ibc[k] = iv_sub(iv_mul(B->ni[k1], C->ni[k2]), iv_mul(B->ni[k2], C->ni[k1]));
        ica[k] = iv_sub(iv_mul(C->ni[k1], A->ni[k2]), iv_mul(C->ni[k2], A->ni[k1]));
        iab[k] = iv_sub(iv_mul(A->ni[k1], B->ni[k2]), iv_mul(A->ni[k2], B->ni[k1]));
    }
    ivl idet = iv_add(iv_add(iv_mul(A->ni[0], ibc[0]), iv_mul(A->ni[1], ibc[1])), iv_mul(A->ni[2], ibc[2]));
    if (iv_has_zero(idet)) {
        /* degenerate enclosure: use a huge box so that every test on this
         * vertex goes to the exact predicate */
        for (int k = 0; k < 3; k++) { v->yi[k].lo = -INFINITY; v->yi[k].hi = INFINITY; }
        return 0;
    }
    for (int k = 0; k < 3; k++) {
        ivl num = iv_add(iv_add(iv_mul(A->hi, ibc[k]), iv_mul(B->hi, ica[k])), iv_mul(C->hi, iab[k]));
        v->yi[k] = iv_div(num, idet);
    }
    return 0;
}

static int add_plane(cellwork *cw, const plane_t *p) {
    if (cw->np >= MAXP) { cw->err = OE_CAP; return -1; }
    cw->pl[cw->np] = *p;
    return cw->np++;
}

static int shares2(const vert_t *u, const vert_t *w, int *pa, int *pb) {
    int cnt = 0, q[3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            if (u->p[a] == w->p[b]) { if (cnt < 3) q[cnt] = u->p[a]; cnt++; }
    if (cnt != 2) return 0;
    *pa = q[0]; *pb = q[1];
    return 1;
}

/* clip the cell by plane p; returns 1 if it cut, 0 if not, <0 on error */
static int clip(cellwork *cw, const plane_t *p) {
    cw->n_tested++;
    int nout = 0;
    for (int k = 0; k < cw->nv; k++) {
        int sd = side_of(cw, &cw->v[k], p);
        if (cw->err) return cw->err;
        cw->side[k] = (int8_t)sd;
        nout += (sd > 0);
    }
    if (nout == 0) return 0;
    int pid = add_plane(cw, p);
    if (pid < 0) return cw->err;
    int m = 0;
    for (int k = 0; k < cw->nv; k++)
        if (cw->side[k] <= 0) cw->tmp[m++] = cw->v[k];
    for (int k = 0; k < cw->nv; k++) {
        if (cw->side[k] <= 0) continue;
        for (int q = 0; q < cw->nv; q++) {
            if (cw->side[q] > 0) continue;
            int pa, pb;
            if (!shares2(&cw->v[k], &cw->v[q], &pa, &pb)) continue;
            if (m >= MAXV) { cw->err = OE_CAP; return cw->err; }
            make_vertex(cw, pa, pb, pid, &cw->tmp[m++]);
        }
    }
    vert_t *t = cw->v; cw->v = cw->tmp; cw->tmp = t;
    cw->nv = m;
    cw->n_cut++;
    return 1;
}

/* upper bound of the largest |y|^2 over the vertices */
static double rmax2_upper(const cellwork *cw) {
    double r = 0.0;
    for (int k = 0; k < cw->nv; k++) {
        ivl s = iv_add(iv_add(iv_sq(cw->v[k].yi[0]), iv_sq(cw->v[k].yi[1])), iv_sq(cw->v[k].yi[2]));
        if (s.hi > r) r = s.hi;
    }
    return r;
}

/* initial polytope: the cube of i's six self images (periodic) or the box */
static void init_cell(cellwork *cw) {
    const problem *pb = cw->pb;
    cw->np = 0; cw->nv = 0; cw->err = 0;
    cw->n_pred = cw->n_exact = cw->n_zero = cw->n_tested = cw->n_cut = 0;
    for (int w = 0; w < 6; w++) {
        plane_t p;
        if (pb->periodic) {
            int s[3] = {0, 0, 0};
            s[w / 2] = (w % 2 == 0) ? 1 : -1;
            make_bisector(pb, cw->i, cw->i, s, &p);
        } else {
            make_wall(pb, cw->i, w, &p);
        }
        add_plane(cw, &p);
    }
    /* plane 2*axis is the upper face, 2*axis+1 the lower face */
    for (int corner = 0; corner < 8; corner++) {
        int a = (corner & 1) ? 1 : 0, b = (corner & 2) ? 3 : 2, c = (corner & 4) ? 5 : 4;
        make_vertex(cw, a, b, c, &cw->v[cw->nv++]);
    }
}

/* ------------------------------------------------------------------ */
/* candidate lists                                                      */
/* ------------------------------------------------------------------ */
/* key: rigorous lower bound of |d|^2 (sort order and stopping test);
 * pkey: the plain FP64 |d|^2 (membership of the radius passes) */
typedef struct { double key, pkey; int64_t j; int s[3]; } cand_t;

static int cand_cmp(const void *A, const void *B) {
    const cand_t *a = (const cand_t *)A, *b = (const cand_t *)B;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    if (a->j != b->j) return a->j < b->j ? -1 : 1;
    for (int c = 0; c < 3; c++) if (a->s[c] != b->s[c]) return a->s[c] < b->s[c] ? -1 : 1;
    return 0;
}

/* clip by a sorted candidate list; stops when no later candidate can cut.
 * returns 1 when stopped by the lemma, 0 when the list ran out, <0 error */
static int clip_sorted(cellwork *cw, const cand_t *c, int64_t n) {
    const problem *pb = cw->pb;
    double r2 = 4.0 * rmax2_upper(cw);
    for (int64_t k = 0; k < n; k++) {
        if (c[k].key > r2) return 1; /* |d| > 2R: this and all later ones cannot cut */
        plane_t p;
        make_bisector(pb, cw->i, c[k].j, c[k].s, &p);
        if (p.key_lo <= 0.0 && p.n[0] == 0.0 && p.n[1] == 0.0 && p.n[2] == 0.0) {
            cw->err = OE_DUP;
            return cw->err;
        }
        int r = clip(cw, &p);
        if (r < 0) return r;
        if (r > 0) r2 = 4.0 * rmax2_upper(cw);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* k-d tree for certified candidate enumeration                         */
/* ------------------------------------------------------------------ */
typedef struct { double lo[3], hi[3]; int64_t a, b; int64_t left, right; } kdnode;
typedef struct { const problem *pb; int64_t *idx; kdnode *nd; int64_t nn, cap; } kdtree;

static void kd_swap(int64_t *a, int64_t *b) { int64_t t = *a; *a = *b; *b = t; }

/* partial sort so that idx[k] holds the k-th smallest along axis, Hoare style */
static void kd_select(const double *x, int64_t *idx, int64_t lo, int64_t hi, int64_t k, int ax) {
    while (hi - lo > 1) {
        double pv = x[3 * idx[lo + (hi - lo) / 2] + ax];
        int64_t i = lo, j = hi - 1;
        while (i <= j) {
            while (x[3 * idx[i] + ax] < pv) i++;
            while (x[3 * idx[j] + ax] > pv) j--;
            if (i <= j) { kd_swap(&idx[i], &idx[j]); i++; j--; }
        }
        if (k <= j) hi = j + 1;
        else if (k >= i) lo = i;
        else return;
    }
}

static int64_t kd_build_rec(kdtree *t, int64_t a, int64_t b) {
    if (t->nn >= t->cap) {
        t->cap *= 2;
        t->nd = (kdnode *)realloc(t->nd, sizeof(kdnode) * t->cap);
    }
    int64_t id = t->nn++;
    kdnode nd;
    nd.a = a; nd.b = b; nd.left = nd.right = -1;
    for (int c = 0; c < 3; c++) { nd.lo[c] = INFINITY; nd.hi[c] = -INFINITY; }
    for (int64_t k = a; k < b; k++)
        for (int c = 0; c < 3; c++) {
            double v = t->pb->x[3 * t->idx[k] + c];
            if (v < nd.lo[c]) nd.lo[c] = v;
            if (v > nd.hi[c]) nd.hi[c] = v;
        }
    if (b - a > 8) {
        int ax = 0;
        for (int c = 1; c < 3; c++) if (nd.hi[c] - nd.lo[c] > nd.hi[ax] - nd.lo[ax]) ax = c;
        int64_t mid = a + (b - a) / 2;
        kd_select(t->pb->x, t->idx, a, b, mid, ax);
        nd.left = kd_build_rec(t, a, mid);
        nd.right = kd_build_rec(t, mid, b);
    }
    t->nd[id] = nd;
    return id;
}

static void kd_build(kdtree *t, const problem *pb) {
    t->pb = pb;
    t->idx = (int64_t *)malloc(sizeof(int64_t) * (pb->N > 0 ? pb->N : 1));
    for (int64_t k = 0; k < pb->N; k++) t->idx[k] = k;
    t->cap = 1024; t->nn = 0;
    t->nd = (kdnode *)malloc(sizeof(kdnode) * t->cap);
    if (pb->N > 0) kd_build_rec(t, 0, pb->N);
}

static void kd_free(kdtree *t) { free(t->idx); free(t->nd); }

typedef struct { cand_t *c; int64_t n, cap; } candbuf;

static void cb_push(candbuf *b, double key, double pkey, int64_t j, const int s[3]) {
    if (b->n >= b->cap) {
        b->cap = b->cap ? 2 * b->cap : 256;
        b->c = (cand_t *)realloc(b->c, sizeof(cand_t) * b->cap);
    }
    cand_t *c = &b->c[b->n++];
    c->key = key; c->pkey = pkey; c->j = j; c->s[0] = s[0]; c->s[1] = s[1]; c->s[2] = s[2];
}

/* plain FP64 |d|^2 of image (j,s) seen from i (*pkey) and a rigorous lower
 * bound of the exact |d|^2 (return value).  Each rounded displacement
 * component fl(fl(x_j - x_i) + sL) is within 4u(|t| + |d~|) of the exact
 * one (u = 2^-53), so |d| >= |d~| - sum of those bounds. */
static double cand_keys(const problem *pb, int64_t i, int64_t j, const int s[3], double *pkey) {
    const double u = ldexp(1.0, -53);
    double k = 0.0, del = 0.0;
    for (int c = 0; c < 3; c++) {
        double t = pb->x[3 * j + c] - pb->x[3 * i + c];
        double d = t + s[c] * pb->L[c];
        k += d * d;
        del += 4.0 * u * (fabs(t) + fabs(d));
    }
    *pkey = k;
    double r = sqrt(k) * (1.0 - 8.0 * u) - del * (1.0 + 8.0 * u);
    if (r <= 0.0) return 0.0;
    return r * r * (1.0 - 8.0 * u);
}

/* collect images (j,s), (j,s) != (i,0), with key in [r_lo2, r_hi2) */
static void kd_query(const kdtree *t, int64_t i, const int s[3], double r_lo2, double r_hi2, double rad,
                     candbuf *out) {
    const problem *pb = t->pb;
    double q[3];
    for (int c = 0; c < 3; c++) q[c] = pb->x[3 * i + c] - s[c] * pb->L[c];
    int64_t stack[256];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const kdnode *nd = &t->nd[stack[--sp]];
        double dd = 0.0;
        for (int c = 0; c < 3; c++) {
            double e = 0.0;
            if (q[c] < nd->lo[c]) e = nd->lo[c] - q[c];
            else if (q[c] > nd->hi[c]) e = q[c] - nd->hi[c];
            dd += e * e;
        }
        if (dd > rad * rad * (1.0 + 1e-9) + 1e-300) continue;
        if (nd->left < 0) {
            for (int64_t k = nd->a; k < nd->b; k++) {
                int64_t j = t->idx[k];
                if (j == i && s[0] == 0 && s[1] == 0 && s[2] == 0) continue;
                double pkey, key = cand_keys(pb, i, j, s, &pkey);
                if (pkey >= r_lo2 && pkey < r_hi2) cb_push(out, key, pkey, j, s);
            }
        } else {
            if (sp + 2 > 256) continue; /* cannot happen for a balanced tree */
            stack[sp++] = nd->left;
            stack[sp++] = nd->right;
        }
    }
}

/* ------------------------------------------------------------------ */
/* per-cell driver                                                      */
/* ------------------------------------------------------------------ */
typedef struct {
    double vol, cen[3], mom2, rmax;
    int nface, nvert, nedge;
    int64_t n_tested, n_cut;
} cellout;

/* largest absolute coordinate scale, for the rounding margin of keys */
static double coord_scale(const problem *pb) {
    double s = 0.0;
    for (int c = 0; c < 3; c++) {
        s = fmax(s, fabs(pb->lo[c])); s = fmax(s, fabs(pb->hi[c])); s = fmax(s, pb->L[c]);
    }
    return s;
}

/* move the k smallest candidates (cand_cmp order) to the front */
static void cand_select(cand_t *c, int64_t n, int64_t k) {
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        cand_t pv = c[lo + (hi - lo) / 2];
        int64_t i = lo, j = hi - 1;
        while (i <= j) {
            while (cand_cmp(&c[i], &pv) < 0) i++;
            while (cand_cmp(&c[j], &pv) > 0) j--;
            if (i <= j) { cand_t t = c[i]; c[i] = c[j]; c[j] = t; i++; j--; }
        }
        if (k <= j) hi = j + 1;
        else if (k >= i) lo = i;
        else return;
    }
}

/* candidates in ascending (key, index) order; an empty list (whose buffer may not exist yet) is left alone */
static void sort_cands(cand_t *c, int64_t n) {
    if (n > 1) qsort(c, (size_t)n, sizeof(cand_t), cand_cmp);
}

/* every image (j,s) != (i,0), s in {-1,0,1}^3 (periodic) or s = 0 */
static int run_brute(cellwork *cw, candbuf *cb) {
    const problem *pb = cw->pb;
    cb->n = 0;
    int smax = pb->periodic ? 1 : 0;
    for (int64_t j = 0; j < pb->N; j++)
        for (int sx = -smax; sx <= smax; sx++)
            for (int sy = -smax; sy <= smax; sy++)
                for (int sz = -smax; sz <= smax; sz++) {
                    int s[3] = {sx, sy, sz};
                    if (j == cw->i && sx == 0 && sy == 0 && sz == 0) continue;
                    double pkey, key = cand_keys(pb, cw->i, j, s, &pkey);
                    cb_push(cb, key, pkey, j, s);
                }
    /* stage 1: the 64 nearest, in order */
    int64_t k1 = cb->n < 64 ? cb->n : 64;
    cand_select(cb->c, cb->n, k1);
    sort_cands(cb->c, k1);
    int r = clip_sorted(cw, cb->c, k1);
    if (r < 0) return r;
    /* stage 2: every other image whose lower bound does not exclude a cut */
    double r2 = 4.0 * rmax2_upper(cw);
    int64_t m = 0;
    for (int64_t k = k1; k < cb->n; k++)
        if (cb->c[k].key <= r2) cb->c[m++] = cb->c[k];
    sort_cands(cb->c, m);
    r = clip_sorted(cw, cb->c, m);
    return r < 0 ? r : 0;
}

static int run_certified(cellwork *cw, const kdtree *t, candbuf *cb, int64_t leaf_of_i) {
    const problem *pb = cw->pb;
    double eps = ldexp(1.0, -52);
    double margin = 8.0 * eps * coord_scale(pb);
    double lmin = fmin(pb->L[0], fmin(pb->L[1], pb->L[2]));
    const kdnode *lf = &t->nd[leaf_of_i];
    double r = 0.0;
    for (int c = 0; c < 3; c++) r = fmax(r, lf->hi[c] - lf->lo[c]);
    if (r <= 0.0) r = 1e-3 * lmin;
    double r_lo2 = 0.0;
    int smax = pb->periodic ? 1 : 0;
    for (int pass = 0; pass < 64; pass++) {
        if (pb->periodic && r > 1.5 * lmin) {
            init_cell(cw); /* start over with every image */
            return run_brute(cw, cb);
        }
        double r_hi2 = r * r;
        cb->n = 0;
        for (int sx = -smax; sx <= smax; sx++)
            for (int sy = -smax; sy <= smax; sy++)
                for (int sz = -smax; sz <= smax; sz++) {
                    int s[3] = {sx, sy, sz};
                    kd_query(t, cw->i, s, r_lo2, r_hi2, r + margin, cb);
                }
        sort_cands(cb->c, cb->n);
        int rc = clip_sorted(cw, cb->c, cb->n);
        if (rc < 0) return rc;
        /* every image with key < r^2 has been examined; unexamined ones have
         * |d| >= r (1 - 2 eps) - margin.  Done when that is >= 2 R. */
        double R = sqrt(rmax2_upper(cw)) * (1.0 + 4 * eps);
        if (r * (1.0 - 4 * eps) - 2.0 * margin >= 2.0 * R) return 0;
        /* next pass: the annulus up to 2R, but at most twice the radius (a cell that is
         * still open after a few candidates closes with a few more) */
        r_lo2 = r_hi2;
        double rn = 2.0 * R * (1.0 + 1e-12) + 4.0 * margin;
        r = rn < 2.0 * r ? rn : 2.0 * r;
    }
    return OE_NUM;
}

/* faces and moments of the final polytope */
/* cubic face moment over a triangle: integral of |y|^2 y dA by the degree-3 rule of Strang and Fix
 * (weight -27/48 at the centroid, 25/48 at the three points with barycentric coordinates (3/5, 1/5, 1/5)),
 * exact for cubic integrands; returns the integral divided by the triangle's area */
static void tri_m3(const double *y0, const double *y1, const double *y2, double *out) {
    double p[4][3];
    for (int c = 0; c < 3; c++) {
        p[0][c] = (y0[c] + y1[c] + y2[c]) / 3.0;
        p[1][c] = 0.6 * y0[c] + 0.2 * y1[c] + 0.2 * y2[c];
        p[2][c] = 0.2 * y0[c] + 0.6 * y1[c] + 0.2 * y2[c];
        p[3][c] = 0.2 * y0[c] + 0.2 * y1[c] + 0.6 * y2[c];
    }
    const double w[4] = {-27.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0, 25.0 / 48.0};
    for (int c = 0; c < 3; c++) out[c] = 0.0;
    for (int k = 0; k < 4; k++) {
        double r2 = p[k][0] * p[k][0] + p[k][1] * p[k][1] + p[k][2] * p[k][2];
        for (int c = 0; c < 3; c++) out[c] += w[k] * r2 * p[k][c];
    }
}

static int extract(cellwork *cw, cellout *co, int face_cap, int64_t *f_nbr, int32_t *f_shift, double *f_area,
                   double *f_cen, double *f_dist, double *f_m3) {
    const problem *pb = cw->pb;
    int *vlist = (int *)malloc(sizeof(int) * (cw->nv + 1));
    int *order = (int *)malloc(sizeof(int) * (cw->nv + 1));
    double vol = 0.0, cz[3] = {0, 0, 0}, m2 = 0.0;
    int nf = 0, nedge2 = 0;
    for (int a = 0; a < cw->np; a++) {
        int nvl = 0;
        for (int k = 0; k < cw->nv; k++) {
            const int *p = cw->v[k].p;
            if (p[0] == a || p[1] == a || p[2] == a) vlist[nvl++] = k;
        }
        if (nvl == 0) continue;
        if (nvl < 3) { free(vlist); free(order); return OE_NUM; }
        nedge2 += nvl;
        /* walk the face boundary: consecutive vertices share plane a and one other plane */
        int start = vlist[0];
        int via;
        { const int *p = cw->v[start].p; via = (p[0] != a) ? p[0] : p[1]; }
        int cur = start, prev = -1, cnt = 0;
        for (;;) {
            order[cnt++] = cur;
            if (cnt > nvl) { free(vlist); free(order); return OE_NUM; }
            int nxt = -1;
            for (int q = 0; q < nvl; q++) {
                int k = vlist[q];
                if (k == cur || k == prev) continue;
                const int *p = cw->v[k].p;
                if (p[0] == via || p[1] == via || p[2] == via) { nxt = k; break; }
            }
            if (nxt < 0) { free(vlist); free(order); return OE_NUM; }
            /* next exit plane: the plane of nxt that is neither a nor via */
            const int *p = cw->v[nxt].p;
            int nvia = -1;
            for (int u = 0; u < 3; u++) if (p[u] != a && p[u] != via) nvia = p[u];
            prev = cur; cur = nxt; via = nvia;
            if (cur == start) break;
        }
        if (cnt != nvl) { free(vlist); free(order); return OE_NUM; }
        /* fan from the first vertex */
        const plane_t *P = &cw->pl[a];
        double nn = sqrt(P->n[0] * P->n[0] + P->n[1] * P->n[1] + P->n[2] * P->n[2]);
        double nh[3] = {P->n[0] / nn, P->n[1] / nn, P->n[2] / nn};
        const double *y0 = cw->v[order[0]].y;
        double A = 0.0, C[3] = {0, 0, 0}, fv = 0.0, fz[3] = {0, 0, 0}, fm2 = 0.0, M3[3] = {0, 0, 0};
        for (int k = 1; k + 1 < cnt; k++) {
            const double *y1 = cw->v[order[k]].y, *y2 = cw->v[order[k + 1]].y;
            double e1[3] = {y1[0] - y0[0], y1[1] - y0[1], y1[2] - y0[2]};
            double e2[3] = {y2[0] - y0[0], y2[1] - y0[1], y2[2] - y0[2]};
            double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
            double at = 0.5 * (cr[0] * nh[0] + cr[1] * nh[1] + cr[2] * nh[2]);
            A += at;
            for (int c = 0; c < 3; c++) C[c] += at * (y0[c] + y1[c] + y2[c]) / 3.0;
            double t3[3];
            tri_m3(y0, y1, y2, t3);
            for (int c = 0; c < 3; c++) M3[c] += at * t3[c];
            /* tetrahedron (site, y0, y1, y2), signed like the fan triangle */
            double tv = (y0[0] * (y1[1] * y2[2] - y1[2] * y2[1]) - y0[1] * (y1[0] * y2[2] - y1[2] * y2[0]) +
                         y0[2] * (y1[0] * y2[1] - y1[1] * y2[0])) / 6.0;
            fv += tv;
            for (int c = 0; c < 3; c++) fz[c] += tv * (y0[c] + y1[c] + y2[c]) / 4.0;
            double s2 = y0[0] * y0[0] + y0[1] * y0[1] + y0[2] * y0[2] + y1[0] * y1[0] + y1[1] * y1[1] +
                        y1[2] * y1[2] + y2[0] * y2[0] + y2[1] * y2[1] + y2[2] * y2[2] +
                        y0[0] * y1[0] + y0[1] * y1[1] + y0[2] * y1[2] + y0[0] * y2[0] + y0[1] * y2[1] +
                        y0[2] * y2[2] + y1[0] * y2[0] + y1[1] * y2[1] + y1[2] * y2[2];
            fm2 += tv * s2 / 10.0;
        }
        /* the walk direction is arbitrary: orient the face outward */
        double sg = (A < 0) ? -1.0 : 1.0;
        vol += sg * fv;
        m2 += sg * fm2;
        for (int c = 0; c < 3; c++) cz[c] += sg * fz[c];
        if (A != 0.0) for (int c = 0; c < 3; c++) C[c] /= A;
        if (A < 0) A = -A;
        if (nf >= face_cap) { free(vlist); free(order); return OE_CAP; }
        f_nbr[nf] = (P->kind == 0) ? P->j : -1 - P->w;
        for (int c = 0; c < 3; c++) {
            f_shift[3 * nf + c] = P->s[c];
            f_cen[3 * nf + c] = C[c] + pb->x[3 * cw->i + c];
        }
        f_area[nf] = A;
        f_dist[nf] = P->h / nn;
        if (f_m3) for (int c = 0; c < 3; c++) f_m3[3 * nf + c] = sg * M3[c];
        nf++;
    }
    co->vol = vol;
    for (int c = 0; c < 3; c++) co->cen[c] = (vol > 0 ? cz[c] / vol : 0.0) + pb->x[3 * cw->i + c];
    co->mom2 = m2;
    co->rmax = 0.0;
    for (int k = 0; k < cw->nv; k++) {
        const double *y = cw->v[k].y;
        double r = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
        if (r > co->rmax) co->rmax = r;
    }
    co->nface = nf;
    co->nvert = cw->nv;
    co->nedge = nedge2 / 2;
    free(vlist); free(order);
    return 0;
}

/* ------------------------------------------------------------------ */
/* public entry points (ctypes)                                         */
/* ------------------------------------------------------------------ */
/*
 * oracle_cells: Voronoi cells of the listed particles.
 *   pos       [N][3] FP64 positions; periodic boxes need them in [lo, hi)
 *   box_lo/hi box corners; periodic != 0 selects the periodic cube
 *   cells     particle ids to compute (NULL: all, n_cells = N)
 *   mode      0 brute force over all 27N-1 images, 1 certified k-d tree
 *   face_cap  face slots per listed cell
 * per listed cell k:  vol[k], cen[3k..], mom2[k] = integral |y - x_i|^2, rmax[k] = largest vertex
 *   distance from x_i,
 *   nface[k] (< 0: error code), nvert[k], nedge[k], ntest[k] (planes
 *   examined), ncut[k] (planes that cut);
 * face slots [k*face_cap, k*face_cap + nface[k]):  f_nbr (neighbour id, or
 *   -1-w for box wall w), f_shift[3] (image shift), f_area, f_cen[3]
 *   (absolute), f_dist (distance from x_i to the facet plane), f_m3[3] (NULL: not
 *   wanted) = integral over the facet of |y - x_i|^2 (y - x_i) dA.
 * counters[0..3] += predicates, exact fallbacks, exact zeros, errors.
 * Returns 0, or the first per-cell error code.
 */
/* a problem with its k-d tree (certified mode), kept across calls by oracle_tree_* */
typedef struct {
    problem pb;
    int has_tree;
    kdtree tree;
    int64_t *leaf_of;
    double t_build;  /* seconds spent building the tree */
} oracle_ctx;

static double wall_seconds(void) {
#ifdef _OPENMP
    return omp_get_wtime();
#else
    return (double)clock() / CLOCKS_PER_SEC;
#endif
}

static void ctx_init(oracle_ctx *cx, int64_t N, const double *pos, const double *box_lo, const double *box_hi,
                     int periodic, int with_tree) {
    memset(cx, 0, sizeof(*cx));
    cx->pb.N = N; cx->pb.x = pos; cx->pb.periodic = periodic;
    for (int c = 0; c < 3; c++) {
        cx->pb.lo[c] = box_lo[c]; cx->pb.hi[c] = box_hi[c]; cx->pb.L[c] = box_hi[c] - box_lo[c];
    }
    if (!with_tree) return;
    double t0 = wall_seconds();
    kd_build(&cx->tree, &cx->pb);
    cx->leaf_of = (int64_t *)malloc(sizeof(int64_t) * (N > 0 ? N : 1));
    for (int64_t n = 0; n < cx->tree.nn; n++)
        if (cx->tree.nd[n].left < 0)
            for (int64_t k = cx->tree.nd[n].a; k < cx->tree.nd[n].b; k++) cx->leaf_of[cx->tree.idx[k]] = n;
    cx->has_tree = 1;
    cx->t_build = wall_seconds() - t0;
}

static void ctx_free(oracle_ctx *cx) {
    if (cx->has_tree) { kd_free(&cx->tree); free(cx->leaf_of); }
    cx->has_tree = 0;
}

/* the cells of the listed particles on a prepared problem: certified mode if it has a tree, else brute force */
static int ctx_cells(const oracle_ctx *cx, const int64_t *cells, int64_t n_cells, int face_cap, double *vol,
                     double *cen, double *mom2, double *rmax, int32_t *nface, int32_t *nvert, int32_t *nedge,
                     int64_t *ntest, int64_t *ncut, int64_t *f_nbr, int32_t *f_shift, double *f_area,
                     double *f_cen, double *f_dist, double *f_m3, int64_t *counters, int nthreads) {
    const problem *pbp = &cx->pb;
    if (cells == NULL) n_cells = pbp->N;
    int64_t tot_pred = 0, tot_exact = 0, tot_zero = 0, tot_err = 0;
    int first_err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel reduction(+ : tot_pred, tot_exact, tot_zero, tot_err)
    {
        cellwork cw;
        cw.pb = pbp;
        cw.pl = (plane_t *)malloc(sizeof(plane_t) * MAXP);
        cw.v = (vert_t *)malloc(sizeof(vert_t) * MAXV);
        cw.tmp = (vert_t *)malloc(sizeof(vert_t) * MAXV);
        cw.side = (int8_t *)malloc(MAXV);
        candbuf cb = {NULL, 0, 0};
#pragma omp for schedule(dynamic, 16)
        for (int64_t k = 0; k < n_cells; k++) {
            int64_t i = cells ? cells[k] : k;
            cw.i = i;
            init_cell(&cw);
            int rc = cx->has_tree ? run_certified(&cw, &cx->tree, &cb, cx->leaf_of[i]) : run_brute(&cw, &cb);
            cellout co;
            memset(&co, 0, sizeof(co));
            if (rc == 0)
                rc = extract(&cw, &co, face_cap, f_nbr + k * face_cap, f_shift + 3 * k * face_cap,
                             f_area + k * face_cap, f_cen + 3 * k * face_cap, f_dist + k * face_cap,
                             f_m3 ? f_m3 + 3 * k * face_cap : NULL);
            tot_pred += cw.n_pred; tot_exact += cw.n_exact; tot_zero += cw.n_zero;
            ntest[k] = cw.n_tested; ncut[k] = cw.n_cut;
            if (rc != 0) {
                tot_err++;
                nface[k] = rc; vol[k] = NAN; mom2[k] = NAN; rmax[k] = NAN;
                for (int c = 0; c < 3; c++) cen[3 * k + c] = NAN;
                nvert[k] = nedge[k] = 0;
#pragma omp critical
                { if (!first_err) first_err = rc; }
            } else {
                nface[k] = co.nface; vol[k] = co.vol; mom2[k] = co.mom2; rmax[k] = co.rmax;
                for (int c = 0; c < 3; c++) cen[3 * k + c] = co.cen[c];
                nvert[k] = co.nvert; nedge[k] = co.nedge;
            }
        }
        free(cw.pl); free(cw.v); free(cw.tmp); free(cw.side); free(cb.c);
    }
    counters[0] += tot_pred; counters[1] += tot_exact; counters[2] += tot_zero; counters[3] += tot_err;
    return first_err;
}

int oracle_cells(int64_t N, const double *pos, const double *box_lo, const double *box_hi, int periodic,
                 const int64_t *cells, int64_t n_cells, int mode, int face_cap, double *vol, double *cen,
                 double *mom2, double *rmax, int32_t *nface, int32_t *nvert, int32_t *nedge, int64_t *ntest,
                 int64_t *ncut,
                 int64_t *f_nbr, int32_t *f_shift, double *f_area, double *f_cen, double *f_dist,
                 double *f_m3, int64_t *counters, int nthreads) {
    oracle_ctx cx;
    ctx_init(&cx, N, pos, box_lo, box_hi, periodic, mode == 1);
    int rc = ctx_cells(&cx, cells, n_cells, face_cap, vol, cen, mom2, rmax, nface, nvert, nedge, ntest, ncut,
                       f_nbr, f_shift, f_area, f_cen, f_dist, f_m3, counters, nthreads);
    ctx_free(&cx);
    return rc;
}

/*
 * oracle_tree_new / oracle_tree_cells / oracle_tree_free: certified mode with the k-d tree built once and kept,
 * so that many calls (or a timed call) on the same point set pay for the tree only once.  `pos` must stay valid
 * until oracle_tree_free.  oracle_tree_build_seconds: the wall time the tree took.  Same outputs as
 * oracle_cells(mode 1).
 */
void *oracle_tree_new(int64_t N, const double *pos, const double *box_lo, const double *box_hi, int periodic) {
    oracle_ctx *cx = (oracle_ctx *)malloc(sizeof(oracle_ctx));
    if (cx) ctx_init(cx, N, pos, box_lo, box_hi, periodic, 1);
    return cx;
}

double oracle_tree_build_seconds(const void *t) { return ((const oracle_ctx *)t)->t_build; }

int oracle_tree_cells(const void *t, const int64_t *cells, int64_t n_cells, int face_cap, double *vol, double *cen,
                      double *mom2, double *rmax, int32_t *nface, int32_t *nvert, int32_t *nedge, int64_t *ntest,
                      int64_t *ncut, int64_t *f_nbr, int32_t *f_shift, double *f_area, double *f_cen,
                      double *f_dist, double *f_m3, int64_t *counters, int nthreads) {
    return ctx_cells((const oracle_ctx *)t, cells, n_cells, face_cap, vol, cen, mom2, rmax, nface, nvert, nedge,
                     ntest, ncut, f_nbr, f_shift, f_area, f_cen, f_dist, f_m3, counters, nthreads);
}

void oracle_tree_free(void *t) {
    if (!t) return;
    ctx_free((oracle_ctx *)t);
    free(t);
}

/*
 * oracle_insphere_side: the exact side predicate on its own, for pinning.
 * The planes are bisectors of x_i with p_a, p_b, p_c (defining the vertex)
 * and p_j, all given as absolute FP64 points.  Returns +1 when the vertex
 * is strictly on p_j's side (p_j strictly inside the circumsphere of
 * x_i, p_a, p_b, p_c), 0 on the sphere, -1 outside.  mode 0: interval
 * filter then exact; mode 1: exact only.
 */
int oracle_insphere_side(const double *xi, const double *pa, const double *pbp, const double *pc,
                         const double *pj, int mode) {
    double pts[15];
    memcpy(pts, xi, 24); memcpy(pts + 3, pa, 24); memcpy(pts + 6, pbp, 24);
    memcpy(pts + 9, pc, 24); memcpy(pts + 12, pj, 24);
    problem pb;
    pb.N = 5; pb.x = pts; pb.periodic = 1;
    for (int c = 0; c < 3; c++) { pb.lo[c] = 0; pb.hi[c] = 1; pb.L[c] = 1; }
    cellwork cw;
    memset(&cw, 0, sizeof(cw));
    cw.pb = &pb; cw.i = 0;
    plane_t pl[4];
    cw.pl = pl;
    int s0[3] = {0, 0, 0};
    for (int k = 0; k < 4; k++) make_bisector(&pb, 0, k + 1, s0, &pl[k]);
    cw.np = 3;
    vert_t v;
    make_vertex(&cw, 0, 1, 2, &v);
    /* orient (a,b,c) so that det N > 0, as in the clipper's vertex records */
    if (mode == 1) {
        g_xp_overflow = 0;
        int r = exact_side(&cw, &v, &pl[3]);
        return cw.err ? 99 : r;
    }
    int r = side_of(&cw, &v, &pl[3]);
    return cw.err ? 99 : r;
}

/*
 * oracle_grid_nearest: for every node centre ((a+1/2)/G ... ) of a G^3 grid
 * over the box, subdivided into S^3 sub-points ((a + (u+1/2)/S)/G ...), the
 * index of the nearest particle under the periodic (or plain) metric, ties
 * to the lower index.  Squared distances use the fixed evaluation order
 * fma(dz,dz, fma(dy,dy, dx*dx)) with minimum-image dx.  Brute force over all
 * particles.  out: [G^3][S^3] int64 in x-fastest order of sub-points and of
 * nodes (node (a,b,c) at ((c*G + b)*G + a)).
 */
int oracle_grid_nearest(int64_t N, const double *pos, const double *box_lo, const double *box_hi, int periodic,
                        int G, int S, int64_t *out, int nthreads) {
    double L[3];
    for (int c = 0; c < 3; c++) L[c] = box_hi[c] - box_lo[c];
    int64_t nodes = (int64_t)G * G * G;
    int64_t sub = (int64_t)S * S * S;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < nodes * sub; q++) {
        int64_t node = q / sub, sp = q % sub;
        int a = (int)(node % G), b = (int)((node / G) % G), c = (int)(node / ((int64_t)G * G));
        int u = (int)(sp % S), v = (int)((sp / S) % S), w = (int)(sp / ((int64_t)S * S));
        double g[3];
        g[0] = box_lo[0] + ((double)a + ((double)u + 0.5) / S) * (L[0] / G);
        g[1] = box_lo[1] + ((double)b + ((double)v + 0.5) / S) * (L[1] / G);
        g[2] = box_lo[2] + ((double)c + ((double)w + 0.5) / S) * (L[2] / G);
        double best = INFINITY;
        int64_t bj = -1;
        for (int64_t j = 0; j < N; j++) {
            double d[3];
            for (int k = 0; k < 3; k++) {
                double t = pos[3 * j + k] - g[k];
                if (periodic) {
                    if (t > 0.5 * L[k]) t -= L[k];
                    else if (t < -0.5 * L[k]) t += L[k];
                }
                d[k] = t;
            }
            double d2 = fma(d[2], d[2], fma(d[1], d[1], d[0] * d[0]));
            if (d2 < best) { best = d2; bj = j; }
        }
        out[q] = bj;
    }
    return 0;
}

/*
 * oracle_nearest_points: for each of M query points q (FP64, [M][3]), the index of the nearest particle under
 * the periodic (or plain) metric, ties to the lower index, with the squared distance evaluated exactly as in
 * oracle_grid_nearest.  Brute force over all particles.  out: [M] int64.
 */
int oracle_nearest_points(int64_t N, const double *pos, const double *box_lo, const double *box_hi, int periodic,
                          int64_t M, const double *q, int64_t *out, int nthreads) {
    double L[3];
    for (int c = 0; c < 3; c++) L[c] = box_hi[c] - box_lo[c];
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t m = 0; m < M; m++) {
        double best = INFINITY;
        int64_t bj = -1;
        for (int64_t j = 0; j < N; j++) {
            double d[3];
            for (int k = 0; k < 3; k++) {
                double t = pos[3 * j + k] - q[3 * m + k];
                if (periodic) {
                    if (t > 0.5 * L[k]) t -= L[k];
                    else if (t < -0.5 * L[k]) t += L[k];
                }
                d[k] = t;
            }
            double d2 = fma(d[2], d[2], fma(d[1], d[1], d[0] * d[0]));
            if (d2 < best) { best = d2; bj = j; }
        }
        out[m] = bj;
    }
    return 0;
}

/* FP64 sample point of grid node (a,b,c), sub-point (u,v,w): helper for tests */
void oracle_grid_point(const double *box_lo, const double *box_hi, int G, int S, int64_t node, int64_t sp,
                       double *g) {
    double L[3];
    for (int c = 0; c < 3; c++) L[c] = box_hi[c] - box_lo[c];
    int a = (int)(node % G), b = (int)((node / G) % G), c = (int)(node / ((int64_t)G * G));
    int u = (int)(sp % S), v = (int)((sp / S) % S), w = (int)(sp / ((int64_t)S * S));
    g[0] = box_lo[0] + ((double)a + ((double)u + 0.5) / S) * (L[0] / G);
    g[1] = box_lo[1] + ((double)b + ((double)v + 0.5) / S) * (L[1] / G);
    g[2] = box_lo[2] + ((double)c + ((double)w + 0.5) / S) * (L[2] / G);
}

/*
 * oracle_grid_volume: the volume-weighted average of the cell densities over
 * each voxel of a regular G^3 grid (the exact reading of the Implementation
 * section's average Voronoi densities on a grid):
 *     grid[v] = sum_i dens[i] |V_i intersect voxel v| / |voxel v|,
 * voxel (a, b, c) = [lo + a h, lo + (a+1) h] per axis, h = L / G (FP64), the
 * coordinates computed as lo + a * h; periodic boxes wrap the voxel indices.
 * Each cell is computed as in oracle_cells (certified mode) and clipped, for
 * every voxel that its box meets, by the voxel's six walls with the same
 * exact predicates; the volume of what remains is the overlap.
 *   grid  [G][G][G] out, index (c * G + b) * G + a (x fastest)
 * counters[0..3] as in oracle_cells.  Returns 0 or the first error code.
 */
int oracle_grid_volume(int64_t N, const double *pos, const double *box_lo, const double *box_hi, int periodic,
                       int G, const double *dens, double *grid, int64_t *counters, int nthreads) {
    problem pb;
    pb.N = N; pb.x = pos; pb.periodic = periodic;
    for (int c = 0; c < 3; c++) { pb.lo[c] = box_lo[c]; pb.hi[c] = box_hi[c]; pb.L[c] = box_hi[c] - box_lo[c]; }
    double h[3];
    for (int c = 0; c < 3; c++) h[c] = pb.L[c] / G;
    const int64_t G3 = (int64_t)G * G * G;
    for (int64_t v = 0; v < G3; v++) grid[v] = 0.0;
    kdtree tree;
    kd_build(&tree, &pb);
    int64_t *leaf_of = (int64_t *)malloc(sizeof(int64_t) * (N > 0 ? N : 1));
    for (int64_t n = 0; n < tree.nn; n++)
        if (tree.nd[n].left < 0)
            for (int64_t k = tree.nd[n].a; k < tree.nd[n].b; k++) leaf_of[tree.idx[k]] = n;
    int64_t tot_pred = 0, tot_exact = 0, tot_zero = 0, tot_err = 0;
    int first_err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel reduction(+ : tot_pred, tot_exact, tot_zero, tot_err)
    {
        cellwork cw, cv;
        cw.pb = &pb; cv.pb = &pb;
        cw.pl = (plane_t *)malloc(sizeof(plane_t) * MAXP);
        cw.v = (vert_t *)malloc(sizeof(vert_t) * MAXV);
        cw.tmp = (vert_t *)malloc(sizeof(vert_t) * MAXV);
        cw.side = (int8_t *)malloc(MAXV);
        cv.pl = (plane_t *)malloc(sizeof(plane_t) * MAXP);
        cv.v = (vert_t *)malloc(sizeof(vert_t) * MAXV);
        cv.tmp = (vert_t *)malloc(sizeof(vert_t) * MAXV);
        cv.side = (int8_t *)malloc(MAXV);
        int64_t *f_nbr = (int64_t *)malloc(sizeof(int64_t) * MAXP);
        int32_t *f_shift = (int32_t *)malloc(sizeof(int32_t) * 3 * MAXP);
        double *f_area = (double *)malloc(sizeof(double) * MAXP);
        double *f_cen = (double *)malloc(sizeof(double) * 3 * MAXP);
        double *f_dist = (double *)malloc(sizeof(double) * MAXP);
        candbuf cb = {NULL, 0, 0};
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < N; i++) {
            cw.i = i;
            init_cell(&cw);
            int rc = run_certified(&cw, &tree, &cb, leaf_of[i]);
            tot_pred += cw.n_pred; tot_exact += cw.n_exact; tot_zero += cw.n_zero;
            if (rc != 0) {
                tot_err++;
#pragma omp critical
                { if (!first_err) first_err = rc; }
                continue;
            }
            /* voxel index range of the cell's enclosing box */
            int64_t a0[3], a1[3];
            for (int c = 0; c < 3; c++) {
                double mn = INFINITY, mx = -INFINITY;
                for (int k = 0; k < cw.nv; k++) {
                    mn = fmin(mn, cw.v[k].yi[c].lo);
                    mx = fmax(mx, cw.v[k].yi[c].hi);
                }
                double xi = pos[3 * i + c];
                a0[c] = (int64_t)floor((xi + mn - pb.lo[c]) / h[c]) - 1;
                a1[c] = (int64_t)floor((xi + mx - pb.lo[c]) / h[c]) + 1;
                if (!periodic) {
                    if (a0[c] < 0) a0[c] = 0;
                    if (a1[c] > G - 1) a1[c] = G - 1;
                }
            }
            for (int64_t az = a0[2]; az <= a1[2]; az++)
                for (int64_t ay = a0[1]; ay <= a1[1]; ay++)
                    for (int64_t ax = a0[0]; ax <= a1[0]; ax++) {
                        int64_t ia[3] = {ax, ay, az}, v[3];
                        double sl[3];
                        for (int c = 0; c < 3; c++) {
                            int64_t q = ia[c] % G;
                            if (q < 0) q += G;
                            v[c] = q;
                            sl[c] = (double)((ia[c] - q) / G) * pb.L[c];
                        }
                        /* copy of the cell, clipped by the voxel's six walls */
                        cv.i = i; cv.np = cw.np; cv.nv = cw.nv; cv.err = 0;
                        cv.n_pred = cv.n_exact = cv.n_zero = cv.n_tested = cv.n_cut = 0;
                        memcpy(cv.pl, cw.pl, sizeof(plane_t) * cw.np);
                        memcpy(cv.v, cw.v, sizeof(vert_t) * cw.nv);
                        for (int w = 0; w < 6 && cv.nv > 0 && !cv.err; w++) {
                            int axis = w / 2, upper = (w % 2) == 0;
                            double bnd = pb.lo[axis] + (double)(v[axis] + (upper ? 1 : 0)) * h[axis];
                            plane_t pw;
                            make_voxel_wall(&pb, i, w, bnd, sl[axis], &pw);
                            clip(&cv, &pw);
                        }
                        tot_pred += cv.n_pred; tot_exact += cv.n_exact; tot_zero += cv.n_zero;
                        if (cv.err) {
                            tot_err++;
#pragma omp critical
                            { if (!first_err) first_err = cv.err; }
                            continue;
                        }
                        if (cv.nv == 0) continue;
                        cellout co;
                        memset(&co, 0, sizeof(co));
                        int e = extract(&cv, &co, MAXP, f_nbr, f_shift, f_area, f_cen, f_dist, NULL);
                        if (e) {
                            tot_err++;
#pragma omp critical
                            { if (!first_err) first_err = e; }
                            continue;
                        }
                        int64_t vi = (v[2] * G + v[1]) * G + v[0];
                        double add = dens[i] * co.vol;
#pragma omp atomic
                        grid[vi] += add;
                    }
        }
        free(cw.pl); free(cw.v); free(cw.tmp); free(cw.side);
        free(cv.pl); free(cv.v); free(cv.tmp); free(cv.side);
        free(f_nbr); free(f_shift); free(f_area); free(f_cen); free(f_dist); free(cb.c);
    }
    kd_free(&tree);
    free(leaf_of);
    const double vv = h[0] * h[1] * h[2];
    for (int64_t v = 0; v < G3; v++) grid[v] /= vv;
    counters[0] += tot_pred; counters[1] += tot_exact; counters[2] += tot_zero; counters[3] += tot_err;
    return first_err;
}

int oracle_abi_version(void) { return 1; }
