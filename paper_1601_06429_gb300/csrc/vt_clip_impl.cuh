// vt_clip_impl.cuh -- per-cell Voronoi clipping on sm_103a (hot-path steps A3-A6).
//
// The paper computes the tessellation of each MPI task with Qhull and then,
// for each particle, walks its facets to get the cell volume, the density
// mass/volume and the neighbours sharing a facet (Implementation section).
// Here every cell is computed on its own by one warp:
//
//  * candidates: all particles within a radius r of x_i, from the bucket tree
//    (minimum periodic image), sorted by (|d|^2, index);
//  * clipping: the cell starts as the cube of i's six periodic self-images
//    (or the box walls) and is cut by the bisector plane  d.y <= |d|^2/2  of
//    each candidate in turn.  The polytope is held as its dual triangulation:
//    one triangle (a,b,c) of plane ids per vertex, oriented consistently.  A
//    cut removes the triangles whose vertex lies strictly beyond the plane and
//    adds one triangle (x,y,p) per boundary edge x->y of the removed region;
//  * security radius: a plane with |d| >= 2 R, R the largest vertex distance,
//    cannot cut; candidates are taken in increasing |d| and the cell is final
//    as soon as the next |d| (or the radius r of the pass) reaches 2 R.
//    Otherwise the next pass collects the annulus r <= |d| < 2R;
//  * side predicate: n.v - h for the vertex v of planes (a,b,c) and plane j,
//    evaluated in the working precision with a rigorous forward error bound;
//    undecided tests are redone in FP64 and, in the exact kernel, decided by
//    expansion arithmetic (Shewchuk 1997) on the input coordinates;
//  * emission: facets walked around each plane of the final triangulation;
//    areas, centroids, volume V = sum of site-apex tetrahedra, centroid and
//    second moment of the cell, facet records for the neighbour list,
//    gradient and adjoint kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "vt_internal.cuh"
#include "vt_kernels.cuh"

namespace vt {

constexpr int CLIP_WARPS = 4;
constexpr int CHUNK = 4;
constexpr int EXACT_WS = 12288;  // doubles per warp for expansion arithmetic

template <typename CT> struct Prec;
template <> struct Prec<float> {
    static __device__ __forceinline__ float u() { return 5.9604644775390625e-08f; }  // 2^-24
};
template <> struct Prec<double> {
    static __device__ __forceinline__ double u() { return 1.1102230246251565e-16; }  // 2^-53
};

template <typename P> struct Stor;
template <> struct Stor<float4> { typedef float T; };
template <> struct Stor<dpt4> { typedef double T; };

// ------------------------------------------------------------------ shared memory
template <typename CT>
struct WarpSmem {
    CT pnx[MAXP], pny[MAXP], pnz[MAXP], ph[MAXP], pnrm[MAXP];
    uint32_t psrc[MAXP];
    uint8_t pcode[MAXP];  // 0..26 image shift code, 27+w box wall w
    union {
        unsigned long long cand[CAND_CAP];
        struct {
            uint32_t tid[MAXT];
            CT tx[MAXT], ty[MAXT], tz[MAXT];
            uint32_t hash[HASH_SZ];
            uint32_t first[MAXP];
        } em;
    } u;
    uint16_t edges[3 * MAXT];
    uint16_t bnd[MAXT];
    uint32_t stack[STACK_CAP];
};

// ------------------------------------------------------------------ small helpers
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ unsigned lanemask_lt() { return (1u << lane_id()) - 1u; }

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) { T w = __shfl_xor_sync(0xffffffffu, v, o); v = v > w ? v : w; }
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int code_of(int sx, int sy, int sz) { return (sx + 1) + 3 * (sy + 1) + 9 * (sz + 1); }
__device__ __forceinline__ void shift_of(int code, int& sx, int& sy, int& sz) {
    sx = code % 3 - 1; sy = (code / 3) % 3 - 1; sz = code / 9 - 1;
}

// exact sum a + b as (s, e) (Knuth); no contraction possible with explicit rounding intrinsics
__device__ __forceinline__ void tsum_f(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void tsum_d(double a, double b, double& s, double& e) {
    s = __dadd_rn(a, b);
    double bb = __dsub_rn(s, a);
    e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

// one displacement component x_j - x_i (+ shift) with relative error <= u of the working precision.
// Without a wrap this is one rounded subtraction; with a wrap, x_j - x_i = t + e exactly and t + sL is
// exact (|t| in [L/2, L]), so one rounding remains.
__device__ __forceinline__ float dcomp_f(float xj, float xi, float L, float halfL, int periodic, int& s) {
    float t = __fsub_rn(xj, xi);
    s = 0;
    if (periodic) {
        if (t > halfL) s = -1;
        else if (t < -halfL) s = 1;
        if (s) {
            float e;
            tsum_f(xj, -xi, t, e);
            t = __fadd_rn(__fadd_rn(t, s > 0 ? L : -L), e);
        }
    }
    return t;
}
__device__ __forceinline__ double dcomp_d(double xj, double xi, double L, double halfL, int periodic, int& s) {
    double t = __dsub_rn(xj, xi);
    s = 0;
    if (periodic) {
        if (t > halfL) s = -1;
        else if (t < -halfL) s = 1;
        if (s) {
            double e;
            tsum_d(xj, -xi, t, e);
            t = __dadd_rn(__dadd_rn(t, s > 0 ? L : -L), e);
        }
    }
    return t;
}
// component with a given shift (FP64), same rounding as dcomp_d
__device__ __forceinline__ double dcomp_shift_d(double xj, double xi, double L, int s) {
    if (s == 0) return __dsub_rn(xj, xi);
    double t, e;
    tsum_d(xj, -xi, t, e);
    return __dadd_rn(__dadd_rn(t, s > 0 ? L : -L), e);
}

template <typename CT> __device__ __forceinline__ CT f_fma(CT a, CT b, CT c);
template <> __device__ __forceinline__ float f_fma<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ double f_fma<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

// displacement of particle j seen from i in precision CT, and the periodic shift used
template <typename P, typename CT> struct DispF;
template <> struct DispF<float4, float> {
    static __device__ __forceinline__ void get(const float4& pj, const float4& pi, const Geometry& g, float& dx,
                                               float& dy, float& dz, int& code) {
        int sx, sy, sz;
        dx = dcomp_f(pj.x, pi.x, g.Lf[0], g.halfLf[0], g.periodic, sx);
        dy = dcomp_f(pj.y, pi.y, g.Lf[1], g.halfLf[1], g.periodic, sy);
        dz = dcomp_f(pj.z, pi.z, g.Lf[2], g.halfLf[2], g.periodic, sz);
        code = code_of(sx, sy, sz);
    }
};
template <typename P> struct DispF<P, double> {
    static __device__ __forceinline__ void get(const P& pj, const P& pi, const Geometry& g, double& dx, double& dy,
                                               double& dz, int& code) {
        int sx, sy, sz;
        dx = dcomp_d((double)pj.x, (double)pi.x, g.L[0], 0.5 * g.L[0], g.periodic, sx);
        dy = dcomp_d((double)pj.y, (double)pi.y, g.L[1], 0.5 * g.L[1], g.periodic, sy);
        dz = dcomp_d((double)pj.z, (double)pi.z, g.L[2], 0.5 * g.L[2], g.periodic, sz);
        code = code_of(sx, sy, sz);
    }
};
template <> struct DispF<dpt4, float> {
    static __device__ __forceinline__ void get(const dpt4& pj, const dpt4& pi, const Geometry& g, float& dx,
                                               float& dy, float& dz, int& code) {
        double a, b, c;
        DispF<dpt4, double>::get(pj, pi, g, a, b, c, code);
        dx = (float)a; dy = (float)b; dz = (float)c;
    }
};

// ------------------------------------------------------------------ vertices
// Vertex of planes A,B,C (n.y <= h) by Cramer's rule and a bound on its distance to the vertex of the
// exact planes.  Inputs carry relative errors <= u (components of n) and <= 6u (h).  With
// S = |nb||nc| + |nc||na| + |na||nb|, H = ha + hb + hc, P = |na||nb||nc|:
//   |v - v*| <= 2 [12u S H + u |v| (S (|na|+|nb|+|nc|) + 6P)] / (|det| - 6uP) + 2u|v|
// (perturbation of the 3x3 system plus the rounding of the evaluation, doubled for second-order terms).
// Returns ev = that bound + 8u|v| (so that a plane test only adds nrm*ev + 16u h) and
// rr >= (|v*|)^2 for the security radius; ill-conditioned vertices get ev = +inf.
template <typename CT>
__device__ __forceinline__ void make_vertex(CT ax, CT ay, CT az, CT ah, CT an, CT bx, CT by, CT bz, CT bh, CT bn,
                                            CT cx, CT cy, CT cz, CT ch, CT cn, CT& vx, CT& vy, CT& vz, CT& ev,
                                            CT& rr) {
    const CT u = Prec<CT>::u();
    CT bcx = f_fma<CT>(by, cz, -bz * cy), bcy = f_fma<CT>(bz, cx, -bx * cz), bcz = f_fma<CT>(bx, cy, -by * cx);
    CT cax = f_fma<CT>(cy, az, -cz * ay), cay = f_fma<CT>(cz, ax, -cx * az), caz = f_fma<CT>(cx, ay, -cy * ax);
    CT abx = f_fma<CT>(ay, bz, -az * by), aby = f_fma<CT>(az, bx, -ax * bz), abz = f_fma<CT>(ax, by, -ay * bx);
    CT det = f_fma<CT>(ax, bcx, f_fma<CT>(ay, bcy, az * bcz));
    CT wx = f_fma<CT>(ah, bcx, f_fma<CT>(bh, cax, ch * abx));
    CT wy = f_fma<CT>(ah, bcy, f_fma<CT>(bh, cay, ch * aby));
    CT wz = f_fma<CT>(ah, bcz, f_fma<CT>(bh, caz, ch * abz));
    CT inv = (CT)1 / det;
    vx = wx * inv; vy = wy * inv; vz = wz * inv;
    CT vn = sqrt(f_fma<CT>(vz, vz, f_fma<CT>(vy, vy, vx * vx)));
    CT S = bn * cn + cn * an + an * bn;
    CT H = ah + bh + ch;
    CT P = an * bn * cn;
    CT ad = fabs(det) - (CT)6 * u * P;
    if (!(ad > (CT)32 * u * P)) {
        ev = (CT)INFINITY;
        rr = (CT)INFINITY;
        return;
    }
    CT e = (CT)2 * ((CT)12 * u * S * H + u * vn * (S * (an + bn + cn) + (CT)6 * P)) / ad + (CT)2 * u * vn;
    e = e * (CT)(1.0 + 1e-3);
    ev = e + (CT)8 * u * vn;
    CT r = (vn * ((CT)1 + (CT)4 * u) + e);
    rr = r * r * ((CT)1 + (CT)4 * u);
}

// ------------------------------------------------------------------ exact predicate (device)
// Expansions: arrays of doubles, nonoverlapping, increasing magnitude (Shewchuk 1997).  The sign of the
// 4x4 lifted determinant is taken by Laplace expansion over the complementary 2x2 minors of columns
// (x,y) and (z,w); det N (3x3) reuses the (x,y) minors.  Workspace: per-warp global scratch, bump
// allocated; every operation checks its capacity.
struct XWork {
    double* base;
    int used, cap;
    bool overflow;
};
struct Xe {
    double* c;
    int n, cap;
};
__device__ __forceinline__ Xe x_alloc(XWork& w, int cap) {
    Xe e;
    e.n = 0;
    if (w.used + cap > w.cap) {
        w.overflow = true;
        e.c = w.base;
        e.cap = 0;
        return e;
    }
    e.c = w.base + w.used;
    e.cap = cap;
    w.used += cap;
    return e;
}
// e += b exactly, zero-eliminating (Grow-Expansion)
static __device__ void x_grow(XWork& w, Xe& e, double b) {
    double q = b;
    int m = 0;
    for (int i = 0; i < e.n; i++) {
        double s, t;
        tsum_d(q, e.c[i], s, t);
        if (t != 0.0) e.c[m++] = t;
        q = s;
    }
    if (q != 0.0) {
        if (m >= e.cap) { w.overflow = true; e.n = m; return; }
        e.c[m++] = q;
    }
    e.n = m;
}
// out = a * b (sign applied), accumulated term by term
static __device__ void x_mul_into(XWork& w, Xe& out, const Xe& a, const Xe& b, bool neg) {
    for (int i = 0; i < a.n; i++)
        for (int k = 0; k < b.n; k++) {
            double p = __dmul_rn(a.c[i], b.c[k]);
            double e = __fma_rn(a.c[i], b.c[k], -p);
            if (neg) { p = -p; e = -e; }
            x_grow(w, out, e);
            x_grow(w, out, p);
        }
}
__device__ __forceinline__ int x_sign(const Xe& e) {
    if (e.n == 0) return 0;
    double t = e.c[e.n - 1];
    return (t > 0) - (t < 0);
}

struct PRef {
    uint32_t src;
    int code;
};

// exact row (n_x, n_y, n_z, w) of a plane, positively scaled: bisector -> (2d, |d|^2), wall -> (n, h)
template <typename P>
__device__ void x_row(XWork& w, Xe row[4], const P* spos, const Geometry& g, uint32_t self, PRef r) {
    P pi = spos[self];
    double xi[3] = {(double)pi.x, (double)pi.y, (double)pi.z};
    if (r.code < 27) {
        P pj = spos[r.src];
        double xj[3] = {(double)pj.x, (double)pj.y, (double)pj.z};
        int s[3];
        shift_of(r.code, s[0], s[1], s[2]);
        Xe d[3];
        row[3] = x_alloc(w, 96);
        for (int c = 0; c < 3; c++) {
            d[c] = x_alloc(w, 4);
            x_grow(w, d[c], xj[c]);
            if (s[c]) x_grow(w, d[c], s[c] > 0 ? g.L[c] : -g.L[c]);
            x_grow(w, d[c], -xi[c]);
            row[c] = x_alloc(w, 4);
            for (int k = 0; k < d[c].n; k++) x_grow(w, row[c], 2.0 * d[c].c[k]);
            x_mul_into(w, row[3], d[c], d[c], false);
        }
    } else {
        int wall = r.code - 27, axis = wall >> 1;
        bool upper = (wall & 1) == 0;
        for (int c = 0; c < 3; c++) {
            row[c] = x_alloc(w, 1);
            if (c == axis) x_grow(w, row[c], upper ? 1.0 : -1.0);
        }
        row[3] = x_alloc(w, 3);
        if (upper) { x_grow(w, row[3], g.hi[axis]); x_grow(w, row[3], -xi[axis]); }
        else { x_grow(w, row[3], xi[axis]); x_grow(w, row[3], -g.lo[axis]); }
    }
}

// +1: vertex of (a,b,c) strictly beyond plane j; -1: strictly inside; 0: on it.  *ovf on workspace overflow.
template <typename P>
__device__ int exact_side(double* ws, const P* spos, const Geometry& g, uint32_t self, PRef a, PRef b, PRef c, PRef j,
                          bool* ovf) {
    XWork w;
    w.base = ws; w.used = 0; w.cap = EXACT_WS; w.overflow = false;
    Xe R[4][4];
    x_row<P>(w, R[0], spos, g, self, a);
    x_row<P>(w, R[1], spos, g, self, b);
    x_row<P>(w, R[2], spos, g, self, c);
    x_row<P>(w, R[3], spos, g, self, j);
    if (w.overflow) { *ovf = true; return 0; }
    // (x,y) minors for all row pairs and (z,w) minors for the complementary pairs
    const int pp[6] = {0, 0, 0, 1, 1, 2}, qq[6] = {1, 2, 3, 2, 3, 3};
    Xe m01[6];
    for (int k = 0; k < 6; k++) {
        const Xe* A = R[pp[k]];
        const Xe* B = R[qq[k]];
        m01[k] = x_alloc(w, 2 * A[0].n * B[1].n + 2 * A[1].n * B[0].n + 2);
        x_mul_into(w, m01[k], A[0], B[1], false);
        x_mul_into(w, m01[k], A[1], B[0], true);
    }
    Xe D = x_alloc(w, 1536);
    // Laplace: det = sum_{p<q} (-1)^(p+q+1) M01(p,q) M23(complement)
    for (int k = 0; k < 6; k++) {
        int p = pp[k], q = qq[k];
        int r0 = -1, r1 = -1;
        for (int r = 0; r < 4; r++)
            if (r != p && r != q) { if (r0 < 0) r0 = r; else r1 = r; }
        const Xe* A = R[r0];
        const Xe* B = R[r1];
        int save = w.used;
        Xe m23 = x_alloc(w, 2 * A[2].n * B[3].n + 2 * A[3].n * B[2].n + 2);
        x_mul_into(w, m23, A[2], B[3], false);
        x_mul_into(w, m23, A[3], B[2], true);
        bool neg = ((p + q + 1) & 1) != 0;
        x_mul_into(w, D, m01[k], m23, neg);
        w.used = save;
        if (w.overflow) break;
    }
    // det N over rows 0,1,2: n0z M01(1,2) - n1z M01(0,2) + n2z M01(0,1)
    Xe dn = x_alloc(w, 2 * (R[0][2].n * m01[3].n + R[1][2].n * m01[1].n + R[2][2].n * m01[0].n) + 2);
    x_mul_into(w, dn, R[0][2], m01[3], false);
    x_mul_into(w, dn, R[1][2], m01[1], true);
    x_mul_into(w, dn, R[2][2], m01[0], false);
    if (w.overflow) { *ovf = true; return 0; }
    int sd = x_sign(D), sn = x_sign(dn);
    return -sd * sn;
}

// FP64 side test of the vertex of planes (a,b,c) against plane j from the input coordinates:
// +1 / -1 when decided, 0 when the error bound does not decide.
template <typename P>
__device__ void plane64(const P* spos, const Geometry& g, uint32_t self, PRef r, double& nx, double& ny, double& nz,
                        double& h, double& nrm) {
    P pi = spos[self];
    if (r.code < 27) {
        P pj = spos[r.src];
        int sx, sy, sz;
        shift_of(r.code, sx, sy, sz);
        nx = dcomp_shift_d((double)pj.x, (double)pi.x, g.L[0], sx);
        ny = dcomp_shift_d((double)pj.y, (double)pi.y, g.L[1], sy);
        nz = dcomp_shift_d((double)pj.z, (double)pi.z, g.L[2], sz);
        h = 0.5 * __fma_rn(nz, nz, __fma_rn(ny, ny, nx * nx));
        nrm = sqrt(2.0 * h);
    } else {
        int wall = r.code - 27, axis = wall >> 1;
        bool upper = (wall & 1) == 0;
        double xi = axis == 0 ? (double)pi.x : axis == 1 ? (double)pi.y : (double)pi.z;
        nx = ny = nz = 0.0;
        double sgn = upper ? 1.0 : -1.0;
        if (axis == 0) nx = sgn; else if (axis == 1) ny = sgn; else nz = sgn;
        h = upper ? __dsub_rn(g.hi[axis], xi) : __dsub_rn(xi, g.lo[axis]);
        nrm = 1.0;
    }
}

template <typename P>
__device__ int side64(const P* spos, const Geometry& g, uint32_t self, PRef a, PRef b, PRef c, PRef j) {
    double ax, ay, az, ah, an, bx, by, bz, bh, bn, cx, cy, cz, chh, cn, jx, jy, jz, jh, jn;
    plane64<P>(spos, g, self, a, ax, ay, az, ah, an);
    plane64<P>(spos, g, self, b, bx, by, bz, bh, bn);
    plane64<P>(spos, g, self, c, cx, cy, cz, chh, cn);
    plane64<P>(spos, g, self, j, jx, jy, jz, jh, jn);
    double vx, vy, vz, ev, rr;
    make_vertex<double>(ax, ay, az, ah, an, bx, by, bz, bh, bn, cx, cy, cz, chh, cn, vx, vy, vz, ev, rr);
    double s = __fma_rn(jx, vx, __fma_rn(jy, vy, __fma_rn(jz, vz, -jh)));
    double bound = jn * ev + 16.0 * Prec<double>::u() * jh;
    if (s > bound) return 1;
    if (s < -bound) return -1;
    return 0;
}

// ------------------------------------------------------------------ per-cell state
template <typename CT>
struct Tris {
    uint32_t id[TPL];
    CT x[TPL], y[TPL], z[TPL], ev[TPL], rr[TPL];
    unsigned vm[TPL];  // warp-uniform validity masks (bit = lane)
};

enum { R_OK = 0, R_NEED_EXACT = 1 };

struct CellCounters {
    unsigned n_cut, n_tested, n_passes, n_fp64, n_exact, n_zero;
};

template <typename CT>
__device__ __forceinline__ void set_plane(WarpSmem<CT>& S, int p, CT nx, CT ny, CT nz, CT h, CT nrm, uint32_t src,
                                          int code) {
    if (lane_id() == 0) {
        S.pnx[p] = nx; S.pny[p] = ny; S.pnz[p] = nz; S.ph[p] = h; S.pnrm[p] = nrm;
        S.psrc[p] = src; S.pcode[p] = (uint8_t)code;
    }
}

template <typename CT>
__device__ __forceinline__ void vertex_from_planes(const WarpSmem<CT>& S, int a, int b, int c, CT& vx, CT& vy, CT& vz,
                                                   CT& ev, CT& rr) {
    make_vertex<CT>(S.pnx[a], S.pny[a], S.pnz[a], S.ph[a], S.pnrm[a], S.pnx[b], S.pny[b], S.pnz[b], S.ph[b], S.pnrm[b],
                    S.pnx[c], S.pny[c], S.pnz[c], S.ph[c], S.pnrm[c], vx, vy, vz, ev, rr);
}

// Clip by a candidate plane.  Returns 0 (no cut), 1 (cut), R_NEED_EXACT encoded as 2, or a VT_ERR_* (<0).
template <typename P, typename CT, bool EXACT>
__device__ int clip_plane(WarpSmem<CT>& S, Tris<CT>& T, int& np, CT nx, CT ny, CT nz, CT h, CT nrm, uint32_t src,
                          int code, const P* spos, const Geometry& g, uint32_t self, double* xws, CellCounters& cc) {
    const unsigned lane = lane_id();
    const CT u = Prec<CT>::u();
    const CT hb = (CT)16 * u * h;
    bool out[TPL];
    bool unc_any = false;
#pragma unroll
    for (int e = 0; e < TPL; e++) {
        out[e] = false;
        if ((T.vm[e] >> lane) & 1u) {
            CT s = f_fma<CT>(nx, T.x[e], f_fma<CT>(ny, T.y[e], f_fma<CT>(nz, T.z[e], -h)));
            CT bound = f_fma<CT>(nrm, T.ev[e], hb);
            if (s > bound) out[e] = true;
            else if (!(s < -bound)) unc_any = true;  // also catches NaN / inf bounds
        }
    }
    if (__any_sync(0xffffffffu, unc_any)) {
        // undecided tests: FP64 from the input coordinates (FP32 kernels), then exactly (exact kernel)
        bool need_exact = false;
        bool pend[TPL];
#pragma unroll
        for (int e = 0; e < TPL; e++) {
            pend[e] = false;
            if ((T.vm[e] >> lane) & 1u) {
                CT s = f_fma<CT>(nx, T.x[e], f_fma<CT>(ny, T.y[e], f_fma<CT>(nz, T.z[e], -h)));
                CT bound = f_fma<CT>(nrm, T.ev[e], hb);
                if (!(s > bound) && !(s < -bound)) {
                    int sd = 0;
                    if (sizeof(CT) == 4) {
                        uint32_t id = T.id[e];
                        int a = id & 255, b = (id >> 8) & 255, c = (id >> 16) & 255;
                        PRef ra = {S.psrc[a], S.pcode[a]}, rb = {S.psrc[b], S.pcode[b]}, rc = {S.psrc[c], S.pcode[c]};
                        PRef rj = {src, code};
                        sd = side64<P>(spos, g, self, ra, rb, rc, rj);
                        cc.n_fp64++;
                    }
                    if (sd != 0) out[e] = (sd > 0);
                    else if (EXACT) pend[e] = true;
                    else need_exact = true;
                }
            }
        }
        if (!EXACT) {
            if (__any_sync(0xffffffffu, need_exact)) return 2;
        } else {
            bool mine = false;
#pragma unroll
            for (int e = 0; e < TPL; e++) mine |= pend[e];
            unsigned todo = __ballot_sync(0xffffffffu, mine);
            bool ovf_any = false;
            while (todo) {
                int L = __ffs(todo) - 1;
                if ((int)lane == L) {  // one lane at a time owns the warp's workspace
#pragma unroll
                    for (int e = 0; e < TPL; e++) {
                        if (pend[e]) {
                            uint32_t id = T.id[e];
                            int a = id & 255, b = (id >> 8) & 255, c = (id >> 16) & 255;
                            PRef ra = {S.psrc[a], S.pcode[a]}, rb = {S.psrc[b], S.pcode[b]},
                                 rc = {S.psrc[c], S.pcode[c]};
                            PRef rj = {src, code};
                            bool ovf = false;
                            int sd = exact_side<P>(xws, spos, g, self, ra, rb, rc, rj, &ovf);
                            cc.n_exact++;
                            if (ovf) ovf_any = true;
                            if (sd == 0) cc.n_zero++;
                            out[e] = (sd > 0);
                        }
                    }
                }
                __syncwarp();
                todo &= todo - 1;
            }
            if (__any_sync(0xffffffffu, ovf_any)) return VT_ERR_NUMERIC;
        }
    }
    // which slots are removed
    unsigned om[TPL];
    bool any = false;
#pragma unroll
    for (int e = 0; e < TPL; e++) {
        om[e] = __ballot_sync(0xffffffffu, out[e]);
        any |= (om[e] != 0);
    }
    if (!any) return 0;
    if (np >= MAXP) return VT_ERR_CAPACITY;
    const int p = np++;
    set_plane<CT>(S, p, nx, ny, nz, h, nrm, src, code);
    // directed edges of the removed triangles
    int nE = 0;
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int e = 0; e < TPL; e++) {
        if (om[e]) {
            if (out[e]) {
                int o = nE + 3 * __popc(om[e] & lt);
                uint32_t id = T.id[e];
                uint32_t a = id & 255, b = (id >> 8) & 255, c = (id >> 16) & 255;
                S.edges[o + 0] = (uint16_t)((a << 8) | b);
                S.edges[o + 1] = (uint16_t)((b << 8) | c);
                S.edges[o + 2] = (uint16_t)((c << 8) | a);
            }
            nE += 3 * __popc(om[e]);
            T.vm[e] &= ~om[e];
        }
    }
    __syncwarp();
    // boundary edges: directed edges whose reverse is not among them
    int nB = 0;
    for (int k0 = 0; k0 < nE; k0 += 32) {
        int k = k0 + (int)lane;
        bool bnd = false;
        uint16_t ed = 0;
        if (k < nE) {
            ed = S.edges[k];
            uint16_t rev = (uint16_t)((ed >> 8) | ((ed & 255) << 8));
            bnd = true;
            for (int q = 0; q < nE; q++)
                if (S.edges[q] == rev) { bnd = false; break; }
        }
        unsigned bm = __ballot_sync(0xffffffffu, bnd);
        if (bnd) {
            int o = nB + __popc(bm & lt);
            if (o < MAXT) S.bnd[o] = ed;
        }
        nB += __popc(bm);
    }
    __syncwarp();
    if (nB > MAXT) return VT_ERR_CAPACITY;
    // new triangles (x, y, p) into the lowest free slots
    int placed = 0;
#pragma unroll
    for (int e = 0; e < TPL; e++) {
        unsigned fm = ~T.vm[e];
        int rank = placed + __popc(fm & lt);
        bool mine = ((fm >> lane) & 1u) && rank < nB;
        if (mine) {
            uint16_t ed = S.bnd[rank];
            int x = ed >> 8, y = ed & 255;
            T.id[e] = (uint32_t)x | ((uint32_t)y << 8) | ((uint32_t)p << 16);
            vertex_from_planes<CT>(S, x, y, p, T.x[e], T.y[e], T.z[e], T.ev[e], T.rr[e]);
        }
        unsigned nm = __ballot_sync(0xffffffffu, mine);
        T.vm[e] |= nm;
        placed += __popc(fm);
    }
    if (placed < nB) return VT_ERR_CAPACITY;
    cc.n_cut++;
    return 1;
}

template <typename CT>
__device__ __forceinline__ CT rmax2(const Tris<CT>& T) {
    CT r = 0;
    const unsigned lane = lane_id();
#pragma unroll
    for (int e = 0; e < TPL; e++)
        if ((T.vm[e] >> lane) & 1u) r = r > T.rr[e] ? r : T.rr[e];
    return warp_max<CT>(r);
}

// ------------------------------------------------------------------ tree search
__device__ __forceinline__ float axis_gap(float q, float lo, float hi, float L, int periodic) {
    float d = fmaxf(fmaxf(lo - q, q - hi), 0.f);
    if (periodic) {
        d = fminf(d, fmaxf(lo + L - q, 0.f));
        d = fminf(d, fmaxf(q + L - hi, 0.f));
    }
    return d;
}

// Collect sorted indices j != self with rlo2 <= |d|^2 < rhi2 (the same |d|^2 as the clipping loop).
// Returns the count, or -1 if more than CAND_CAP, or -2 on stack overflow.
template <typename P, typename CT>
__device__ int collect(WarpSmem<CT>& S, const P* spos, int64_t N, const Geometry& g, const Tree& t, uint32_t self,
                       const P& pi, CT rlo2, CT rhi2) {
    const unsigned lane = lane_id(), lt = lanemask_lt();
    // conservative float radius for box pruning
    float rad = (float)sqrt((double)rhi2) * 1.0001f + 1e-30f;
    float rad2 = rad * rad;
    float qx = (float)pi.x, qy = (float)pi.y, qz = (float)pi.z;
    // float rounding of q: widen by one ulp of the box scale
    float slack = 2.0f * 1.2e-7f * fmaxf(fmaxf(fabsf(g.hif[0]), fabsf(g.lof[0])),
                                         fmaxf(fmaxf(fabsf(g.hif[1]), fabsf(g.lof[1])),
                                               fmaxf(fabsf(g.hif[2]), fabsf(g.lof[2]))));
    int sp = 0;
    int top = t.levels;
    {
        int64_t nt = t.count[top];
        bool hit = false;
        if ((int64_t)lane < nt) {
            float4 lo = t.lo[t.off[top] + lane], hi = t.hi[t.off[top] + lane];
            float dx = fmaxf(axis_gap(qx, lo.x, hi.x, g.Lf[0], g.periodic) - slack, 0.f);
            float dy = fmaxf(axis_gap(qy, lo.y, hi.y, g.Lf[1], g.periodic) - slack, 0.f);
            float dz = fmaxf(axis_gap(qz, lo.z, hi.z, g.Lf[2], g.periodic) - slack, 0.f);
            hit = dx * dx + dy * dy + dz * dz <= rad2;
        }
        unsigned m = __ballot_sync(0xffffffffu, hit);
        if (hit) S.stack[__popc(m & lt)] = ((uint32_t)top << 27) | lane;
        sp = __popc(m);
    }
    __syncwarp();
    int count = 0;
    while (sp > 0) {
        uint32_t ent = S.stack[sp - 1];
        sp--;
        __syncwarp();
        int lvl = ent >> 27;
        int64_t node = ent & ((1u << 27) - 1);
        if (lvl == 1) {
            int64_t j = node * 32 + lane;
            bool hit = false;
            unsigned long long key = 0ull;
            if (j < N && (uint32_t)j != self) {
                P pj = spos[j];
                CT dx, dy, dz;
                int code;
                DispF<P, CT>::get(pj, pi, g, dx, dy, dz, code);
                CT d2 = f_fma<CT>(dz, dz, f_fma<CT>(dy, dy, dx * dx));
                hit = (d2 >= rlo2) && (d2 < rhi2);
                // order-preserving key: d2 >= 0 so its float bits sort like the value; FP64 values are
                // rounded down so that a key never exceeds the |d|^2 it stands for
                float kf = (sizeof(CT) == 4) ? (float)d2 : __double2float_rd((double)d2);
                key = ((unsigned long long)__float_as_uint(kf) << 32) | (uint32_t)j;
            }
            unsigned m = __ballot_sync(0xffffffffu, hit);
            int o = count + __popc(m & lt);
            if (hit && o < CAND_CAP) S.u.cand[o] = key;
            count += __popc(m);
            if (count > CAND_CAP) return -1;
        } else {
            int cl = lvl - 1;
            int64_t c = node * 32 + lane;
            bool hit = false;
            if (c < t.count[cl]) {
                float4 lo = t.lo[t.off[cl] + c], hi = t.hi[t.off[cl] + c];
                float dx = fmaxf(axis_gap(qx, lo.x, hi.x, g.Lf[0], g.periodic) - slack, 0.f);
                float dy = fmaxf(axis_gap(qy, lo.y, hi.y, g.Lf[1], g.periodic) - slack, 0.f);
                float dz = fmaxf(axis_gap(qz, lo.z, hi.z, g.Lf[2], g.periodic) - slack, 0.f);
                hit = dx * dx + dy * dy + dz * dz <= rad2;
            }
            unsigned m = __ballot_sync(0xffffffffu, hit);
            if (sp + __popc(m) > STACK_CAP) return -2;
            if (hit) S.stack[sp + __popc(m & lt)] = ((uint32_t)cl << 27) | (uint32_t)c;
            sp += __popc(m);
            __syncwarp();
        }
    }
    return count;
}

// bitonic sort of S.u.cand[0..n) (padded to a power of two with +inf keys)
template <typename CT>
__device__ void sort_cand(WarpSmem<CT>& S, int n) {
    const unsigned lane = lane_id();
    int m = 1;
    while (m < n) m <<= 1;
    if (m < 2) return;
    for (int k = n + (int)lane; k < m; k += 32) S.u.cand[k] = ~0ull;
    __syncwarp();
    for (int k = 2; k <= m; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int i = (int)lane; i < m; i += 32) {
                int ixj = i ^ jj;
                if (ixj > i) {
                    unsigned long long a = S.u.cand[i], b = S.u.cand[ixj];
                    bool asc = (i & k) == 0;
                    if ((a > b) == asc) { S.u.cand[i] = b; S.u.cand[ixj] = a; }
                }
            }
            __syncwarp();
        }
    }
}

// ------------------------------------------------------------------ the cell
constexpr int RC_NEED_EXACT = 1000;
constexpr int RC_POOL = 1001;

// successor of triangle t around plane p: the triangle holding the directed edge p -> (corner before p in t)
template <typename CT>
__device__ __forceinline__ uint32_t succ_tri(const WarpSmem<CT>& S, uint32_t t, int p) {
    uint32_t id = S.u.em.tid[t];
    uint32_t a = id & 255, b = (id >> 8) & 255, c = (id >> 16) & 255;
    uint32_t before = (a == (uint32_t)p) ? c : (b == (uint32_t)p) ? a : b;
    uint32_t key = ((uint32_t)p << 8) | before;
    uint32_t hsh = (key * 2654435761u) >> 23;
    for (int probe = 0; probe < HASH_SZ; probe++) {
        uint32_t ent = S.u.em.hash[hsh];
        if (ent == 0xffffffffu) return 0xffffffffu;
        if ((ent >> 8) == key) return ent & 255;
        hsh = (hsh + 1) & (HASH_SZ - 1);
    }
    return 0xffffffffu;
}

template <typename P, typename CT, bool EXACT>
__device__ int do_cell(WarpSmem<CT>& S, const ClipArgs& A, uint32_t self, double* xws, CellCounters& cc) {
    const P* spos = (const P*)A.spos;
    const Geometry& g = A.geo;
    const unsigned lane = lane_id(), lt = lanemask_lt();
    const CT u = Prec<CT>::u();
    const P pi = spos[self];
    Tris<CT> T;
#pragma unroll
    for (int e = 0; e < TPL; e++) T.vm[e] = 0u;
    int np = 6;
    // initial planes: periodic self-images (+x,-x,+y,-y,+z,-z) or box walls
    if (lane < 6) {
        int axis = lane >> 1;
        bool upper = (lane & 1) == 0;
        CT nx = 0, ny = 0, nz = 0, h, nrm;
        int code;
        if (g.periodic) {
            CT Lc = (CT)g.L[axis];
            CT sg = upper ? Lc : -Lc;
            if (axis == 0) nx = sg; else if (axis == 1) ny = sg; else nz = sg;
            h = (CT)(0.5 * g.L[axis] * g.L[axis]);
            nrm = Lc;
            int s[3] = {0, 0, 0};
            s[axis] = upper ? 1 : -1;
            code = (s[0] + 1) + 3 * (s[1] + 1) + 9 * (s[2] + 1);
        } else {
            CT sg = upper ? (CT)1 : (CT)-1;
            if (axis == 0) nx = sg; else if (axis == 1) ny = sg; else nz = sg;
            double xi = axis == 0 ? (double)pi.x : axis == 1 ? (double)pi.y : (double)pi.z;
            h = (CT)(upper ? (g.hi[axis] - xi) : (xi - g.lo[axis]));
            nrm = (CT)1;
            code = 27 + (int)lane;
        }
        S.pnx[lane] = nx; S.pny[lane] = ny; S.pnz[lane] = nz; S.ph[lane] = h; S.pnrm[lane] = nrm;
        S.psrc[lane] = self; S.pcode[lane] = (uint8_t)code;
    }
    __syncwarp();
    // 8 corners: plane ids upper x=0/lower x=1, y 2/3, z 4/5; orientation (X,Y,Z) if the sign product is
    // positive, else (X,Z,Y): every triangle then lists its planes counter-clockwise seen from outside
    if (lane < 8) {
        int sx = (lane & 1) ? -1 : 1, sy = (lane & 2) ? -1 : 1, sz = (lane & 4) ? -1 : 1;
        uint32_t X = (lane & 1) ? 1 : 0, Y = (lane & 2) ? 3 : 2, Z = (lane & 4) ? 5 : 4;
        uint32_t id = (sx * sy * sz > 0) ? (X | (Y << 8) | (Z << 16)) : (X | (Z << 8) | (Y << 16));
        T.id[0] = id;
        vertex_from_planes<CT>(S, id & 255, (id >> 8) & 255, (id >> 16) & 255, T.x[0], T.y[0], T.z[0], T.ev[0],
                               T.rr[0]);
    }
    T.vm[0] = 0xFFu;
    CT R2 = rmax2<CT>(T);

    // first radius from the bucket mates: 1.6 x the distance of the ~12th nearest
    CT rhi2;
    {
        int64_t b0 = ((int64_t)self / 32) * 32;
        int64_t j = b0 + lane;
        float d2f = INFINITY;
        if (j < A.N && (uint32_t)j != self) {
            P pj = spos[j];
            CT dx, dy, dz;
            int code;
            DispF<P, CT>::get(pj, pi, g, dx, dy, dz, code);
            d2f = (float)f_fma<CT>(dz, dz, f_fma<CT>(dy, dy, dx * dx));
        }
        // bitonic sort across lanes (ascending)
        for (int k = 2; k <= 32; k <<= 1)
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                float o = __shfl_xor_sync(0xffffffffu, d2f, jj);
                bool up = ((lane & k) == 0);
                bool lower = (lane & jj) == 0;
                float mn = fminf(d2f, o), mx = fmaxf(d2f, o);
                d2f = (lower == up) ? mn : mx;
            }
        int kk = min(max(A.k_target / 4, 4), 30);
        float dk = __shfl_sync(0xffffffffu, d2f, kk);
        if (!(dk < INFINITY)) {
            // fewer mates than needed: the largest finite one, else a mean-spacing guess
            float mx = d2f < INFINITY ? d2f : 0.f;
            mx = warp_max<float>(mx);
            if (mx > 0.f) dk = mx;
            else {
                double vol = g.L[0] * g.L[1] * g.L[2];
                double sp = cbrt(vol / (double)A.N);
                dk = (float)(4.0 * sp * sp);
            }
        }
        rhi2 = (CT)dk * (CT)2.6;
    }
    CT rlo2 = 0;
    CT cap2 = g.periodic ? (CT)(0.249 * fmin(g.L[0], fmin(g.L[1], g.L[2])) * fmin(g.L[0], fmin(g.L[1], g.L[2])))
                         : (CT)(4.0 * (g.L[0] * g.L[0] + g.L[1] * g.L[1] + g.L[2] * g.L[2]));
    bool done = false;
    for (int pass = 0; pass < A.max_passes && !done; pass++) {
        cc.n_passes++;
        if (rhi2 > cap2) rhi2 = cap2;
        int cnt = -1;
        for (int shrink = 0; shrink < 40; shrink++) {
            cnt = collect<P, CT>(S, spos, A.N, g, A.tree, self, pi, rlo2, rhi2);
            if (cnt == -2) return VT_ERR_CAPACITY;
            if (cnt >= 0) break;
            rhi2 = rlo2 + (rhi2 - rlo2) * (CT)0.5;
        }
        if (cnt < 0) return VT_ERR_CAPACITY;
        __syncwarp();
        sort_cand<CT>(S, cnt);
        // clip in increasing distance
        for (int k = 0; k < cnt; k++) {
            unsigned long long key = S.u.cand[k];
            uint32_t j = (uint32_t)(key & 0xffffffffu);
            float kf = __uint_as_float((uint32_t)(key >> 32));
            if ((CT)kf * ((CT)1 - (CT)8 * u) > (CT)4 * R2) { done = true; break; }
            P pj = spos[j];
            CT dx, dy, dz;
            int code;
            DispF<P, CT>::get(pj, pi, g, dx, dy, dz, code);
            CT d2 = f_fma<CT>(dz, dz, f_fma<CT>(dy, dy, dx * dx));
            if (d2 == (CT)0) return VT_ERR_DUPLICATE;
            CT h = (CT)0.5 * d2;
            CT nrm = sqrt(d2);
            cc.n_tested++;
            int r = clip_plane<P, CT, EXACT>(S, T, np, dx, dy, dz, h, nrm, j, code, spos, g, self, xws, cc);
            if (r < 0) return r;
            if (r == 2) return RC_NEED_EXACT;
            if (r == 1) R2 = rmax2<CT>(T);
        }
        __syncwarp();
        if (done) break;
        // every particle with |d|^2 < rhi2 has been examined
        if (rhi2 * ((CT)1 - (CT)8 * u) >= (CT)4 * R2) { done = true; break; }
        // an ill-conditioned vertex (infinite error bound) blocks the certificate: redo the cell in FP64
        if (!EXACT && !(R2 < (CT)INFINITY)) return RC_NEED_EXACT;
        if (rhi2 >= cap2) return g.periodic ? VT_ERR_UNSUPPORTED : VT_ERR_SECURITY;
        // next pass: the annulus up to 2R, but at most twice the radius
        rlo2 = rhi2;
        CT nxt = (CT)4 * R2 * ((CT)1 + (CT)32 * u);
        rhi2 = nxt < rhi2 * (CT)4 ? nxt : rhi2 * (CT)4;
    }
    if (!done) return (!EXACT && !(R2 < (CT)INFINITY)) ? RC_NEED_EXACT : VT_ERR_SECURITY;
    if (g.periodic && !((CT)16 * R2 < (CT)(fmin(g.L[0], fmin(g.L[1], g.L[2])) * fmin(g.L[0], fmin(g.L[1], g.L[2])))))
        return VT_ERR_UNSUPPORTED;

    // ---------------- emission: triangles and directed-edge hash into shared memory
    __syncwarp();
    for (int k = (int)lane; k < HASH_SZ; k += 32) S.u.em.hash[k] = 0xffffffffu;
    for (int k = (int)lane; k < MAXP; k += 32) S.u.em.first[k] = 0xffffffffu;
    __syncwarp();
#pragma unroll
    for (int e = 0; e < TPL; e++) {
        if ((T.vm[e] >> lane) & 1u) {
            uint32_t t = e * 32 + lane;
            uint32_t id = T.id[e];
            S.u.em.tid[t] = id;
            S.u.em.tx[t] = T.x[e]; S.u.em.ty[t] = T.y[e]; S.u.em.tz[t] = T.z[e];
            uint32_t a = id & 255, b = (id >> 8) & 255, c = (id >> 16) & 255;
            uint32_t keys[3] = {(a << 8) | b, (b << 8) | c, (c << 8) | a};
#pragma unroll
            for (int q = 0; q < 3; q++) {
                uint32_t key = keys[q];
                uint32_t ent = (key << 8) | t;
                uint32_t hsh = (key * 2654435761u) >> 23;
                for (int probe = 0; probe < HASH_SZ; probe++) {
                    uint32_t prev = atomicCAS(&S.u.em.hash[hsh], 0xffffffffu, ent);
                    if (prev == 0xffffffffu) break;
                    hsh = (hsh + 1) & (HASH_SZ - 1);
                }
            }
            atomicMin(&S.u.em.first[a], t);
            atomicMin(&S.u.em.first[b], t);
            atomicMin(&S.u.em.first[c], t);
        }
    }
    __syncwarp();
    // a facet on an initial plane: box wall (bounded) is fine; own periodic image is not supported
    if (g.periodic) {
        bool bad = (lane < 6) && S.u.em.first[lane] != 0xffffffffu;
        if (__any_sync(0xffffffffu, bad)) return VT_ERR_UNSUPPORTED;
    }
    // facets: lane (chunk c) walks plane c*32+lane; fan from the facet's first vertex
    constexpr int PCH = MAXP / 32;
    double vol = 0.0, mzx = 0.0, mzy = 0.0, mzz = 0.0, m2 = 0.0;
    CT fA[PCH], fcx[PCH], fcy[PCH], fcz[PCH];
    bool fem[PCH];
#pragma unroll
    for (int c = 0; c < PCH; c++) {
        fem[c] = false;
        fA[c] = fcx[c] = fcy[c] = fcz[c] = (CT)0;
        if (c * 32 >= np) continue;
        int p = c * 32 + (int)lane;
        bool present = p < np && S.u.em.first[p] != 0xffffffffu;
        if (!present) continue;
        uint32_t t0 = S.u.em.first[p];
        CT x0 = S.u.em.tx[t0], y0 = S.u.em.ty[t0], z0 = S.u.em.tz[t0];
        CT inrm = (CT)1 / S.pnrm[p];
        CT nhx = S.pnx[p] * inrm, nhy = S.pny[p] * inrm, nhz = S.pnz[p] * inrm;
        CT A_ = 0, csx = 0, csy = 0, csz = 0, sm2 = 0;
        uint32_t cur = succ_tri<CT>(S, t0, p);
        for (int guard = 0; guard < MAXT && cur != 0xffffffffu; guard++) {
            uint32_t nxt = succ_tri<CT>(S, cur, p);
            if (nxt == t0 || nxt == 0xffffffffu) break;
            CT x1 = S.u.em.tx[cur], y1 = S.u.em.ty[cur], z1 = S.u.em.tz[cur];
            CT x2 = S.u.em.tx[nxt], y2 = S.u.em.ty[nxt], z2 = S.u.em.tz[nxt];
            CT e1x = x1 - x0, e1y = y1 - y0, e1z = z1 - z0;
            CT e2x = x2 - x0, e2y = y2 - y0, e2z = z2 - z0;
            CT crx = f_fma<CT>(e1y, e2z, -e1z * e2y), cry = f_fma<CT>(e1z, e2x, -e1x * e2z),
               crz = f_fma<CT>(e1x, e2y, -e1y * e2x);
            CT at = (CT)0.5 * f_fma<CT>(crx, nhx, f_fma<CT>(cry, nhy, crz * nhz));
            A_ += at;
            CT third = (CT)(1.0 / 3.0);
            csx = f_fma<CT>(at * third, x0 + x1 + x2, csx);
            csy = f_fma<CT>(at * third, y0 + y1 + y2, csy);
            csz = f_fma<CT>(at * third, z0 + z1 + z2, csz);
            // |y|^2 moment of the tetrahedron (site, v0, v1, v2) without its volume factor
            CT s2 = f_fma<CT>(x0, x0 + x1 + x2, f_fma<CT>(y0, y0 + y1 + y2, z0 * (z0 + z1 + z2)));
            s2 = f_fma<CT>(x1, x1 + x2, f_fma<CT>(y1, y1 + y2, f_fma<CT>(z1, z1 + z2, s2)));
            s2 = f_fma<CT>(x2, x2, f_fma<CT>(y2, y2, f_fma<CT>(z2, z2, s2)));
            sm2 = f_fma<CT>(at, s2, sm2);
            cur = nxt;
        }
        // distance from the site to the facet plane; tetrahedra (site, fan triangle) give
        // V_f = dist A_f / 3, first moment dist * sum(at (v0+v1+v2)/3) / 4, second moment dist/30 * sum(at s2)
        CT dist = S.ph[p] * inrm;
        vol += (double)(dist * A_) * (1.0 / 3.0);
        mzx += (double)(dist * csx) * 0.25;
        mzy += (double)(dist * csy) * 0.25;
        mzz += (double)(dist * csz) * 0.25;
        m2 += (double)(dist * sm2) * (1.0 / 30.0);
        if (A_ != (CT)0) { fcx[c] = csx / A_; fcy[c] = csy / A_; fcz[c] = csz / A_; }
        fA[c] = A_;
        fem[c] = (p >= 6) && S.pcode[p] < 27;
    }
    vol = warp_sum_d(vol);
    m2 = warp_sum_d(m2);
    mzx = warp_sum_d(mzx); mzy = warp_sum_d(mzy); mzz = warp_sum_d(mzz);
    const double sg = vol < 0 ? -1.0 : 1.0;
    vol *= sg; m2 *= sg;
    int nf_total = 0;
#pragma unroll
    for (int c = 0; c < PCH; c++) nf_total += __popc(__ballot_sync(0xffffffffu, fem[c]));
    // reserve facet records
    uint32_t start = 0;
    if (lane == 0 && nf_total > 0) {
        unsigned long long s0 = atomicAdd(&A.st->face_next, (unsigned long long)nf_total);
        start = (s0 + nf_total <= A.face_cap) ? (uint32_t)s0 : 0xffffffffu;
    }
    start = __shfl_sync(0xffffffffu, start, 0);
    if (start == 0xffffffffu) return RC_POOL;
    {
        int acc = 0;
#pragma unroll
        for (int c = 0; c < PCH; c++) {
            unsigned m = __ballot_sync(0xffffffffu, fem[c]);
            if (fem[c]) {
                int p = c * 32 + (int)lane;
                Face f;
                f.dx = (float)S.pnx[p]; f.dy = (float)S.pny[p]; f.dz = (float)S.pnz[p];
                f.area = (float)(sg * (double)fA[c]);
                f.cx = (float)fcx[c]; f.cy = (float)fcy[c]; f.cz = (float)fcz[c];
                f.nbr = S.psrc[p];
                A.faces[start + acc + __popc(m & lt)] = f;
            }
            acc += __popc(m);
        }
    }
    if (lane == 0) {
        CellOut co;
        co.vol = vol;
        co.zx = (float)(vol > 0 ? sg * mzx / vol : 0.0);
        co.zy = (float)(vol > 0 ? sg * mzy / vol : 0.0);
        co.zz = (float)(vol > 0 ? sg * mzz / vol : 0.0);
        co.mom2 = (float)m2;
        A.cell[self] = co;
        A.face_start[self] = start;
        A.face_count[self] = (uint16_t)nf_total;
        atomicMax(&A.st->max_faces, (unsigned)nf_total);
        atomicAdd(&A.st->n_faces, (unsigned long long)nf_total);
    }
    return 0;
}

template <typename P, typename CT, bool EXACT>
__global__ void __launch_bounds__(CLIP_WARPS * 32) k_clip(ClipArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int w = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    WarpSmem<CT>& S = reinterpret_cast<WarpSmem<CT>*>(smem_raw)[w];
    const int gw = blockIdx.x * CLIP_WARPS + w;
    double* xws = EXACT ? (A.xws + (size_t)gw * EXACT_WS) : nullptr;
    CellCounters cc = {0, 0, 0, 0, 0, 0};
    const uint32_t total = EXACT ? 0u : (uint32_t)A.N;
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(EXACT ? &A.st->work_next_exact : &A.st->work_next, (unsigned)CHUNK);
        base = __shfl_sync(0xffffffffu, base, 0);
        uint32_t lim = EXACT ? *((volatile unsigned*)&A.st->n_exact_cells) : total;
        if (base >= lim) break;
        for (uint32_t q = base; q < base + CHUNK && q < lim; q++) {
            uint32_t self = EXACT ? A.exact_list[q] : q;
            int rc = do_cell<P, CT, EXACT>(S, A, self, xws, cc);
            __syncwarp();
            if (lane == 0) {
                if (rc == 0) {
                    A.cstat[self] = CS_DONE;
                } else if (rc == RC_NEED_EXACT) {
                    A.cstat[self] = CS_NEED_EXACT;
                    unsigned slot = atomicAdd(&A.st->n_exact_cells, 1u);
                    A.exact_list[slot] = self;
                } else {
                    A.cstat[self] = CS_ERROR;
                    if (atomicCAS(&A.st->error, 0, rc) == 0) A.st->error_cell = (int)self;
                }
            }
        }
    }
    if (lane == 0) {
        atomicAdd(&A.st->n_cut, (unsigned long long)cc.n_cut);
        atomicAdd(&A.st->n_tested, (unsigned long long)cc.n_tested);
        atomicAdd(&A.st->n_passes, (unsigned long long)cc.n_passes);
        atomicAdd(&A.st->n_fp64, (unsigned long long)cc.n_fp64);
        atomicAdd(&A.st->n_exact_preds, (unsigned long long)cc.n_exact);
        atomicAdd(&A.st->n_exact_zero, (unsigned long long)cc.n_zero);
    }
}

}  // namespace vt

namespace vt {
template <typename P, typename CT, bool EXACT>
static void launch_one(const ClipArgs& a, int sm_count, cudaStream_t s) {
    size_t smem = sizeof(WarpSmem<CT>) * CLIP_WARPS;
    cudaFuncSetAttribute(k_clip<P, CT, EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_clip<P, CT, EXACT>, CLIP_WARPS * 32, smem);
    if (per_sm < 1) per_sm = 1;
    int blocks = sm_count * per_sm;
    if (EXACT) blocks = a.xws_warps / CLIP_WARPS;
    k_clip<P, CT, EXACT><<<blocks, CLIP_WARPS * 32, smem, s>>>(a);
}
}  // namespace vt
