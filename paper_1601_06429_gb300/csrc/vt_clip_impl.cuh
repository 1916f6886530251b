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
constexpr int HIST_BINS = 64;

// Per-cell capacities.  TP = vertex slots per lane.  The fast kernels use Cap<4> (128 vertices, 128 planes with
// 8-bit ids); cells that overflow them, and cells whose FP64 tests stay undecided, are redone by the exact
// kernel with Cap<16> (512 vertices, 512 planes with 10-bit ids).
template <int TP>
struct Cap {
    static constexpr int TPL = TP;
    static constexpr int MAXT = 32 * TP;
    static constexpr int IDB = TP <= 4 ? 8 : 10;          // bits of a plane id in a packed triangle
    static constexpr int MAXP = TP <= 4 ? 128 : 512;
    static constexpr uint32_t IDM = (1u << IDB) - 1u;
    static constexpr int SB = TP <= 4 ? 7 : 9;            // bits of a vertex slot
    static constexpr int CAND = 256;                      // candidates per radius pass
    static constexpr int STACK = TP <= 4 ? STACK_CAP : 4 * STACK_CAP;
};
constexpr int CHUNK = 4;

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
// a vertex's position (relative to the site) and the bound of its error, read and written as one record
template <typename CT> struct Vtx;
template <> struct __align__(16) Vtx<float> { float x, y, z, ev; };
template <> struct __align__(32) Vtx<double> { double x, y, z, ev; };

// a plane n.y <= h (n the displacement, or a unit wall normal) as one record; its norm |n| is kept apart
template <typename CT> struct Pln;
template <> struct __align__(16) Pln<float> { float x, y, z, h; };
template <> struct __align__(32) Pln<double> { double x, y, z, h; };

template <typename CT, int TP>
struct WarpSmem {
    typedef Cap<TP> K;
    // planes that have cut the cell: n.y <= h with |n| = nrm, source particle and image shift
    Pln<CT> pl[K::MAXP];
    CT pnrm[K::MAXP];
    uint32_t psrc[K::MAXP];
    uint8_t pcode[K::MAXP];  // 0..26 image shift code, 27+w box wall w
    // vertices = triangles of the dual triangulation: packed plane ids, position, error bound, R^2 bound
    uint32_t tid[K::MAXT];
    uint32_t tadj[K::MAXT];  // neighbour slot across edge k (k = 0: a->b, 1: b->c, 2: c->a), 10 bits each
    Vtx<CT> tv[K::MAXT];
    CT trr[K::MAXT];
    union {
        struct {
            unsigned long long key[K::CAND];  // (|d|^2 as float bits) << 32 | slot
            uint32_t j[K::CAND];               // the candidate (its displacement is recomputed when it is used)
        } cd;
        struct {
            uint32_t first[K::MAXP];
        } em;
    } u;
    uint32_t bnd[K::MAXT];       // boundary records of a cut: x, y, kept neighbour slot, its edge index
    uint16_t lnk_s[K::MAXP];     // new triangle whose boundary edge starts at plane x
    uint16_t lnk_e[K::MAXP];     // new triangle whose boundary edge ends at plane y
    uint32_t stack[K::STACK];
    uint32_t hist[HIST_BINS];  // radial histogram of an overflowing candidate pass
    uint16_t live[K::MAXP];    // plane-id compaction
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
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
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

// Compensated summation (Kahan's method in Neumaier's form): s + c carries the running sum with the rounding
// error of every addition kept in c, so the result is the exact sum of the terms to within about one rounding
// of it plus u^2 times the sum of their magnitudes.  FP32 geometry accumulates its facet areas and cell volumes
// this way; FP64 geometry sums plainly (its rounding is far below its vertex error).
template <typename CT>
struct KSum {
    CT s, c;
    __device__ __forceinline__ void zero() { s = (CT)0; c = (CT)0; }
    __device__ __forceinline__ void add(CT x) { s += x; }
    __device__ __forceinline__ CT value() const { return s; }
    __device__ __forceinline__ void warp_reduce() {
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
};
template <>
struct KSum<float> {
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float x) {
        float t, e;
        tsum_f(s, x, t, e);
        s = t;
        c = __fadd_rn(c, e);
    }
    __device__ __forceinline__ float value() const { return __fadd_rn(s, c); }
    // all lanes: the compensated sum over the warp (pairwise, with every level's rounding error kept)
    __device__ __forceinline__ void warp_reduce() {
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const float so = __shfl_xor_sync(0xffffffffu, s, o), co = __shfl_xor_sync(0xffffffffu, c, o);
            float t, e;
            tsum_f(s, so, t, e);
            s = t;
            c = __fadd_rn(__fadd_rn(c, co), e);
        }
    }
};

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

// x - e rounded down and x + e rounded up, as floats
__device__ __forceinline__ float sub_dn(float x, float e) { return __fsub_rd(x, e); }
__device__ __forceinline__ float add_up(float x, float e) { return __fadd_ru(x, e); }
__device__ __forceinline__ float sub_dn(double x, double e) { return __double2float_rd(x - e); }
__device__ __forceinline__ float add_up(double x, double e) { return __double2float_ru(x + e); }

// bit pattern of a non-negative value (order preserving), and back
template <typename CT> __device__ __forceinline__ unsigned long long fbits(CT v);
template <> __device__ __forceinline__ unsigned long long fbits<float>(float v) { return __float_as_uint(v); }
template <> __device__ __forceinline__ unsigned long long fbits<double>(double v) {
    return (unsigned long long)__double_as_longlong(v);
}
template <typename CT> __device__ __forceinline__ CT fromfbits(unsigned long long b);
template <> __device__ __forceinline__ float fromfbits<float>(unsigned long long b) { return __uint_as_float((uint32_t)b); }
template <> __device__ __forceinline__ double fromfbits<double>(unsigned long long b) {
    return __longlong_as_double((long long)b);
}

// displacement of particle j seen from i without a periodic shift: the shift-free path of DispF, rounded the same way
template <typename P, typename CT> struct DispPlain;
template <> struct DispPlain<float4, float> {
    static __device__ __forceinline__ void get(const float4& pj, const float4& pi, float& dx, float& dy, float& dz) {
        dx = __fsub_rn(pj.x, pi.x); dy = __fsub_rn(pj.y, pi.y); dz = __fsub_rn(pj.z, pi.z);
    }
};
template <typename P> struct DispPlain<P, double> {
    static __device__ __forceinline__ void get(const P& pj, const P& pi, double& dx, double& dy, double& dz) {
        dx = __dsub_rn((double)pj.x, (double)pi.x);
        dy = __dsub_rn((double)pj.y, (double)pi.y);
        dz = __dsub_rn((double)pj.z, (double)pi.z);
    }
};
template <> struct DispPlain<dpt4, float> {
    static __device__ __forceinline__ void get(const dpt4& pj, const dpt4& pi, float& dx, float& dy, float& dz) {
        dx = (float)__dsub_rn(pj.x, pi.x); dy = (float)__dsub_rn(pj.y, pi.y); dz = (float)__dsub_rn(pj.z, pi.z);
    }
};

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
    CT H = fabs(ah) + fabs(bh) + fabs(ch);  // offsets are >= 0 except for the voxel walls of the grid average
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

// A plane's source: code 0..26 = bisector with particle src under image shift `code`; 27..32 = box wall
// (27 + w); 33..38 = artificial wall 33 + w at distance B from the site, with B's float bits in src.
struct PRef {
    uint32_t src;
    int code;
};
constexpr int CODE_WALL = 27, CODE_ART = 33;

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
        int wall = r.code - (r.code >= CODE_ART ? CODE_ART : CODE_WALL), axis = wall >> 1;
        bool upper = (wall & 1) == 0;
        for (int c = 0; c < 3; c++) {
            row[c] = x_alloc(w, 1);
            if (c == axis) x_grow(w, row[c], upper ? 1.0 : -1.0);
        }
        row[3] = x_alloc(w, 3);
        if (r.code >= CODE_ART) x_grow(w, row[3], (double)__uint_as_float(r.src));
        else if (upper) { x_grow(w, row[3], g.hi[axis]); x_grow(w, row[3], -xi[axis]); }
        else { x_grow(w, row[3], xi[axis]); x_grow(w, row[3], -g.lo[axis]); }
    }
}

// +1: vertex of (a,b,c) strictly beyond plane j; -1: strictly inside; 0: on it.  *ovf on workspace overflow.
template <typename P>
__device__ __noinline__ int exact_side(double* ws, const P* spos, const Geometry& g, uint32_t self, PRef a, PRef b, PRef c, PRef j,
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
        int wall = r.code - (r.code >= CODE_ART ? CODE_ART : CODE_WALL), axis = wall >> 1;
        bool upper = (wall & 1) == 0;
        double xi = axis == 0 ? (double)pi.x : axis == 1 ? (double)pi.y : (double)pi.z;
        nx = ny = nz = 0.0;
        double sgn = upper ? 1.0 : -1.0;
        if (axis == 0) nx = sgn; else if (axis == 1) ny = sgn; else nz = sgn;
        if (r.code >= CODE_ART) h = (double)__uint_as_float(r.src);
        else h = upper ? __dsub_rn(g.hi[axis], xi) : __dsub_rn(xi, g.lo[axis]);
        nrm = 1.0;
    }
}

template <typename P>
__device__ __noinline__ int side64(const P* spos, const Geometry& g, uint32_t self, PRef a, PRef b, PRef c, PRef j) {
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
// The cell's vertices live in shared memory slots; which slots are in use is kept in four warp-uniform
// 32-bit masks (slot = 32 e + lane), with hw an upper bound of the used slots.
template <int TP>
struct CellState {
    unsigned vm[TP];
    int hw;
    int np;
};

template <int TP>
__device__ __forceinline__ void unpack(uint32_t id, uint32_t& a, uint32_t& b, uint32_t& c) {
    typedef Cap<TP> K;
    a = id & K::IDM; b = (id >> K::IDB) & K::IDM; c = (id >> (2 * K::IDB)) & K::IDM;
}
template <int TP>
__device__ __forceinline__ uint32_t pack(uint32_t a, uint32_t b, uint32_t c) {
    typedef Cap<TP> K;
    return a | (b << K::IDB) | (c << (2 * K::IDB));
}
__device__ __forceinline__ uint32_t adj_get(uint32_t adj, int k) { return (adj >> (10 * k)) & 1023u; }
__device__ __forceinline__ uint32_t adj_pack(uint32_t n0, uint32_t n1, uint32_t n2) {
    return n0 | (n1 << 10) | (n2 << 20);
}
// position of plane p in a packed triangle (0, 1 or 2)
template <int TP>
__device__ __forceinline__ int pos_of(uint32_t id, uint32_t p) {
    uint32_t a, b, c;
    unpack<TP>(id, a, b, c);
    return a == p ? 0 : (b == p ? 1 : 2);
}
// is slot n in the mask set m[]
template <int TP>
__device__ __forceinline__ bool in_mask(const unsigned* m, uint32_t n) {
    bool r = false;
#pragma unroll
    for (int q = 0; q < TP; q++)
        if ((int)(n >> 5) == q) r = ((m[q] >> (n & 31)) & 1u) != 0;
    return r;
}

struct CellCounters {
    unsigned n_cut, n_tested, n_passes, n_fp64, n_exact, n_zero, n_collect, n_collected;
#ifdef VT_PHASE_TIMERS
    unsigned long long t[10];  // cycles: collect, sort, plane tests, candidate batches, emit, total, apply_cut, -, box,
                               // undecided tests on start-box vertices (count)
#endif
};

// Optional per-phase cycle counters (compile with -DVT_PHASE_TIMERS; off in normal builds).
#ifdef VT_PHASE_TIMERS
#define VT_T0(name) long long name = clock64()
#define VT_T1(cc, k, name) (cc).t[k] += (unsigned long long)(clock64() - name)
#else
#define VT_T0(name)
#define VT_T1(cc, k, name)
#endif

// Capacity failures carry a reason (reported through the device status): -100 - reason.
constexpr int CAP_PLANES = -101, CAP_TRIS = -102, CAP_BOUNDARY = -103, CAP_CAND = -104, CAP_STACK = -105,
              CAP_FACETS = -106;

template <typename CT, int TP>
__device__ __forceinline__ void tri_vertex(WarpSmem<CT, TP>& S, int s) {
    typedef Cap<TP> K;
    uint32_t a, b, c;
    unpack<TP>(S.tid[s], a, b, c);
    Vtx<CT> v;
    CT rr;
    const Pln<CT> A = S.pl[a], B = S.pl[b], C = S.pl[c];
    make_vertex<CT>(A.x, A.y, A.z, A.h, S.pnrm[a], B.x, B.y, B.z, B.h, S.pnrm[b], C.x, C.y, C.z, C.h, S.pnrm[c], v.x, v.y,
                    v.z, v.ev, rr);
    S.tv[s] = v;
    S.trr[s] = rr;
}

// Drop the planes that no vertex uses any more (their facets were cut away) and renumber the rest; the six
// initial planes keep ids 0..5.  Entries only move to lower ids, so each chunk of 32 is read, then written
// in place.  Returns the new plane count.
template <typename CT, int TP>
__device__ __noinline__ int compact_planes(WarpSmem<CT, TP>& S, const unsigned* vm, int np) {
    typedef Cap<TP> K;
    const unsigned lane = lane_id(), lt = lanemask_lt();
    for (int p = (int)lane; p < K::MAXP; p += 32) S.live[p] = (p < 6) ? 1 : 0;
    __syncwarp();
    for (int e = 0; e < TP; e++)
        if ((vm[e] >> lane) & 1u) {
            uint32_t a, b, c;
            unpack<TP>(S.tid[e * 32 + lane], a, b, c);
            S.live[a] = 1; S.live[b] = 1; S.live[c] = 1;
        }
    __syncwarp();
    int base = 0;
    for (int c = 0; c < K::MAXP / 32; c++) {
        int p = c * 32 + (int)lane;
        bool lv = p < np && S.live[p];
        CT qx = 0, qy = 0, qz = 0, qh = 0, qn = 0;
        uint32_t qs = 0;
        uint8_t qc = 0;
        if (lv) {
            const Pln<CT> pq = S.pl[p];
            qx = pq.x; qy = pq.y; qz = pq.z; qh = pq.h; qn = S.pnrm[p];
            qs = S.psrc[p]; qc = S.pcode[p];
        }
        unsigned m = __ballot_sync(0xffffffffu, lv);
        int q = base + __popc(m & lt);
        base += __popc(m);
        __syncwarp();
        if (lv) {
            Pln<CT> pq;
            pq.x = qx; pq.y = qy; pq.z = qz; pq.h = qh;
            S.pl[q] = pq;
            S.pnrm[q] = qn;
            S.psrc[q] = qs; S.pcode[q] = qc;
            S.live[p] = (uint16_t)q;  // now the renumbering table
        }
        __syncwarp();
    }
    for (int e = 0; e < TP; e++)
        if ((vm[e] >> lane) & 1u) {
            int t = e * 32 + lane;
            uint32_t a, b, c;
            unpack<TP>(S.tid[t], a, b, c);
            S.tid[t] = pack<TP>(S.live[a], S.live[b], S.live[c]);
        }
    __syncwarp();
    return base;
}

// Side of vertex slot s w.r.t. the lane's plane in the working precision: +1 strictly beyond, -1 strictly
// inside, 0 when the error bound does not decide.
template <typename CT, int TP>
__device__ __forceinline__ int side_fast(const WarpSmem<CT, TP>& S, int s, CT nx, CT ny, CT nz, CT h, CT nrm, CT hb) {
    const Vtx<CT> v = S.tv[s];
    CT sv = f_fma<CT>(nx, v.x, f_fma<CT>(ny, v.y, f_fma<CT>(nz, v.z, -h)));
    CT bound = f_fma<CT>(nrm, v.ev, hb);
    if (sv > bound) return 1;
    if (sv < -bound) return -1;
    return 0;  // includes NaN / infinite bounds
}

// Decide the lanes flagged `need` (vertex slot s against each lane's plane): FP64 from the inputs in the FP32
// kernels, then exact expansion arithmetic in the exact kernel (lanes take the warp's workspace in turn).
// Returns +1/-1 per lane (0 if undecided in a non-exact kernel: *need_exact is set).
template <typename P, typename CT, bool EXACT, int TP>
__device__ int resolve(const WarpSmem<CT, TP>& S, int s, bool need, uint32_t src, int code, const P* spos,
                       const Geometry& g, uint32_t self, double* xws, CellCounters& cc, bool& need_exact,
                       bool& ovf) {
    const unsigned lane = lane_id();
    int sd = 0;
    uint32_t a, b, c;
    unpack<TP>(S.tid[s], a, b, c);
    PRef ra = {S.psrc[a], S.pcode[a]}, rb = {S.psrc[b], S.pcode[b]}, rc = {S.psrc[c], S.pcode[c]};
    PRef rj = {src, code};
    if (need && sizeof(CT) == 4) {
        sd = side64<P>(spos, g, self, ra, rb, rc, rj);
        cc.n_fp64++;
#ifdef VT_PHASE_TIMERS
        if (a < 6 || b < 6 || c < 6) cc.t[9]++;  // undecided test on a vertex that still touches the initial cube
#endif
    }
    bool pending = need && sd == 0;
    if (!EXACT) {
        if (pending) need_exact = true;
        return sd;
    }
    unsigned todo = __ballot_sync(0xffffffffu, pending);
    while (todo) {
        int L = __ffs(todo) - 1;
        if ((int)lane == L) {
            bool o = false;
            sd = exact_side<P>(xws, spos, g, self, ra, rb, rc, rj, &o);
            cc.n_exact++;
            if (o) ovf = true;
            if (sd == 0) cc.n_zero++;
            if (sd == 0) sd = -1;  // on the plane: kept (not strictly beyond)
        }
        __syncwarp();
        todo &= todo - 1;
    }
    return sd;
}

// position of the k-th (from 0) set bit of m; m must have more than k set bits
__device__ __forceinline__ int nth_set_bit(unsigned m, int k) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w; w >>= 1) {
        const unsigned lo = m & ((1u << w) - 1u);
        const int c = __popc(lo);
        if (k >= c) { k -= c; m >>= w; pos += w; }
        else m = lo;
    }
    return pos;
}
// the k lowest set bits of m (all of them if it has k or fewer)
__device__ __forceinline__ unsigned lowest_set_bits(unsigned m, int k) {
    if (k <= 0) return 0u;
    if (k >= __popc(m)) return m;
    return m & ((1u << nth_set_bit(m, k)) - 1u);
}
// element e of a small per-chunk mask array without dynamic register indexing
template <int TP>
__device__ __forceinline__ unsigned pick(const unsigned* a, int e) {
    unsigned r = a[0];
#pragma unroll
    for (int q = 1; q < TP; q++)
        if (e == q) r = a[q];
    return r;
}

// Cut the cell by a plane known to remove exactly the vertex slots rem[].  The plane gets an id; every edge
// x->y of a removed triangle whose neighbour across it is kept lies on the boundary of the removed region and
// becomes a new triangle (x, y, p); the k-th boundary edge takes the k-th lowest free slot.  Adjacency: across
// x->y the kept neighbour (whose pointer is redirected to the new triangle), across y->p the new triangle
// starting at y, across p->x the new triangle ending at x.  newm[] returns the new slots.  Returns 0 or a CAP_*
// code.  Each per-slot step is written once (loops over chunks and over boundary ranks), which keeps the
// kernel's instruction footprint small.
template <typename CT, int TP>
__device__ int apply_cut(WarpSmem<CT, TP>& S, CellState<TP>& C, const unsigned* rem, CT nx, CT ny, CT nz, CT h, CT nrm,
                         uint32_t src, int code, unsigned* newm) {
    typedef Cap<TP> K;
    const unsigned lane = lane_id(), lt = lanemask_lt();
    if (C.np >= K::MAXP) {
        C.np = compact_planes<CT, TP>(S, C.vm, C.np);
        if (C.np >= K::MAXP) return CAP_PLANES;
    }
    const int p = C.np++;
    if (lane == 0) {
        Pln<CT> pq;
        pq.x = nx; pq.y = ny; pq.z = nz; pq.h = h;
        S.pl[p] = pq;
        S.pnrm[p] = nrm;
        S.psrc[p] = src; S.pcode[p] = (uint8_t)code;
    }
    // boundary records, chunk by chunk (the lane's slot of chunk e is e * 32 + lane)
    int nB = 0;
    const int nch = (C.hw + 31) >> 5;
#pragma unroll 1
    for (int e = 0; e < nch; e++) {
        const unsigned re = pick<TP>(rem, e);
        if (!re) continue;
        const bool mine = (re >> lane) & 1u;
        uint32_t ids[3] = {0u, 0u, 0u}, adj = 0u;
        const uint32_t t = e * 32 + lane;
        if (mine) {
            unpack<TP>(S.tid[t], ids[0], ids[1], ids[2]);
            adj = S.tadj[t];
        }
#pragma unroll
        for (int k = 0; k < 3; k++) {
            uint32_t n = adj_get(adj, k);
            bool bnd = mine && !in_mask<TP>(rem, n);
            unsigned bm = __ballot_sync(0xffffffffu, bnd);
            if (bnd) {
                int o = nB + __popc(bm & lt);
                uint32_t nadj = S.tadj[n];
                uint32_t kn = adj_get(nadj, 0) == t ? 0u : (adj_get(nadj, 1) == t ? 1u : 2u);
                if (o < K::MAXT)
                    S.bnd[o] = ids[k] | (ids[(k + 1) % 3] << K::IDB) | (n << (2 * K::IDB)) | (kn << (2 * K::IDB + K::SB));
            }
            nB += __popc(bm);
        }
    }
#pragma unroll
    for (int e = 0; e < TP; e++) C.vm[e] &= ~rem[e];
    __syncwarp();
    if (nB > K::MAXT) return CAP_BOUNDARY;
    // the new triangles take the nB lowest free slots: masks per chunk (warp-uniform)
    int placed = 0;
#pragma unroll
    for (int e = 0; e < TP; e++) {
        const unsigned fm = ~C.vm[e];
        const unsigned nm = lowest_set_bits(fm, nB - placed);
        newm[e] = nm;
        placed += __popc(fm);
    }
    if (placed < nB) return CAP_TRIS;
    // the k-th lowest new slot takes boundary record k (its rank among the new slots, counted chunk by chunk);
    // first the link tables by plane id, then the triangles
#pragma unroll 1
    for (int e = 0, acc = 0; e < TP && acc < nB; e++) {
        const unsigned nm = pick<TP>(newm, e);
        if ((nm >> lane) & 1u) {
            const uint32_t rec = S.bnd[acc + __popc(nm & lt)];
            const uint32_t t = (uint32_t)(e * 32) + lane;
            S.lnk_s[rec & K::IDM] = (uint16_t)t;
            S.lnk_e[(rec >> K::IDB) & K::IDM] = (uint16_t)t;
        }
        acc += __popc(nm);
    }
    __syncwarp();
#pragma unroll 1
    for (int e = 0, acc = 0; e < TP && acc < nB; e++) {
        const unsigned nm = pick<TP>(newm, e);
        if ((nm >> lane) & 1u) {
            const uint32_t rec = S.bnd[acc + __popc(nm & lt)];
            const uint32_t x = rec & K::IDM, y = (rec >> K::IDB) & K::IDM;
            const uint32_t n = (rec >> (2 * K::IDB)) & ((1u << K::SB) - 1u), kn = rec >> (2 * K::IDB + K::SB);
            const uint32_t t = (uint32_t)(e * 32) + lane;
            S.tid[t] = pack<TP>(x, y, (uint32_t)p);
            S.tadj[t] = adj_pack(n, S.lnk_s[y], S.lnk_e[x]);
            // redirect the kept neighbour's pointer (fields of one word may be updated by two new triangles)
            atomicAnd(&S.tadj[n], ~(1023u << (10 * kn)));
            atomicOr(&S.tadj[n], t << (10 * kn));
            tri_vertex<CT, TP>(S, t);
        }
        acc += __popc(nm);
    }
#pragma unroll
    for (int e = 0; e < TP; e++) {
        C.vm[e] |= newm[e];
        if (newm[e]) C.hw = max(C.hw, e * 32 + 32 - __clz(newm[e]));
    }
    __syncwarp();
    return 0;
}

// One pass over the vertices: the bound of |v|^2 (returned; the security radius is twice its root) and the box
// around the exact vertices (positions widened by their error bounds), as floats rounded outward
template <typename CT, int TP>
__device__ __forceinline__ CT radius_box(const WarpSmem<CT, TP>& S, const CellState<TP>& C, float* bmin, float* bmax) {
    const unsigned lane = lane_id();
    CT r = 0;
    float lo0 = 0.f, lo1 = 0.f, lo2 = 0.f, hi0 = 0.f, hi1 = 0.f, hi2 = 0.f;  // the site is inside
    bool inf = false;
#pragma unroll
    for (int e = 0; e < TP; e++)
        if ((C.vm[e] >> lane) & 1u) {
            const int s = e * 32 + lane;
            const CT rr = S.trr[s];
            r = r > rr ? r : rr;
            const Vtx<CT> v = S.tv[s];
            const CT ev = v.ev;
            if (!(ev < (CT)INFINITY)) inf = true;
            lo0 = fminf(lo0, sub_dn(v.x, ev));
            lo1 = fminf(lo1, sub_dn(v.y, ev));
            lo2 = fminf(lo2, sub_dn(v.z, ev));
            hi0 = fmaxf(hi0, add_up(v.x, ev));
            hi1 = fmaxf(hi1, add_up(v.y, ev));
            hi2 = fmaxf(hi2, add_up(v.z, ev));
        }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const CT ro = __shfl_xor_sync(0xffffffffu, r, o);
        r = r > ro ? r : ro;
        lo0 = fminf(lo0, __shfl_xor_sync(0xffffffffu, lo0, o));
        lo1 = fminf(lo1, __shfl_xor_sync(0xffffffffu, lo1, o));
        lo2 = fminf(lo2, __shfl_xor_sync(0xffffffffu, lo2, o));
        hi0 = fmaxf(hi0, __shfl_xor_sync(0xffffffffu, hi0, o));
        hi1 = fmaxf(hi1, __shfl_xor_sync(0xffffffffu, hi1, o));
        hi2 = fmaxf(hi2, __shfl_xor_sync(0xffffffffu, hi2, o));
    }
    if (__any_sync(0xffffffffu, inf)) {  // unknown vertex: no filtering
        lo0 = lo1 = lo2 = -INFINITY;
        hi0 = hi1 = hi2 = INFINITY;
    }
    bmin[0] = lo0; bmin[1] = lo1; bmin[2] = lo2;
    bmax[0] = hi0; bmax[1] = hi1; bmax[2] = hi2;
    return r;
}

// ------------------------------------------------------------------ tree search
// Support-function filter.  With [bmin, bmax] (bmin <= 0 <= bmax) a box around the exact vertices of the cell
// (site at the origin), a point p can cut the cell only if some vertex v has 2 p.v > |p|^2, and
// p.v <= sum_a max(p_a bmin_a, p_a bmax_a); so p cannot cut when
//     sum_a g_a(p_a) <= 0,   g_a(t) = 2 max(t bmin_a, t bmax_a) - t^2.
// g_a is concave on each sign of t, with its peak at bmax_a (t >= 0) and at bmin_a (t <= 0).
__device__ __forceinline__ float supp_g(float t, float bmin, float bmax) {
    return 2.f * fmaxf(t * bmin, t * bmax) - t * t;
}
// largest g over [t0, t1]
__device__ __forceinline__ float supp_gmax(float t0, float t1, float bmin, float bmax) {
    float best = -INFINITY;
    if (t1 >= 0.f) best = fmaxf(best, supp_g(fminf(fmaxf(bmax, fmaxf(t0, 0.f)), t1), bmin, bmax));
    if (t0 <= 0.f) best = fmaxf(best, supp_g(fmaxf(fminf(bmin, fminf(t1, 0.f)), t0), bmin, bmax));
    return best;
}
// largest g over the node's extent along one axis, relative to q, for its minimum-image shifts
__device__ __forceinline__ float supp_axis(float q, float lo, float hi, float L, int periodic, float bmin,
                                           float bmax) {
    float m = supp_gmax(lo - q, hi - q, bmin, bmax);
    if (periodic) {
        m = fmaxf(m, supp_gmax(lo - q - L, hi - q - L, bmin, bmax));
        m = fmaxf(m, supp_gmax(lo - q + L, hi - q + L, bmin, bmax));
    }
    return m;
}

// upper bound of the (minimum-image) distance along one axis from q to any point of [lo, hi]
__device__ __forceinline__ float axis_far(float q, float lo, float hi, float L, int periodic) {
    float d = fmaxf(fabsf(q - lo), fabsf(q - hi));
    if (periodic) {
        d = fminf(d, fmaxf(fabsf(q - lo - L), fabsf(q - hi - L)));
        d = fminf(d, fmaxf(fabsf(q - lo + L), fabsf(q - hi + L)));
    }
    return d;
}
__device__ __forceinline__ float axis_gap(float q, float lo, float hi, float L, int periodic) {
    float d = fmaxf(fmaxf(lo - q, q - hi), 0.f);
    if (periodic) {
        d = fminf(d, fmaxf(lo + L - q, 0.f));
        d = fminf(d, fmaxf(q + L - hi, 0.f));
    }
    return d;
}

// Collect sorted indices j != self with rlo2 <= |d|^2 < rhi2 (the same |d|^2 as the clipping loop).
// Every hit is also counted in a radial histogram of |d|^2 over [rlo2, rhi2) (HIST_BINS bins), so that an
// overflowing pass can pick a smaller rhi2 that fits.  Returns the count (which may exceed the capacity: only the
// first Cap::CAND are stored) or -2 on stack overflow.
template <typename P, typename CT, int TP>
__device__ int collect(WarpSmem<CT, TP>& S, const P* spos, int64_t N, const Geometry& g, const Tree& t, uint32_t self,
                       const P& pi, CT rlo2, CT rhi2, const float* bmin, const float* bmax, int64_t slo,
                       int64_t shi) {
    const unsigned lane = lane_id(), lt = lanemask_lt();
    for (int k = (int)lane; k < HIST_BINS; k += 32) S.hist[k] = 0u;
    __syncwarp();
    // bins over the bit patterns of the non-negative |d|^2 (monotone), so narrowing never underflows
    const unsigned long long blo = fbits<CT>(rlo2), bhi = fbits<CT>(rhi2);
    const unsigned long long bwidth = bhi > blo ? bhi - blo : 1ull;
    const float binsc = (float)HIST_BINS / (float)bwidth;
    // conservative float radius for box pruning
    float rad = sqrtf((float)rhi2) * 1.0001f + 1e-30f;
    float rad2 = rad * rad;
    // nodes entirely within the inner radius hold only examined points
    float inner2 = (float)rlo2 * 0.9999f;
    // rounding tolerance of the support test: relative 1e-5 of its terms
    const float bext = fmaxf(fmaxf(fmaxf(-bmin[0], bmax[0]), fmaxf(-bmin[1], bmax[1])), fmaxf(-bmin[2], bmax[2]));
    const float stol = 1e-5f * (4.f * bext * rad + rad2) + 1e-30f;
    float qx = (float)pi.x, qy = (float)pi.y, qz = (float)pi.z;
    // float rounding of q: widen by one ulp of the box scale
    float slack = 2.0f * 1.2e-7f * fmaxf(fmaxf(fabsf(g.hif[0]), fabsf(g.lof[0])),
                                         fmaxf(fmaxf(fabsf(g.hif[1]), fabsf(g.lof[1])),
                                               fmaxf(fabsf(g.hif[2]), fabsf(g.lof[2]))));
    // a search ball that stays inside the periodic box meets no image across it: the node tests then need no
    // shifted copies (points beyond the box are farther than the radius in their minimum image too)
    const float reach = rad + 4.f * slack;
    const int per = g.periodic && !(qx - reach > g.lof[0] && qx + reach < g.hif[0] && qy - reach > g.lof[1] &&
                                    qy + reach < g.hif[1] && qz - reach > g.lof[2] && qz + reach < g.hif[2]);
    // the root: a virtual node one level above the top, whose children are the top-level nodes
    if (lane == 0) S.stack[0] = ((uint32_t)(t.levels + 1) << 27) | 0u;
    int sp = 1;
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
            CT d2 = (CT)0, dx = (CT)0, dy = (CT)0, dz = (CT)0;
            int code = 13;
            if (j >= slo && j < shi && (uint32_t)j != self) {
                P pj = spos[j];
                // a search ball inside the periodic box holds no shifted image (an image lies outside the box), and
                // a point's unshifted distance is at least its minimum-image one: the same points pass the radius
                // test, with the same displacements, as with the shifts
                if (per) DispF<P, CT>::get(pj, pi, g, dx, dy, dz, code);
                else DispPlain<P, CT>::get(pj, pi, dx, dy, dz);
                d2 = f_fma<CT>(dz, dz, f_fma<CT>(dy, dy, dx * dx));
                hit = (d2 >= rlo2) && (d2 < rhi2);
                if (hit) {
                    float fx = (float)dx, fy = (float)dy, fz = (float)dz;
                    float sg = supp_g(fx, bmin[0], bmax[0]) + supp_g(fy, bmin[1], bmax[1]) + supp_g(fz, bmin[2], bmax[2]);
                    if (sg < -stol) hit = false;
                }
                // order-preserving key: d2 >= 0 so its float bits sort like the value; FP64 values are
                // rounded down so that a key never exceeds the |d|^2 it stands for
                float kf = (sizeof(CT) == 4) ? (float)d2 : __double2float_rd((double)d2);
                key = (unsigned long long)__float_as_uint(kf) << 32;
            }
            unsigned m = __ballot_sync(0xffffffffu, hit);
            int o = count + __popc(m & lt);
            if (hit && o < Cap<TP>::CAND) {
                S.u.cd.key[o] = key | (uint32_t)o;
                S.u.cd.j[o] = (uint32_t)j;
            }
            if (hit) {
                unsigned long long bb = fbits<CT>(d2);
                int b = bb <= blo ? 0 : min(HIST_BINS - 1, (int)((float)(bb - blo) * binsc));
                atomicAdd(&S.hist[b], 1u);
            }
            count += __popc(m);
            if (count > 4 * Cap<TP>::CAND) return -3;  // far too many: the caller shrinks the radius
        } else {
            int cl = lvl - 1;
            int64_t c = node * 32 + lane;
            bool hit = false;
            const int64_t span = (int64_t)1 << (5 * cl);  // sorted particles under a node of level cl
            if (c < t.count[cl] && c * span < shi && (c + 1) * span > slo) {
                float4 lo = t.lo[t.off[cl] + c], hi = t.hi[t.off[cl] + c];
                float dx = fmaxf(axis_gap(qx, lo.x, hi.x, g.Lf[0], per) - slack, 0.f);
                float dy = fmaxf(axis_gap(qy, lo.y, hi.y, g.Lf[1], per) - slack, 0.f);
                float dz = fmaxf(axis_gap(qz, lo.z, hi.z, g.Lf[2], per) - slack, 0.f);
                hit = dx * dx + dy * dy + dz * dz <= rad2;
                if (hit && inner2 > 0.f) {
                    // every point of the node already examined in an earlier pass: skip it
                    float fx = axis_far(qx, lo.x, hi.x, g.Lf[0], per) + slack;
                    float fy = axis_far(qy, lo.y, hi.y, g.Lf[1], per) + slack;
                    float fz = axis_far(qz, lo.z, hi.z, g.Lf[2], per) + slack;
                    if (fx * fx + fy * fy + fz * fz < inner2) hit = false;
                }
                if (hit) {
                    // no point of the node can cut the cell (node widened by the rounding slack of q)
                    float sx = supp_axis(qx, lo.x - slack, hi.x + slack, g.Lf[0], per, bmin[0], bmax[0]);
                    float sy = supp_axis(qy, lo.y - slack, hi.y + slack, g.Lf[1], per, bmin[1], bmax[1]);
                    float sz = supp_axis(qz, lo.z - slack, hi.z + slack, g.Lf[2], per, bmin[2], bmax[2]);
                    if (sx + sy + sz < -stol) hit = false;
                }
            }
            unsigned m = __ballot_sync(0xffffffffu, hit);
            if (sp + __popc(m) > Cap<TP>::STACK) return -2;
            if (hit) S.stack[sp + __popc(m & lt)] = ((uint32_t)cl << 27) | (uint32_t)c;
            sp += __popc(m);
            __syncwarp();
        }
    }
    return count;
}

// Bitonic sort of the candidate keys [0, n) in increasing order, in the form whose compare-exchanges
// all put the smaller key at the lower index (each merge starts by comparing every element of a block's lower half
// with its mirror in the upper half).  Keys past n stand for +inf and are never touched: a comparison with one of
// them at the higher index would leave both in place.  Keys are distinct (the collection slot is in the low bits).
template <typename CT, int TP>
__device__ void sort_cand(WarpSmem<CT, TP>& S, int n) {
    const unsigned lane = lane_id();
    unsigned long long* key = S.u.cd.key;
    int m = 1;
    while (m < n) m <<= 1;
    const int half = m >> 1;
    for (int k = 2; k <= m; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            // the first stage of a merge pairs a with its mirror a ^ (k - 1), the later ones a with a + jj
            const bool flip = jj == (k >> 1);
            for (int i = (int)lane; i < half; i += 64) {
                // pairs i and i + 32 (disjoint: every index is in one pair of a stage)
                const int i1 = i + 32;
                const int a0 = ((i & ~(jj - 1)) << 1) | (i & (jj - 1));
                const int b0 = flip ? (a0 ^ (k - 1)) : (a0 + jj);
                const int a1 = ((i1 & ~(jj - 1)) << 1) | (i1 & (jj - 1));
                const int b1 = flip ? (a1 ^ (k - 1)) : (a1 + jj);
                const bool v0 = b0 < n, v1 = i1 < half && b1 < n;
                unsigned long long x0 = 0ull, y0 = 0ull, x1 = 0ull, y1 = 0ull;
                if (v0) { x0 = key[a0]; y0 = key[b0]; }
                if (v1) { x1 = key[a1]; y1 = key[b1]; }
                if (v0 && x0 > y0) { key[a0] = y0; key[b0] = x0; }
                if (v1 && x1 > y1) { key[a1] = y1; key[b1] = x1; }
            }
            __syncwarp();
        }
    }
}

// ------------------------------------------------------------------ the cell
constexpr int RC_NEED_EXACT = 1000;
constexpr int RC_POOL = 1001;
constexpr int RC_RETRY_BOX = 1002;

// any of the six start planes an artificial wall (the small start box)
template <typename CT, int TP>
__device__ __forceinline__ bool art_walls(const WarpSmem<CT, TP>& S) {
    bool a = false;
#pragma unroll
    for (int k = 0; k < 6; k++) a |= S.pcode[k] >= CODE_ART;
    return a;
}

// successor of triangle t around plane p: the neighbour across the edge (corner before p) -> p
template <typename CT, int TP>
__device__ __forceinline__ uint32_t succ_tri(const WarpSmem<CT, TP>& S, uint32_t t, int p) {
    int k = pos_of<TP>(S.tid[t], (uint32_t)p);
    return adj_get(S.tadj[t], (k + 2) % 3);
}

// Test the lanes' planes against the vertex slots in masks[] and OR the beyond-the-plane slots into outm[].  One
// vertex per iteration, against every lane's plane; the chunks of 32 slots are taken in turn by one loop (one
// copy of the per-vertex body).  masks[] is consumed.
template <typename P, typename CT, bool EXACT, int TP>
__device__ __forceinline__ void test_slots(const WarpSmem<CT, TP>& S, unsigned* masks, bool act, CT nx, CT ny, CT nz,
                                           CT h, CT nrm, CT hb, uint32_t src, int code, unsigned* outm,
                                           const P* spos, const Geometry& g, uint32_t self, double* xws,
                                           CellCounters& cc, bool& need_exact, bool& ovf) {
#pragma unroll 1
    for (int e = 0; e < TP; e++) {
        unsigned m = pick<TP>(masks, e);
        if (!m) continue;
        unsigned o = 0u, um = 0u;
        do {
            // two slots per iteration (the second repeats the first when one is left: the same result)
            const int l0 = __ffs(m) - 1;
            m &= m - 1;
            const int l1 = m ? __ffs(m) - 1 : l0;
            m &= m - 1;
            const int sd0 = act ? side_fast<CT, TP>(S, e * 32 + l0, nx, ny, nz, h, nrm, hb) : -1;
            const int sd1 = act ? side_fast<CT, TP>(S, e * 32 + l1, nx, ny, nz, h, nrm, hb) : -1;
            o |= (sd0 > 0 ? 1u << l0 : 0u) | (sd1 > 0 ? 1u << l1 : 0u);
            um |= (sd0 == 0 ? 1u << l0 : 0u) | (sd1 == 0 ? 1u << l1 : 0u);
        } while (m);
        // the tests the error bound left undecided, slot by slot (every lane calls: resolve may use warp
        // collectives)
        unsigned ua = __reduce_or_sync(0xffffffffu, um);
        while (ua) {
            const int l = __ffs(ua) - 1;
            ua &= ua - 1;
            const bool und = (um >> l) & 1u;
            const int r = resolve<P, CT, EXACT, TP>(S, e * 32 + l, und, src, code, spos, g, self, xws, cc, need_exact, ovf);
            if (und && r > 0) o |= 1u << l;
        }
#pragma unroll
        for (int q = 0; q < TP; q++)
            if (q == e) outm[q] |= o;
    }
#pragma unroll
    for (int q = 0; q < TP; q++) masks[q] = 0u;
}

template <typename P, typename CT, bool EXACT, int TP, bool SETS>
__device__ int do_cell(WarpSmem<CT, TP>& S, const ClipArgs& A, uint32_t self, double* xws,
                                    CellCounters& cc, bool small_box) {
    const P* spos = (const P*)A.spos;
    // geometry and sorted index range of the cell's point set
    // a batch of sets: the cell's set; one set: the launch's box, read where it is used
    Geometry gs;
    int64_t slo = 0, shi = A.N;
    int k_target = A.k_target;
    if (SETS) {
        const uint32_t s = A.sset[self];
        gs = A.sgeo[s];
        slo = A.soff[s];
        shi = A.soff[s + 1];
        if (A.set_cfg) k_target = A.set_cfg[s] & 0xffff;
    }
    const Geometry& g = SETS ? gs : A.geo;
    const unsigned lane = lane_id(), lt = lanemask_lt();
    const CT u = Prec<CT>::u();
    const P pi = spos[self];
    typedef Cap<TP> K;
    CellState<TP> C;
#pragma unroll
    for (int e = 0; e < TP; e++) C.vm[e] = 0u;
    C.np = 6;
    // first radius from the bucket mates: 1.6 x the distance of the ~11th nearest
    CT rhi2;
    {
        int64_t b0 = ((int64_t)self / 32) * 32;
        int64_t j = b0 + lane;
        float d2f = INFINITY;
        if (j >= slo && j < shi && (uint32_t)j != self) {
            P pj = spos[j];
            CT dx, dy, dz;
            int code;
            DispF<P, CT>::get(pj, pi, g, dx, dy, dz, code);
            d2f = (float)f_fma<CT>(dz, dz, f_fma<CT>(dy, dy, dx * dx));
        }
        for (int k = 2; k <= 32; k <<= 1)
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                float o = __shfl_xor_sync(0xffffffffu, d2f, jj);
                bool up = ((lane & k) == 0);
                bool lower = (lane & jj) == 0;
                float mn = fminf(d2f, o), mx = fmaxf(d2f, o);
                d2f = (lower == up) ? mn : mx;
            }
        int kk = min(max(k_target / 4, 4), 30);
        float dk = __shfl_sync(0xffffffffu, d2f, kk);
        if (!(dk < INFINITY)) {
            float mx = d2f < INFINITY ? d2f : 0.f;
            mx = warp_max<float>(mx);
            if (mx > 0.f) dk = mx;
            else {
                double vol = g.L[0] * g.L[1] * g.L[2];
                double sp = cbrt(vol / (double)(shi - slo));
                dk = (float)(4.0 * sp * sp);
            }
        }
        rhi2 = (CT)dk * (CT)2.6;
    }
    // Initial polytope.  With small_box the cell starts as a cube of half-side B = 3 r (r the first search
    // radius) made of artificial walls: a polytope on the scale of the cell keeps the vertex error bounds
    // small (the box of the periodic self-images has vertices at L/2).  If the final cell still touches an
    // artificial wall the box was too small and the caller redoes the cell without it.  Otherwise the
    // periodic self-images (x_i +- L e_k) or the box walls bound the cell.
    const double lminb = fmin(g.L[0], fmin(g.L[1], g.L[2]));
    const float Bf = small_box ? (float)(3.0 * sqrt((double)rhi2)) : 0.f;
    if (lane < 6) {
        int axis = lane >> 1;
        bool upper = (lane & 1) == 0;
        CT nx = 0, ny = 0, nz = 0, h, nrm;
        int code;
        uint32_t src = self;
        double xi = axis == 0 ? (double)pi.x : axis == 1 ? (double)pi.y : (double)pi.z;
        double real = g.periodic ? 0.5 * g.L[axis] : (upper ? g.hi[axis] - xi : xi - g.lo[axis]);
        if (small_box && (double)Bf < (g.periodic ? 0.49 * lminb : real)) {
            CT sg = upper ? (CT)1 : (CT)-1;
            if (axis == 0) nx = sg; else if (axis == 1) ny = sg; else nz = sg;
            h = (CT)Bf;
            nrm = (CT)1;
            code = CODE_ART + (int)lane;
            src = __float_as_uint(Bf);
        } else if (g.periodic) {
            CT Lc = (CT)g.L[axis];
            CT sg = upper ? Lc : -Lc;
            if (axis == 0) nx = sg; else if (axis == 1) ny = sg; else nz = sg;
            h = (CT)(0.5 * g.L[axis] * g.L[axis]);
            nrm = Lc;
            int sh[3] = {0, 0, 0};
            sh[axis] = upper ? 1 : -1;
            code = code_of(sh[0], sh[1], sh[2]);
        } else {
            CT sg = upper ? (CT)1 : (CT)-1;
            if (axis == 0) nx = sg; else if (axis == 1) ny = sg; else nz = sg;
            h = (CT)real;
            nrm = (CT)1;
            code = CODE_WALL + (int)lane;
        }
        Pln<CT> pq;
        pq.x = nx; pq.y = ny; pq.z = nz; pq.h = h;
        S.pl[lane] = pq;
        S.pnrm[lane] = nrm;
        S.psrc[lane] = src; S.pcode[lane] = (uint8_t)code;
    }
    __syncwarp();
    // 8 corners: planes x upper 0 / lower 1, y 2/3, z 4/5; (X,Y,Z) if the sign product is positive, else
    // (X,Z,Y): every triangle then lists its planes counter-clockwise seen from outside
    if (lane < 8) {
        int sx = (lane & 1) ? -1 : 1, sy = (lane & 2) ? -1 : 1, sz = (lane & 4) ? -1 : 1;
        uint32_t X = (lane & 1) ? 1 : 0, Y = (lane & 2) ? 3 : 2, Z = (lane & 4) ? 5 : 4;
        S.tid[lane] = (sx * sy * sz > 0) ? pack<TP>(X, Y, Z) : pack<TP>(X, Z, Y);
        tri_vertex<CT, TP>(S, lane);
    }
    __syncwarp();
    if (lane < 8) {
        // adjacency of the initial octahedron: the triangles above list planes (0,2,4), (1,4,2), (0,4,3), (1,3,4),
        // (0,5,2), (1,2,5), (0,3,5), (1,5,3); across each edge x->y lies the triangle holding y->x, packed as
        // adj_pack(n0, n1, n2): lane 0 (4,1,2), 1 (3,0,5), 2 (0,3,6), 3 (7,2,1), 4 (6,5,0), 5 (1,4,7), 6 (2,7,4),
        // 7 (5,6,3)
        const uint32_t adj = lane == 0 ? adj_pack(4, 1, 2) : lane == 1 ? adj_pack(3, 0, 5) : lane == 2 ? adj_pack(0, 3, 6)
                           : lane == 3 ? adj_pack(7, 2, 1) : lane == 4 ? adj_pack(6, 5, 0) : lane == 5 ? adj_pack(1, 4, 7)
                           : lane == 6 ? adj_pack(2, 7, 4) : adj_pack(5, 6, 3);
        S.tadj[lane] = adj;
    }
    C.vm[0] = 0xFFu;
    C.hw = 8;
    __syncwarp();
    float bmin[3], bmax[3];
    CT R2 = radius_box<CT, TP>(S, C, bmin, bmax);

    CT rlo2 = 0;
    const double lmin = fmin(g.L[0], fmin(g.L[1], g.L[2]));
    CT cap2 = g.periodic ? (CT)(0.249 * lmin * lmin)
                         : (CT)(4.0 * (g.L[0] * g.L[0] + g.L[1] * g.L[1] + g.L[2] * g.L[2]));
    bool done = false;
    bool need_exact = false, ovf = false;
    for (int pass = 0; pass < A.max_passes && !done; pass++) {
        cc.n_passes++;
        if (rhi2 > cap2) rhi2 = cap2;
        int cnt = -1;
        VT_T0(tc0);
        for (int shrink = 0; shrink < 64; shrink++) {
            cnt = collect<P, CT, TP>(S, spos, A.N, g, A.tree, self, pi, rlo2, rhi2, bmin, bmax, slo, shi);
            cc.n_collect++;
            if (cnt > 0) cc.n_collected += cnt;
            if (cnt == -2) return CAP_STACK;
            if (cnt == -3) {  // aborted: halve the radius step and retry
                CT r = sqrt(rhi2), rl = sqrt(rlo2);
                CT rn = rl + (CT)0.5 * (r - rl);
                CT rn2 = rn * rn;
                rhi2 = rn2 > rlo2 ? rn2 : fromfbits<CT>(fbits<CT>(rlo2) + 1);
                cnt = -1;
                continue;
            }
            if (cnt <= K::CAND) break;
            // too many: keep the largest prefix of histogram bins that fits (at least the first bin, narrowed
            // again if needed)
            __syncwarp();
            int keep = 0, acc = 0;
            for (int b = 0; b < HIST_BINS; b++) {
                acc += (int)S.hist[b];
                if (acc > K::CAND) break;
                keep = b + 1;
            }
            unsigned long long blo = fbits<CT>(rlo2), bhi = fbits<CT>(rhi2);
            // exact integer split of the bit-pattern range (a bin that the float binning put a point in may
            // shift by one; the loop only needs the count to drop)
            unsigned long long nb = blo + (bhi - blo) / HIST_BINS * (unsigned long long)(keep > 0 ? keep : 1);
            if (nb <= blo) nb = blo + 1;
            if (nb >= bhi) return CAP_CAND;
            rhi2 = fromfbits<CT>(nb);
            cnt = -1;
        }
        if (cnt < 0 || cnt > K::CAND) return CAP_CAND;
        __syncwarp();
        VT_T1(cc, 0, tc0);
        VT_T0(ts0);
        sort_cand<CT, TP>(S, cnt);
        VT_T1(cc, 1, ts0);
        // candidates in batches of 32, one per lane, in increasing distance
        for (int k0 = 0; k0 < cnt && !done; k0 += 32) {
            const int k = k0 + (int)lane;
            const bool valid = k < cnt;
            CT dx = 0, dy = 0, dz = 0;
            uint32_t j = 0;
            int code = 13;
            float kf = INFINITY;
            if (valid) {
                unsigned long long key = S.u.cd.key[k];
                uint32_t slot = (uint32_t)(key & 0xffffffffu);
                kf = __uint_as_float((uint32_t)(key >> 32));
                j = S.u.cd.j[slot];
                // the displacement exactly as the search computed it (the same rounding; no shift for a point
                // the search found without one)
                DispF<P, CT>::get(spos[j], pi, g, dx, dy, dz, code);
            }
            // security radius: a plane at |d| >= 2R cannot cut; keys only grow along the list
            const bool far = valid && (CT)kf * ((CT)1 - (CT)8 * u) > (CT)4 * R2;
            const unsigned farm = __ballot_sync(0xffffffffu, far);
            const unsigned valm = __ballot_sync(0xffffffffu, valid);
            const int nact = farm ? __ffs(farm) - 1 : __popc(valm);
            const bool act = (int)lane < nact;
            CT d2 = f_fma<CT>(dz, dz, f_fma<CT>(dy, dy, dx * dx));
            if (__any_sync(0xffffffffu, act && d2 == (CT)0)) return VT_ERR_DUPLICATE;
            const CT h = (CT)0.5 * d2;
            const CT nrm = sqrt(d2);
            const CT hb = (CT)16 * u * h;
            // test every vertex against the batch's planes; then apply the cutting planes in order, re-testing
            // only the new vertices against the later planes (a plane that misses a polytope misses every subset)
            unsigned outm[TP], tmask[TP];
#pragma unroll
            for (int e = 0; e < TP; e++) { outm[e] = 0u; tmask[e] = nact > 0 ? C.vm[e] : 0u; }
            cc.n_tested += nact;
            bool any_cut = false;
            int last = -1;
            VT_T0(tk0);
#pragma unroll 1
            for (;;) {
                VT_T0(tt0);
                test_slots<P, CT, EXACT, TP>(S, tmask, act && (int)lane > last, dx, dy, dz, h, nrm, hb, j, code, outm,
                                             spos, g, self, xws, cc, need_exact, ovf);
                VT_T1(cc, 2, tt0);
                if (!EXACT && __any_sync(0xffffffffu, need_exact)) return RC_NEED_EXACT;
                if (EXACT && __any_sync(0xffffffffu, ovf)) return VT_ERR_NUMERIC;
                unsigned anyo = 0u;
#pragma unroll
                for (int e = 0; e < TP; e++) anyo |= outm[e];
                const unsigned cutm = __ballot_sync(0xffffffffu, act && (int)lane > last && anyo);
                if (!cutm) break;
                const int L = __ffs(cutm) - 1;
                unsigned rem[TP];
#pragma unroll
                for (int e = 0; e < TP; e++) rem[e] = __shfl_sync(0xffffffffu, outm[e], L);
                CT px = __shfl_sync(0xffffffffu, dx, L), py = __shfl_sync(0xffffffffu, dy, L),
                   pz = __shfl_sync(0xffffffffu, dz, L), ph = __shfl_sync(0xffffffffu, h, L),
                   pn = __shfl_sync(0xffffffffu, nrm, L);
                uint32_t pj = __shfl_sync(0xffffffffu, j, L);
                int pc = __shfl_sync(0xffffffffu, code, L);
                VT_T0(ta0);
                int rc = apply_cut<CT, TP>(S, C, rem, px, py, pz, ph, pn, pj, pc, tmask);
                VT_T1(cc, 6, ta0);
                if (rc) return rc;
                cc.n_cut++;
                any_cut = true;
                last = L;
#pragma unroll
                for (int e = 0; e < TP; e++) outm[e] &= ~rem[e];
            }
            if (any_cut) {
                VT_T0(tb0);
                R2 = radius_box<CT, TP>(S, C, bmin, bmax);
                VT_T1(cc, 8, tb0);
            }
            VT_T1(cc, 3, tk0);
            if (farm) done = true;  // the list reached |d| > 2R: certified
        }
        __syncwarp();
        if (done) break;
        // every particle with |d|^2 < rhi2 has been examined
        if (rhi2 * ((CT)1 - (CT)8 * u) >= (CT)4 * R2) { done = true; break; }
        // an ill-conditioned vertex (infinite error bound) blocks the certificate: redo the cell in FP64
        if (!EXACT && !(R2 < (CT)INFINITY)) return RC_NEED_EXACT;
        // the widest search did not certify the cell: if an artificial wall of the small start box still bounds
        // it (a cell in a void larger than the box), redo it from the true walls; otherwise give up
        if (rhi2 >= cap2) return art_walls(S) ? RC_RETRY_BOX : g.periodic ? VT_ERR_UNSUPPORTED : VT_ERR_SECURITY;
        // next pass: the annulus up to 2R, at most twice the radius (policy 1: also no further than the radius
        // that the density seen so far says holds about 3/4 of a pass's capacity)
        {
            CT nxt = (CT)4 * R2 * ((CT)1 + (CT)32 * u);
            float lim = 4.f * (float)rhi2;
            if (A.radius_policy == 1 && cnt > 0) {
                float rh = sqrtf((float)rhi2), rl = sqrtf((float)rlo2);
                float shell = rh * rh * rh - rl * rl * rl;
                if (shell > 0.f) {
                    float r = cbrtf(rh * rh * rh + 0.75f * K::CAND * shell / (float)cnt);
                    lim = fminf(lim, fmaxf(r * r, 1.21f * (float)rhi2));
                }
            }
            rlo2 = rhi2;
            rhi2 = nxt < (CT)lim ? nxt : (CT)lim;
        }
    }
    if (!done) return art_walls(S) ? RC_RETRY_BOX : (!EXACT && !(R2 < (CT)INFINITY)) ? RC_NEED_EXACT : VT_ERR_SECURITY;
    if (g.periodic && !((CT)16 * R2 < (CT)(lmin * lmin))) return VT_ERR_UNSUPPORTED;

    // ---------------- emission: one triangle per plane present, then walks along the adjacency
    __syncwarp();
    VT_T0(te0);
    for (int k = (int)lane; k < K::MAXP; k += 32) S.u.em.first[k] = 0xffffffffu;
    __syncwarp();
#pragma unroll
    for (int e = 0; e < TP; e++) {
        if ((C.vm[e] >> lane) & 1u) {
            uint32_t t = e * 32 + lane;
            uint32_t a, b, c;
            unpack<TP>(S.tid[t], a, b, c);
            atomicMin(&S.u.em.first[a], t);
            atomicMin(&S.u.em.first[b], t);
            atomicMin(&S.u.em.first[c], t);
        }
    }
    __syncwarp();
    // a facet on an initial plane: an artificial wall means the start box was too small (redo without it);
    // a box wall (bounded) is fine; an own periodic image is not supported
    {
        bool on = (lane < 6) && S.u.em.first[lane] != 0xffffffffu;
        bool art = on && S.pcode[lane] >= CODE_ART;
        if (__any_sync(0xffffffffu, art)) return RC_RETRY_BOX;
        if (g.periodic && __any_sync(0xffffffffu, on)) return VT_ERR_UNSUPPORTED;
    }
    // facets: lane (chunk c) walks plane c*32+lane; fan from the facet's first vertex.  The facet records are
    // reserved first (a facet is a plane present that is a bisector) and written as their sums come out.
    constexpr int PCH = K::MAXP / 32;
    int nf_total = 0;
#pragma unroll
    for (int c = 0; c < PCH; c++) {
        const int p = c * 32 + (int)lane;
        const bool f = p < C.np && p >= 6 && S.pcode[p] < 27 && S.u.em.first[p] != 0xffffffffu;
        nf_total += __popc(__ballot_sync(0xffffffffu, f));
    }
    uint32_t start = 0;
    if (lane == 0 && nf_total > 0) {
        unsigned long long s0 = atomicAdd(&A.st->face_next, (unsigned long long)nf_total);
        start = (s0 + nf_total <= A.face_cap) ? (uint32_t)s0 : 0xffffffffu;
    }
    start = __shfl_sync(0xffffffffu, start, 0);
    if (start == 0xffffffffu) return RC_POOL;
    // the volume (and each facet area) is summed with compensation; the moments plainly
    KSum<CT> kvol;
    kvol.zero();
    CT mzx = 0, mzy = 0, mzz = 0, m2 = 0;
    int acc = 0;
#pragma unroll 1
    for (int c = 0; c < PCH; c++) {
        if (c * 32 >= C.np) break;
        int p = c * 32 + (int)lane;
        bool present = p < C.np && S.u.em.first[p] != 0xffffffffu;
        const bool fem = present && (p >= 6) && S.pcode[p] < 27;
        const unsigned fm = __ballot_sync(0xffffffffu, fem);
        if (present) {
            uint32_t t0 = S.u.em.first[p];
            const Vtx<CT> v0 = S.tv[t0];
            CT x0 = v0.x, y0 = v0.y, z0 = v0.z;
            CT inrm = (CT)1 / S.pnrm[p];
            const Pln<CT> pp = S.pl[p];
            CT nhx = pp.x * inrm, nhy = pp.y * inrm, nhz = pp.z * inrm;
            KSum<CT> kA;
            kA.zero();
            CT csx = 0, csy = 0, csz = 0, sm2 = 0;
            uint32_t cur = succ_tri<CT, TP>(S, t0, p);
            for (int guard = 0; guard < K::MAXT && cur != t0; guard++) {
                uint32_t nxt = succ_tri<CT, TP>(S, cur, p);
                if (nxt == t0) break;
                const Vtx<CT> v1 = S.tv[cur], v2 = S.tv[nxt];
                CT x1 = v1.x, y1 = v1.y, z1 = v1.z;
                CT x2 = v2.x, y2 = v2.y, z2 = v2.z;
                CT e1x = x1 - x0, e1y = y1 - y0, e1z = z1 - z0;
                CT e2x = x2 - x0, e2y = y2 - y0, e2z = z2 - z0;
                CT crx = f_fma<CT>(e1y, e2z, -e1z * e2y), cry = f_fma<CT>(e1z, e2x, -e1x * e2z),
                   crz = f_fma<CT>(e1x, e2y, -e1y * e2x);
                CT at = (CT)0.5 * f_fma<CT>(crx, nhx, f_fma<CT>(cry, nhy, crz * nhz));
                kA.add(at);
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
            const CT A_ = kA.value();
            // distance from the site to the facet plane; tetrahedra (site, fan triangle) give
            // V_f = dist A_f / 3, first moment dist * sum(at (v0+v1+v2)/3) / 4, second moment dist/30 * sum(at s2)
            CT dist = pp.h * inrm;
            kvol.add(dist * A_ * (CT)(1.0 / 3.0));
            mzx += dist * csx * (CT)0.25;
            mzy += dist * csy * (CT)0.25;
            mzz += dist * csz * (CT)0.25;
            m2 += dist * sm2 * (CT)(1.0 / 30.0);
            if (fem) {
                Face f;
                f.dx = (float)pp.x; f.dy = (float)pp.y; f.dz = (float)pp.z;
                f.area = (float)A_;
                if (A_ != (CT)0) { f.cx = (float)(csx / A_); f.cy = (float)(csy / A_); f.cz = (float)(csz / A_); }
                else { f.cx = f.cy = f.cz = 0.f; }
                f.nbr = S.psrc[p];
                A.faces[start + acc + __popc(fm & lanemask_lt())] = f;
            }
        }
        acc += __popc(fm);
    }
    kvol.warp_reduce();
    CT vol = kvol.value();
    m2 = warp_sum<CT>(m2);
    mzx = warp_sum<CT>(mzx); mzy = warp_sum<CT>(mzy); mzz = warp_sum<CT>(mzz);
    const CT sg = vol < 0 ? (CT)-1 : (CT)1;
    vol *= sg; m2 *= sg;
    if (sg < 0) {
        // reversed orientation: the areas were written with the opposite sign
        for (int k = (int)lane; k < nf_total; k += 32) A.faces[start + k].area = -A.faces[start + k].area;
    }
    if (lane == 0) {
        CellOut co;
        co.vol = (double)vol;
        co.zx = (float)(vol > 0 ? sg * mzx / vol : (CT)0);
        co.zy = (float)(vol > 0 ? sg * mzy / vol : (CT)0);
        co.zz = (float)(vol > 0 ? sg * mzz / vol : (CT)0);
        co.mom2 = (float)m2;
        A.cell[self] = co;
        if (A.rad) A.rad[self] = (float)sqrt((double)R2) * (1.f + 1e-6f);
        A.face_start[self] = start;
        A.face_count[self] = (uint16_t)nf_total;
        atomicMax(&A.st->max_faces, (unsigned)nf_total);
        atomicAdd(&A.st->n_faces, (unsigned long long)nf_total);
    }
    VT_T1(cc, 4, te0);
    return 0;
}

// Fast kernels: Cap<4>, CLIP_WARPS warps per block, every cell; cells they cannot finish (an undecided FP64
// test, an ill-conditioned vertex or a capacity overflow) are appended to the exact list.
// Exact kernel: Cap<16>, one warp per block, the listed cells, exact predicates.
template <typename P, typename CT, bool EXACT, int TP, int WPB, bool SETS>
__global__ void __launch_bounds__(WPB * 32) k_clip(ClipArgs A) {
    extern __shared__ __align__(32) unsigned char smem_raw[];
    const int w = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    WarpSmem<CT, TP>& S = reinterpret_cast<WarpSmem<CT, TP>*>(smem_raw)[w];
    const int gw = blockIdx.x * WPB + w;
    double* xws = EXACT ? (A.xws + (size_t)gw * EXACT_WS) : nullptr;
    // rejected input (NaN or out-of-box coordinates, recorded by the key kernel before this launch): no cells
    if (*((volatile unsigned*)&A.st->invalid_input)) return;
    CellCounters cc = {};
    const uint32_t total = EXACT ? 0u : (uint32_t)A.N;
    for (;;) {
        uint32_t base = 0;
        const unsigned chunk = EXACT ? 1u : (unsigned)CHUNK;
        if (lane == 0) base = atomicAdd(EXACT ? &A.st->work_next_exact : &A.st->work_next, chunk);
        base = __shfl_sync(0xffffffffu, base, 0);
        const bool listed = !EXACT && A.warp_list != nullptr;
        uint32_t lim = EXACT ? *((volatile unsigned*)&A.st->n_exact_cells)
                             : listed ? *((volatile unsigned*)&A.st->n_warp_cells) : total;
        if (base >= lim) break;
        for (uint32_t q = base; q < base + chunk && q < lim; q++) {
            uint32_t self = EXACT ? A.exact_list[q] : listed ? A.warp_list[q] : q;
            VT_T0(tall);
            const unsigned f64_before = cc.n_fp64;
            // one call site (the cell routine is inlined once): the small start box first, then, if the cell
            // reached one of its artificial walls, the true walls
            int rc = 0;
#pragma unroll 1
            for (int attempt = 0; attempt < 2; attempt++) {
                rc = do_cell<P, CT, EXACT, TP, SETS>(S, A, self, xws, cc, !EXACT && attempt == 0);
                if (rc != RC_RETRY_BOX) break;
            }
            VT_T1(cc, 5, tall);
            const bool used64 = __any_sync(0xffffffffu, cc.n_fp64 != f64_before);
            __syncwarp();
            if (!EXACT && rc <= -100) rc = RC_NEED_EXACT;  // capacity: the larger exact kernel takes the cell
            if (lane == 0) {
                if (rc == 0) {
                    A.cstat[self] = EXACT ? (uint8_t)(CS_DONE | CS_EXACT | (A.cstat[self] & CS_FP64))
                                          : (uint8_t)(CS_DONE | (used64 ? CS_FP64 : 0));
                } else if (rc == RC_NEED_EXACT) {
                    A.cstat[self] = (uint8_t)(CS_NEED_EXACT | (used64 ? CS_FP64 : 0));
                    unsigned slot = atomicAdd(&A.st->n_exact_cells, 1u);
                    A.exact_list[slot] = self;
                } else {
                    A.cstat[self] = CS_ERROR;
                    int code = rc <= -100 ? VT_ERR_CAPACITY : rc;
                    if (atomicCAS(&A.st->error, 0, code) == 0) {
                        A.st->error_cell = (int)self;
                        A.st->error_detail = rc;
                    }
                }
            }
        }
    }
    // n_fp64 / n_exact / n_zero are counted by the lanes that did the work; the others are warp-uniform
    unsigned f64 = cc.n_fp64, xe = cc.n_exact, xz = cc.n_zero;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        f64 += __shfl_xor_sync(0xffffffffu, f64, o);
        xe += __shfl_xor_sync(0xffffffffu, xe, o);
        xz += __shfl_xor_sync(0xffffffffu, xz, o);
    }
    cc.n_fp64 = f64; cc.n_exact = xe; cc.n_zero = xz;
#ifdef VT_PHASE_TIMERS
    {
        unsigned long long t9 = cc.t[9];
        for (int o = 16; o; o >>= 1) t9 += __shfl_xor_sync(0xffffffffu, t9, o);
        cc.t[9] = t9;
    }
#endif
    if (lane == 0) {
        atomicAdd(&A.st->n_cut, (unsigned long long)cc.n_cut);
        atomicAdd(&A.st->n_tested, (unsigned long long)cc.n_tested);
        atomicAdd(&A.st->n_passes, (unsigned long long)cc.n_passes);
        atomicAdd(&A.st->n_fp64, (unsigned long long)cc.n_fp64);
        atomicAdd(&A.st->n_exact_preds, (unsigned long long)cc.n_exact);
        atomicAdd(&A.st->n_exact_zero, (unsigned long long)cc.n_zero);
        atomicAdd(&A.st->n_collect, (unsigned long long)cc.n_collect);
        atomicAdd(&A.st->n_collected, (unsigned long long)cc.n_collected);
#ifdef VT_PHASE_TIMERS
        for (int k = 0; k < 10; k++) atomicAdd(&A.st->t_phase[k], cc.t[k]);
#endif
    }
}

}  // namespace vt

namespace vt {
template <typename P, typename CT, bool EXACT, bool SETS>
static void launch_one_t(const ClipArgs& a, int sm_count, cudaStream_t s) {
    constexpr int TP = EXACT ? 16 : 4;
    constexpr int WPB = EXACT ? 1 : CLIP_WARPS;
    size_t smem = sizeof(WarpSmem<CT, TP>) * WPB;
    // the shared-memory attribute and the occupancy are set up once per device (no such call is made while a
    // stream is being captured, after the first launch)
    static int per_sm_dev[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    int per_sm = (dev >= 0 && dev < 64) ? per_sm_dev[dev] : 0;
    if (per_sm == 0) {
        cudaFuncSetAttribute(k_clip<P, CT, EXACT, TP, WPB, SETS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_clip<P, CT, EXACT, TP, WPB, SETS>, WPB * 32, smem);
        if (per_sm < 1) per_sm = 1;
        if (dev >= 0 && dev < 64) per_sm_dev[dev] = per_sm;
    }
    int blocks = sm_count * per_sm;
    if (EXACT) blocks = a.xws_warps < blocks ? a.xws_warps : blocks;
    k_clip<P, CT, EXACT, TP, WPB, SETS><<<blocks, WPB * 32, smem, s>>>(a);
}
template <typename P, typename CT, bool EXACT>
static void launch_one(const ClipArgs& a, int sm_count, cudaStream_t s) {
    if (a.sset) launch_one_t<P, CT, EXACT, true>(a, sm_count, s);
    else launch_one_t<P, CT, EXACT, false>(a, sm_count, s);
}
}  // namespace vt
