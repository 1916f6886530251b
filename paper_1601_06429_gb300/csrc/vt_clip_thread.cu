// vt_clip_thread.cu -- the bulk clipping kernels: one thread per cell (a warp per bucket of 32 cells), or 4 or 8
// lanes per cell (further down); and the voxel-grid and weighted-moment kernels that rebuild cells from their facets.
//
// The warp kernel (vt_clip_impl.cuh) spends a whole warp on one cell, and most of its instructions on
// cross-lane steps (candidate search, ballots, shuffles).  Here the 32 cells of a tree bucket (32 consecutive
// particles in Morton order, so neighbours in space) share one candidate search: the warp walks the tree once
// per radius pass and streams the points near the bucket's box through shared memory in chunks; every lane then
// clips its own cell against the chunk, in registers and its own local memory.  The clipping, the predicates
// and the emitted records are those of the warp kernel:
//   * the cell is the intersection of half-spaces n.y <= h (n = x_j - x_i, h = |n|^2/2), held as its dual
//     triangulation (one triangle of plane ids per vertex, listed counter-clockwise seen from outside);
//   * a vertex is strictly beyond a plane when n.v - h exceeds the forward error bound of make_vertex; an
//     undecided test is redone in FP64 from the input coordinates (side64);
//   * a plane at |n| >= 2R (R bounds the distance of every vertex) cannot cut, and a cell is final once every
//     point closer than 2R has been examined (the security radius).
// A cell this kernel cannot finish -- an FP64 test that stays undecided, an ill-conditioned vertex, a cell
// larger than its capacities, a start box that was too small, a duplicate point, or a security radius beyond
// the passes it makes -- goes to a list that the warp kernel then takes (and from there, if needed, the exact
// kernel).  Every decision this kernel takes is certified, so both kernels produce the same cells.
#include <climits>

#include "vt_clip_impl.cuh"

namespace vt {
namespace {

constexpr int TT = 64;        // triangles (cell vertices) per cell
constexpr int TPL = 40;       // planes per cell: the six start walls and the cuts
constexpr int TCH = 256;      // points per chunk
constexpr int TSTK = 256;     // traversal stack entries per warp
constexpr int TWARPS = 4;     // warps per block
constexpr int TPASSES = 6;    // radius passes per bucket
constexpr int TMAXPTS = 16384;  // points streamed per bucket before the remaining cells are handed over

// lane-local cell.  V: vertex (x, y, z) relative to the site and its error bound; Tr: three 8-bit plane ids;
// Pl: plane (n, h); Pn: |n|; Ps / Pc: the plane's source (sorted index, or the bits of an artificial wall's h)
// and code (periodic image 0..26, box wall 27+w, artificial wall 33+w).
template <int NT, int NP>
struct TCellT {
    static constexpr int MT = NT, MP = NP;  // capacities: triangles (a multiple of 32), planes (at most 255)
    float4 V[NT];
    uint32_t Tr[NT];
    float4 Pl[NP];
    float Pn[NP];
    uint32_t Ps[NP];
    uint8_t Pc[NP];
    int nT, nP;
    float R2;          // >= the squared distance of every exact vertex
    float bmin[3], bmax[3];
};
typedef TCellT<TT, TPL> TCell;       // the clipping kernel's cell
typedef TCellT<128, 96> TCellBig;   // grid averages of cells beyond it

struct TSmem {
    float4 chunk[TCH];     // x, y, z, sorted index (bits)
    uint32_t key[TCH];     // distance-to-box-centre bits (low 8 bits cleared) | slot
    uint32_t stack[TSTK];  // level << 27 | node
};

// local failure codes (the cell goes to the warp kernel)
constexpr int TF_CAP = 1, TF_ILL = 2, TF_UNDECIDED = 3, TF_DUP = 4, TF_WALL = 5, TF_RADIUS = 6, TF_CAP_CUT = 7,
              TF_CAP_PLANES = 8, TF_SKIP = 9;  // TF_SKIP: the cell's set is configured for the warp kernel

__device__ __forceinline__ void tri_ids(uint32_t t, uint32_t& a, uint32_t& b, uint32_t& c) {
    a = t & 255u; b = (t >> 8) & 255u; c = (t >> 16) & 255u;
}

template <class CL>
__device__ __forceinline__ bool vertex_of(const CL& C, uint32_t a, uint32_t b, uint32_t c, float4& v) {
    const float4 A = C.Pl[a], B = C.Pl[b], Cc = C.Pl[c];
    float vx, vy, vz, ev, rr;
    make_vertex<float>(A.x, A.y, A.z, A.w, C.Pn[a], B.x, B.y, B.z, B.w, C.Pn[b], Cc.x, Cc.y, Cc.z, Cc.w, C.Pn[c],
                       vx, vy, vz, ev, rr);
    v = make_float4(vx, vy, vz, ev);
    return ev < INFINITY;
}

// R2 and the outward-rounded box of the exact vertices
template <class CL>
__device__ void bound_cell(CL& C) {
    float r2 = 0.f, lo0 = 0.f, lo1 = 0.f, lo2 = 0.f, hi0 = 0.f, hi1 = 0.f, hi2 = 0.f;
    for (int t = 0; t < C.nT; t++) {
        const float4 v = C.V[t];
        float r = __fadd_ru(__fsqrt_ru(__fmaf_ru(v.z, v.z, __fmaf_ru(v.y, v.y, __fmul_ru(v.x, v.x)))), v.w);
        r2 = fmaxf(r2, __fmul_ru(r, r));
        lo0 = fminf(lo0, __fsub_rd(v.x, v.w)); hi0 = fmaxf(hi0, __fadd_ru(v.x, v.w));
        lo1 = fminf(lo1, __fsub_rd(v.y, v.w)); hi1 = fmaxf(hi1, __fadd_ru(v.y, v.w));
        lo2 = fminf(lo2, __fsub_rd(v.z, v.w)); hi2 = fmaxf(hi2, __fadd_ru(v.z, v.w));
    }
    C.R2 = r2 * (1.f + 1e-6f);
    C.bmin[0] = lo0; C.bmin[1] = lo1; C.bmin[2] = lo2;
    C.bmax[0] = hi0; C.bmax[1] = hi1; C.bmax[2] = hi2;
}

// Start polytope: the box of half-side B around the site (artificial walls), cut by the real box walls when
// the set is bounded and a wall is closer.  Returns 0 or a failure code.
template <typename P, class CL>
__device__ int init_cell(CL& C, const Geometry& g, const P& pi, uint32_t self, float B) {
    for (int w = 0; w < 6; w++) {
        const int axis = w >> 1;
        const bool upper = (w & 1) == 0;
        const double xi = axis == 0 ? (double)pi.x : axis == 1 ? (double)pi.y : (double)pi.z;
        const double real = upper ? g.hi[axis] - xi : xi - g.lo[axis];
        const float sg = upper ? 1.f : -1.f;
        float4 pl = make_float4(axis == 0 ? sg : 0.f, axis == 1 ? sg : 0.f, axis == 2 ? sg : 0.f, 0.f);
        if (!g.periodic && real <= (double)B) {
            pl.w = (float)real;
            C.Ps[w] = self;
            C.Pc[w] = (uint8_t)(CODE_WALL + w);
        } else {
            pl.w = B;
            C.Ps[w] = __float_as_uint(B);
            C.Pc[w] = (uint8_t)(CODE_ART + w);
        }
        C.Pl[w] = pl;
        C.Pn[w] = 1.f;
    }
    C.nP = 6;
    // corners: planes x upper 0 / lower 1, y 2/3, z 4/5, counter-clockwise seen from outside
    for (int k = 0; k < 8; k++) {
        const int sx = (k & 1) ? -1 : 1, sy = (k & 2) ? -1 : 1, sz = (k & 4) ? -1 : 1;
        const uint32_t X = (k & 1) ? 1 : 0, Y = (k & 2) ? 3 : 2, Z = (k & 4) ? 5 : 4;
        const uint32_t t = (sx * sy * sz > 0) ? (X | (Y << 8) | (Z << 16)) : (X | (Z << 8) | (Y << 16));
        C.Tr[k] = t;
        float4 v;
        uint32_t a, b, c;
        tri_ids(t, a, b, c);
        if (!vertex_of(C, a, b, c, v)) return TF_ILL;
        C.V[k] = v;
    }
    C.nT = 8;
    bound_cell(C);
    return 0;
}

// Drop plane ids that no triangle uses (the start walls keep theirs).  Returns false if none is free.
template <class CL>
__device__ bool compact_planes(CL& C) {
    uint32_t used[(CL::MP + 31) / 32];
    for (int w = 0; w < (CL::MP + 31) / 32; w++) used[w] = 0u;
    used[0] = 0x3fu;
    for (int t = 0; t < C.nT; t++) {
        uint32_t a, b, c;
        tri_ids(C.Tr[t], a, b, c);
        used[a >> 5] |= 1u << (a & 31);
        used[b >> 5] |= 1u << (b & 31);
        used[c >> 5] |= 1u << (c & 31);
    }
    uint8_t map[CL::MP];
    int n = 0;
    for (int p = 0; p < C.nP; p++) {
        if ((used[p >> 5] >> (p & 31)) & 1u) {
            if (n != p) {
                C.Pl[n] = C.Pl[p]; C.Pn[n] = C.Pn[p]; C.Ps[n] = C.Ps[p]; C.Pc[n] = C.Pc[p];
            }
            map[p] = (uint8_t)n++;
        }
    }
    if (n == C.nP) return false;
    for (int t = 0; t < C.nT; t++) {
        uint32_t a, b, c;
        tri_ids(C.Tr[t], a, b, c);
        C.Tr[t] = (uint32_t)map[a] | ((uint32_t)map[b] << 8) | ((uint32_t)map[c] << 16);
    }
    C.nP = n;
    return true;
}

// Cut by plane (n, h) known to remove exactly the triangles in bm[].  Every directed edge x->y of a removed
// triangle whose reverse y->x is in no removed triangle lies on the boundary of the removed region (its
// neighbour across is kept) and becomes the new triangle (x, y, p).  New triangles fill the removed slots; the
// array is then compacted.  Returns 0 or a failure code.
template <class CL>
__device__ int cut_cell(CL& C, const unsigned* bm, float nx, float ny, float nz, float h, float nrm, uint32_t src,
                        int code) {
    if (C.nP >= CL::MP && !compact_planes(C)) return TF_CAP_PLANES;
    const uint32_t p = (uint32_t)C.nP++;
    C.Pl[p] = make_float4(nx, ny, nz, h);
    C.Pn[p] = nrm;
    C.Ps[p] = src;
    C.Pc[p] = (uint8_t)code;
    uint8_t rem[CL::MT];
    uint32_t rtri[CL::MT];
    int r = 0;
    for (int w = 0; w < CL::MT / 32; w++) {
        unsigned m = bm[w];
        while (m) {
            const int t = w * 32 + __ffs(m) - 1;
            m &= m - 1;
            if (r == CL::MT) return TF_CAP_CUT;
            rtri[r] = C.Tr[t];
            rem[r++] = (uint8_t)t;
        }
    }
    uint8_t bx[CL::MT + 2], by[CL::MT + 2];
    int nb = 0;
    for (int k = 0; k < r; k++) {
        uint32_t id[3];
        tri_ids(rtri[k], id[0], id[1], id[2]);
        for (int e = 0; e < 3; e++) {
            const uint32_t x = id[e], y = id[e == 2 ? 0 : e + 1];
            bool inner = false;
            for (int k2 = 0; k2 < r && !inner; k2++) {
                if (k2 == k) continue;
                uint32_t a, b, c;
                tri_ids(rtri[k2], a, b, c);
                inner = (a == y && b == x) || (b == y && c == x) || (c == y && a == x);
            }
            if (!inner) {
                if (nb == CL::MT + 2) return TF_CAP_CUT;
                bx[nb] = (uint8_t)x;
                by[nb] = (uint8_t)y;
                nb++;
            }
        }
    }
    if (nb < 3) return TF_CAP_CUT;
    if (C.nT - r + nb > CL::MT) return TF_CAP;
    for (int i = 0; i < nb; i++) {
        const int slot = i < r ? (int)rem[i] : C.nT + (i - r);
        const uint32_t t = (uint32_t)bx[i] | ((uint32_t)by[i] << 8) | (p << 16);
        float4 v;
        if (!vertex_of(C, bx[i], by[i], p, v)) return TF_ILL;
        C.Tr[slot] = t;
        C.V[slot] = v;
    }
    if (nb >= r) {
        C.nT += nb - r;
    } else {
        // holes rem[nb..r) (ascending): move the last live triangles into those below the new count
        const int n2 = C.nT - (r - nb);
        unsigned hm[CL::MT / 32];
        for (int w = 0; w < CL::MT / 32; w++) hm[w] = 0u;
        for (int i = nb; i < r; i++) hm[rem[i] >> 5] |= 1u << (rem[i] & 31);
        int top = C.nT - 1;
        for (int i = nb; i < r; i++) {
            const int hole = rem[i];
            if (hole >= n2) break;
            while (top >= n2 && ((hm[top >> 5] >> (top & 31)) & 1u)) top--;
            C.Tr[hole] = C.Tr[top];
            C.V[hole] = C.V[top];
            top--;
        }
        C.nT = n2;
    }
    return 0;
}

// n.v - h against the error bound for every vertex: beyond -> bm, undecided -> um
template <class CL>
__device__ __forceinline__ void test_plane(const CL& C, float nx, float ny, float nz, float h, float nrm, float hb,
                                           unsigned* bm, unsigned* um) {
    for (int w = 0; w < CL::MT / 32; w++) bm[w] = um[w] = 0u;
    for (int t = 0; t < C.nT; t++) {
        const float4 v = C.V[t];
        const float s = __fmaf_rn(nx, v.x, __fmaf_rn(ny, v.y, __fmaf_rn(nz, v.z, -h)));
        const float bound = __fmaf_rn(nrm, v.w, hb);
        const unsigned bit = 1u << (t & 31);
        if (s > bound) bm[t >> 5] |= bit;
        else if (!(s < -bound)) um[t >> 5] |= bit;
    }
}

// gap between [lo, hi] and [blo, bhi] along one axis (minimum image when periodic)
__device__ __forceinline__ float iv_gap(float lo, float hi, float blo, float bhi, float L, int periodic) {
    float d = fmaxf(fmaxf(lo - bhi, blo - hi), 0.f);
    if (periodic) {
        d = fminf(d, fmaxf(fmaxf(lo + L - bhi, blo - hi - L), 0.f));
        d = fminf(d, fmaxf(fmaxf(lo - L - bhi, blo - hi + L), 0.f));
    }
    return d;
}

// Sort (key, val) across the warp by decreasing key (bitonic network over the lanes).
__device__ __forceinline__ void warp_sort_desc(float& key, uint32_t& val) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            const float ok = __shfl_xor_sync(0xffffffffu, key, jj);
            const uint32_t ov = __shfl_xor_sync(0xffffffffu, val, jj);
            const bool down = ((lane & k) == 0);     // this half ends decreasing
            const bool lower = (lane & jj) == 0;
            const bool take_big = (lower == down);
            const bool other_bigger = ok > key || (ok == key && ov < val);
            if (take_big == other_bigger) { key = ok; val = ov; }
        }
}

// Resume the warp's walk of the tree: points (sorted index in [ilo, ihi)) whose gap to the bucket box has
// g2lo <= gap^2 < g2hi are appended to the chunk until fewer than 32 slots are free or the stack is empty.
__device__ int walk(TSmem& S, int& sp, int cnt, const float4* spos4, const void* spos, bool f64, const Tree& t,
                    const Geometry& g, const float* blo, const float* bhi, float g2lo, float g2hi, int64_t ilo,
                    int64_t ihi, bool& stack_ovf) {
    const unsigned lane = lane_id(), lt = lanemask_lt();
    while (sp > 0 && cnt <= TCH - 32) {
        const uint32_t ent = S.stack[sp - 1];
        sp--;
        __syncwarp();
        const int lvl = (int)(ent >> 27);
        const int64_t node = ent & ((1u << 27) - 1);
        if (lvl == 1) {
            const int64_t j = node * 32 + lane;
            bool hit = false;
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j >= ilo && j < ihi) {
                if (f64) {
                    const dpt4 d = ((const dpt4*)spos)[j];
                    q = make_float4((float)d.x, (float)d.y, (float)d.z, 0.f);
                } else {
                    q = spos4[j];
                }
                const float dx = axis_gap(q.x, blo[0], bhi[0], g.Lf[0], g.periodic);
                const float dy = axis_gap(q.y, blo[1], bhi[1], g.Lf[1], g.periodic);
                const float dz = axis_gap(q.z, blo[2], bhi[2], g.Lf[2], g.periodic);
                const float g2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, dx * dx));
                hit = g2 >= g2lo && g2 < g2hi;
            }
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                q.w = __uint_as_float((uint32_t)j);
                S.chunk[cnt + __popc(m & lt)] = q;
            }
            cnt += __popc(m);
        } else {
            const int cl = lvl - 1;
            const int64_t c = node * 32 + lane;
            const int64_t span = (int64_t)1 << (5 * cl);
            bool hit = false;
            float gap2 = -1.f;
            if (c < t.count[cl] && c * span < ihi && (c + 1) * span > ilo) {
                const float4 lo = t.lo[t.off[cl] + c], hi = t.hi[t.off[cl] + c];
                const float dx = iv_gap(lo.x, hi.x, blo[0], bhi[0], g.Lf[0], g.periodic);
                const float dy = iv_gap(lo.y, hi.y, blo[1], bhi[1], g.Lf[1], g.periodic);
                const float dz = iv_gap(lo.z, hi.z, blo[2], bhi[2], g.Lf[2], g.periodic);
                gap2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, dx * dx));
                hit = gap2 < g2hi * 1.0001f + 1e-30f;
            }
            const int nh = __popc(__ballot_sync(0xffffffffu, hit));
            if (sp + nh > TSTK) {
                stack_ovf = true;
                return cnt;
            }
            // nearest child on top of the stack: the points arrive roughly by distance from the bucket
            float key = hit ? gap2 : -1.f;
            uint32_t val = hit ? (((uint32_t)cl << 27) | (uint32_t)c) : 0xffffffffu;
            warp_sort_desc(key, val);
            if ((int)lane < nh) S.stack[sp + lane] = val;
            sp += nh;
            __syncwarp();
        }
    }
    return cnt;
}

// bitonic sort of the chunk keys [0, n) padded to a power of two
__device__ void sort_keys(TSmem& S, int n) {
    const unsigned lane = lane_id();
    int m = 32;
    while (m < n) m <<= 1;
    for (int k = n + (int)lane; k < m; k += 32) S.key[k] = 0xffffffffu;
    __syncwarp();
    for (int k = 2; k <= m; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int i = (int)lane; i < m; i += 32) {
                const int ixj = i ^ jj;
                if (ixj > i) {
                    const uint32_t a = S.key[i], b = S.key[ixj];
                    const bool asc = (i & k) == 0;
                    if ((a > b) == asc) { S.key[i] = b; S.key[ixj] = a; }
                }
            }
            __syncwarp();
        }
    }
}

struct TCount {
    unsigned long long tested, cut, fp64, passes, collected;
};

// Filter the chunk for one lane's cell, then test the survivors and cut (lanes in step).  The filter works on
// a cheap displacement (one rounding per component, periodic shift by rint) and keeps a point unless it is
// farther than 2R, or its plane misses the cell's box, by more than the margin `slack` covers.  Survivors are
// taken in six distance classes (near2 x 1, 2, 4, 8, 16, more), nearest first; each is re-checked against the
// shrunken cell with the exact displacement before its test.  Returns 0 or a failure code for the lane.
template <typename P>
__device__ int clip_chunk(const TSmem& S, int cnt, TCell& C, const P* spos, const Geometry& g, const P& pi,
                          uint32_t self, int64_t slo, int64_t shi, bool active, float near2, float slack,
                          TCount& tc) {
    const float u = Prec<float>::u();
    uint8_t pend[TCH];
    int np = 0;
    if (active) {
        uint16_t lv[TCH];
        int nl[6] = {0, 0, 0, 0, 0, 0};
        const float qx = (float)pi.x, qy = (float)pi.y, qz = (float)pi.z;
        const float iLx = 1.f / g.Lf[0], iLy = 1.f / g.Lf[1], iLz = 1.f / g.Lf[2];
        const float bext = fmaxf(fmaxf(fmaxf(-C.bmin[0], C.bmax[0]), fmaxf(-C.bmin[1], C.bmax[1])),
                                 fmaxf(-C.bmin[2], C.bmax[2]));
        const float rad = 2.f * sqrtf(C.R2);
        const float rskip = rad * (1.f + 1e-5f) + 4.f * slack;
        const float rskip2 = rskip * rskip;
        const float stol = 1e-5f * (4.f * bext * rad + rad * rad) + 8.f * slack * (bext + rad) + 1e-30f;
        for (int k = 0; k < cnt; k++) {
            const uint32_t e = S.key[k] & 255u;
            const float4 q = S.chunk[e];
            const uint32_t j = __float_as_uint(q.w);
            float dx = q.x - qx, dy = q.y - qy, dz = q.z - qz;
            if (g.periodic) {
                dx -= g.Lf[0] * rintf(dx * iLx);
                dy -= g.Lf[1] * rintf(dy * iLy);
                dz -= g.Lf[2] * rintf(dz * iLz);
            }
            const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, dx * dx));
            if (d2 > rskip2) continue;
            if (j == self || (int64_t)j < slo || (int64_t)j >= shi) continue;
            const float sg = supp_g(dx, C.bmin[0], C.bmax[0]) + supp_g(dy, C.bmin[1], C.bmax[1]) +
                             supp_g(dz, C.bmin[2], C.bmax[2]);
            if (sg < -stol) continue;
            const int l = (d2 >= near2) + (d2 >= 2.f * near2) + (d2 >= 4.f * near2) + (d2 >= 8.f * near2) +
                          (d2 >= 16.f * near2);
            lv[np++] = (uint16_t)(e | (l << 8));
            nl[l]++;
        }
        int o[6];
        o[0] = 0;
#pragma unroll
        for (int l = 1; l < 6; l++) o[l] = o[l - 1] + nl[l - 1];
        for (int k = 0; k < np; k++) {
            const int l = lv[k] >> 8;
            pend[o[l]++] = (uint8_t)(lv[k] & 255u);
        }
    }
    int kmax = np;
#pragma unroll
    for (int o = 16; o; o >>= 1) kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    int fail = 0;
    for (int k = 0; k < kmax; k++) {
        if (!active || fail || k >= np) continue;
        const float4 q = S.chunk[pend[k]];
        const uint32_t j = __float_as_uint(q.w);
        float dx, dy, dz;
        int code;
        DispF<P, float>::get(spos[j], pi, g, dx, dy, dz, code);
        const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, dx * dx));
        if (d2 == 0.f) { fail = TF_DUP; continue; }
        if (d2 * (1.f - 8.f * u) > 4.f * C.R2) continue;
        {
            // the cell's box has shrunk since the filter
            const float bext = fmaxf(fmaxf(fmaxf(-C.bmin[0], C.bmax[0]), fmaxf(-C.bmin[1], C.bmax[1])),
                                     fmaxf(-C.bmin[2], C.bmax[2]));
            const float rad2 = 4.f * C.R2;
            const float stol = 1e-5f * (4.f * bext * sqrtf(rad2) + rad2) + 1e-30f;
            const float sg = supp_g(dx, C.bmin[0], C.bmax[0]) + supp_g(dy, C.bmin[1], C.bmax[1]) +
                             supp_g(dz, C.bmin[2], C.bmax[2]);
            if (sg < -stol) continue;
        }
        const float h = 0.5f * d2;
        const float nrm = sqrtf(d2);
        const float hb = 16.f * u * h;
        unsigned bm[TT / 32], um[TT / 32];
        test_plane(C, dx, dy, dz, h, nrm, hb, bm, um);
        tc.tested++;
        // undecided vertices: FP64 from the inputs
        for (int w = 0; w < TT / 32 && !fail; w++) {
            unsigned m = um[w];
            while (m) {
                const int t = w * 32 + __ffs(m) - 1;
                m &= m - 1;
                uint32_t a, b, c;
                tri_ids(C.Tr[t], a, b, c);
                const PRef ra = {C.Ps[a], C.Pc[a]}, rb = {C.Ps[b], C.Pc[b]}, rc = {C.Ps[c], C.Pc[c]};
                const PRef rj = {j, (uint8_t)code};
                const int sd = side64<P>(spos, g, self, ra, rb, rc, rj);
                tc.fp64++;
                if (sd == 0) { fail = TF_UNDECIDED; break; }
                if (sd > 0) bm[w] |= 1u << (t & 31);
            }
        }
        if (fail) continue;
        if ((bm[0] | bm[1]) == 0u) continue;
        fail = cut_cell(C, bm, dx, dy, dz, h, nrm, j, code);
        if (fail) continue;
        tc.cut++;
        bound_cell(C);
    }
    return fail;
}

// Planes that carry a facet (appear in a triangle) and the number of facet records (planes between particles);
// -1 when the cell touches an artificial wall (its start box was too small).
__device__ int count_faces(const TCell& C, uint64_t* present) {
    uint64_t pm = 0ull;
    for (int t = 0; t < C.nT; t++) {
        uint32_t a, b, c;
        tri_ids(C.Tr[t], a, b, c);
        pm |= (1ull << a) | (1ull << b) | (1ull << c);
    }
    int nf = 0;
    for (int p = 0; p < C.nP; p++) {
        if (!((pm >> p) & 1ull)) continue;
        if (C.Pc[p] >= CODE_ART) return -1;
        if (p >= 6 && C.Pc[p] < 27) nf++;
    }
    *present = pm;
    return nf;
}

// Facets of a finished cell: per plane, its triangles walked around the plane (the successor of (p, q, r) is the
// triangle (p, r, s)) and fanned from the first vertex, with the formulas of the warp kernel's emission; facet
// records go to out[] in plane order.  Returns false if a facet cannot be walked or the volume is not positive.
__device__ bool emit_faces(const TCell& C, uint64_t present, Face* out, float& vol, float& mzx, float& mzy,
                           float& mzz, float& m2) {
    KSum<float> kvol;
    kvol.zero();
    mzx = mzy = mzz = m2 = 0.f;
    int w = 0;
    for (int p = 0; p < C.nP; p++) {
        if (!((present >> p) & 1ull)) continue;
        uint8_t ft[32], fq[32], fr[32];
        int m = 0;
        for (int t = 0; t < C.nT; t++) {
            uint32_t a, b, c;
            tri_ids(C.Tr[t], a, b, c);
            uint32_t q, r;
            if (a == (uint32_t)p) { q = b; r = c; }
            else if (b == (uint32_t)p) { q = c; r = a; }
            else if (c == (uint32_t)p) { q = a; r = b; }
            else continue;
            if (m == 32) return false;
            ft[m] = (uint8_t)t; fq[m] = (uint8_t)q; fr[m] = (uint8_t)r;
            m++;
        }
        if (m < 3) return false;
        const float4 v0 = C.V[ft[0]];
        const float4 pl = C.Pl[p];
        const float inrm = 1.f / C.Pn[p];
        const float nhx = pl.x * inrm, nhy = pl.y * inrm, nhz = pl.z * inrm;
        KSum<float> kA;
        kA.zero();
        float csx = 0.f, csy = 0.f, csz = 0.f, sm2 = 0.f;
        int cur = -1, steps = 1;
        for (int k = 1; k < m; k++)
            if (fq[k] == fr[0]) { cur = k; break; }
        for (int guard = 0; guard < m && cur > 0; guard++) {
            int nxt = -1;
            for (int k = 0; k < m; k++)
                if (fq[k] == fr[cur]) { nxt = k; break; }
            steps++;
            if (nxt <= 0) break;
            const float4 v1 = C.V[ft[cur]], v2 = C.V[ft[nxt]];
            const float e1x = v1.x - v0.x, e1y = v1.y - v0.y, e1z = v1.z - v0.z;
            const float e2x = v2.x - v0.x, e2y = v2.y - v0.y, e2z = v2.z - v0.z;
            const float crx = __fmaf_rn(e1y, e2z, -e1z * e2y), cry = __fmaf_rn(e1z, e2x, -e1x * e2z),
                        crz = __fmaf_rn(e1x, e2y, -e1y * e2x);
            const float at = 0.5f * __fmaf_rn(crx, nhx, __fmaf_rn(cry, nhy, crz * nhz));
            kA.add(at);
            const float third = (float)(1.0 / 3.0);
            csx = __fmaf_rn(at * third, v0.x + v1.x + v2.x, csx);
            csy = __fmaf_rn(at * third, v0.y + v1.y + v2.y, csy);
            csz = __fmaf_rn(at * third, v0.z + v1.z + v2.z, csz);
            float s2 = __fmaf_rn(v0.x, v0.x + v1.x + v2.x, __fmaf_rn(v0.y, v0.y + v1.y + v2.y, v0.z * (v0.z + v1.z + v2.z)));
            s2 = __fmaf_rn(v1.x, v1.x + v2.x, __fmaf_rn(v1.y, v1.y + v2.y, __fmaf_rn(v1.z, v1.z + v2.z, s2)));
            s2 = __fmaf_rn(v2.x, v2.x, __fmaf_rn(v2.y, v2.y, __fmaf_rn(v2.z, v2.z, s2)));
            sm2 = __fmaf_rn(at, s2, sm2);
            cur = nxt;
        }
        if (steps != m) return false;  // the walk did not close over all of the plane's triangles
        const float A_ = kA.value();
        const float dist = pl.w * inrm;
        kvol.add(dist * A_ * (float)(1.0 / 3.0));
        mzx += dist * csx * 0.25f;
        mzy += dist * csy * 0.25f;
        mzz += dist * csz * 0.25f;
        m2 += dist * sm2 * (float)(1.0 / 30.0);
        if (p >= 6 && C.Pc[p] < 27) {
            Face f;
            f.dx = pl.x; f.dy = pl.y; f.dz = pl.z;
            f.area = A_;
            if (A_ != 0.f) { f.cx = csx / A_; f.cy = csy / A_; f.cz = csz / A_; }
            else { f.cx = f.cy = f.cz = 0.f; }
            f.nbr = C.Ps[p];
            out[w++] = f;
        }
    }
    vol = kvol.value();
    return vol > 0.f;
}

template <typename P>
__global__ void __launch_bounds__(TWARPS * 32) k_clip_thread(ClipArgs A) {
    __shared__ TSmem smem[TWARPS];
    TSmem& S = smem[threadIdx.x >> 5];
    const unsigned lane = lane_id(), lt = lanemask_lt();
    if (*((volatile unsigned*)&A.st->invalid_input)) return;
    const P* spos = (const P*)A.spos;
    const bool f64 = sizeof(P) != 16;
    const float u = Prec<float>::u();
    const int64_t nbuckets = (A.N + 31) / 32;
    TCount tc = {0ull, 0ull, 0ull, 0ull, 0ull};
    TCell C;
    for (;;) {
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(&A.st->work_next_bucket, 1ull);
        b = __shfl_sync(0xffffffffu, b, 0);
        if ((int64_t)b >= nbuckets) break;
        const int64_t self64 = (int64_t)b * 32 + lane;
        bool alive = self64 < A.N;
        const uint32_t self = alive ? (uint32_t)self64 : 0u;
        Geometry g = A.geo;
        int64_t slo = 0, shi = A.N;
        int mode = A.tpc_mode;
        if (A.sset && alive) {
            const uint32_t s = A.sset[self];
            g = A.sgeo[s];
            slo = A.soff[s];
            shi = A.soff[s + 1];
            if (A.set_cfg) mode = (A.set_cfg[s] >> 16) & 3;
        }
        // this kernel's cells (mode 1); those of the warp kernel (mode 0) are handed over as they are, and those
        // of the lane-group kernels (modes 2, 3) are left to them
        if (mode >= 2) alive = false;
        const bool mine = alive && mode == 1;
        if (!__any_sync(0xffffffffu, mine)) {
            // a bucket of warp-kernel sets: hand its cells over as they are
            const unsigned hm = __ballot_sync(0xffffffffu, alive);
            unsigned slot0 = 0;
            if (lane == 0) slot0 = atomicAdd(&A.st->n_warp_cells, (unsigned)__popc(hm));
            slot0 = __shfl_sync(0xffffffffu, slot0, 0);
            if (alive) A.warp_list[slot0 + __popc(hm & lt)] = self;
            continue;
        }
        const P pi = spos[self];
        const float qx = (float)pi.x, qy = (float)pi.y, qz = (float)pi.z;
        // the bucket's box (over its live cells) and index range
        float blo[3] = {alive ? qx : INFINITY, alive ? qy : INFINITY, alive ? qz : INFINITY};
        float bhi[3] = {alive ? qx : -INFINITY, alive ? qy : -INFINITY, alive ? qz : -INFINITY};
        int64_t ilo = alive ? slo : INT64_MAX, ihi = alive ? shi : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
#pragma unroll
            for (int a = 0; a < 3; a++) {
                blo[a] = fminf(blo[a], __shfl_xor_sync(0xffffffffu, blo[a], o));
                bhi[a] = fmaxf(bhi[a], __shfl_xor_sync(0xffffffffu, bhi[a], o));
            }
            ilo = min(ilo, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)ilo, o));
            ihi = max(ihi, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)ihi, o));
        }
        // first radius: 1.6 x the median over the lanes of the distance to the 4th nearest bucket mate (about the
        // reach of a cell's facets; later passes widen it to what the unfinished cells need)
        float d4, near2;
        {
            float k0 = INFINITY, k1 = INFINITY, k2 = INFINITY, k3 = INFINITY;
            for (int l = 0; l < 32; l++) {
                const float ox = __shfl_sync(0xffffffffu, qx, l), oy = __shfl_sync(0xffffffffu, qy, l),
                            oz = __shfl_sync(0xffffffffu, qz, l);
                const int oi = __shfl_sync(0xffffffffu, (int)alive, l);
                const int64_t ol = (int64_t)b * 32 + l;
                if (!oi || l == (int)lane || ol < slo || ol >= shi) continue;
                float dx = fabsf(ox - qx), dy = fabsf(oy - qy), dz = fabsf(oz - qz);
                if (g.periodic) {
                    dx = fminf(dx, g.Lf[0] - dx); dy = fminf(dy, g.Lf[1] - dy); dz = fminf(dz, g.Lf[2] - dz);
                }
                float d2 = dx * dx + dy * dy + dz * dz;
                if (d2 < k3) {
                    if (d2 < k2) { k3 = k2; if (d2 < k1) { k2 = k1; if (d2 < k0) { k1 = k0; k0 = d2; } else k1 = d2; } else k2 = d2; }
                    else k3 = d2;
                }
            }
            d4 = alive ? k3 : INFINITY;
            near2 = k3;
            // median over the lanes (infinite values sort last)
            for (int k = 2; k <= 32; k <<= 1)
                for (int jj = k >> 1; jj > 0; jj >>= 1) {
                    const float o = __shfl_xor_sync(0xffffffffu, d4, jj);
                    const bool up = ((lane & k) == 0), lower = (lane & jj) == 0;
                    const float mn = fminf(d4, o), mx = fmaxf(d4, o);
                    d4 = (lower == up) ? mn : mx;
                }
            const int n_alive = __popc(__ballot_sync(0xffffffffu, alive));
            d4 = __shfl_sync(0xffffffffu, d4, n_alive / 2);
        }
        const double lmin = fmin(g.L[0], fmin(g.L[1], g.L[2]));
        float rho;
        if (d4 < INFINITY && d4 > 0.f) rho = 1.6f * sqrtf(d4);
        else rho = (float)(2.0 * cbrt(g.L[0] * g.L[1] * g.L[2] / (double)max((int64_t)1, shi - slo)));
        rho = __shfl_sync(0xffffffffu, rho, 0);  // lanes of one bucket share the radius
        const float rho_cap = g.periodic ? (float)(0.24 * lmin) : INFINITY;
        if (rho > rho_cap) rho = rho_cap;
        if (!(near2 < INFINITY) || near2 <= 0.f) near2 = rho * rho * (1.f / 16.f);
        // rounding of the gaps (coordinates, box ends and periodic shifts carry a few ulps of the box scale);
        // the same for every lane of the bucket
        float slack = 16.f * u * fmaxf(fmaxf(fmaxf(fabsf(g.hif[0]), fabsf(g.lof[0])), fmaxf(fabsf(g.hif[1]), fabsf(g.lof[1]))),
                                        fmaxf(fmaxf(fabsf(g.hif[2]), fabsf(g.lof[2])), fmaxf(g.Lf[0], fmaxf(g.Lf[1], g.Lf[2])))) + 1e-30f;
        slack = warp_max<float>(alive ? slack : 0.f);
        int fail = alive && !mine ? TF_SKIP : 0;
        // start box on the scale of the lane's own neighbourhood (a box that proves too small sends the cell to
        // the warp kernel)
        const float Bown = fminf(4.f * rho, 3.f * sqrtf(near2));
        if (alive && mine) fail = init_cell<P>(C, g, pi, self, Bown);
        const unsigned long long f64_before = tc.fp64;
        bool done = !alive;
        float g2prev = -1.f;
        int streamed = 0;
        for (int pass = 0; pass < TPASSES; pass++) {
            const bool want = alive && !done && !fail;
            if (!__any_sync(0xffffffffu, want)) break;
            if (lane == 0) tc.passes++;
            const float gr = rho * (1.f + 4.f * u) + slack;
            const float g2hi = gr * gr * (1.f + 4.f * u);
            // top level into the stack
            int sp = 0;
            {
                const Tree& t = A.tree;
                const int top = t.levels;
                const int64_t span = (int64_t)1 << (5 * top);
                bool hit = false;
                if ((int64_t)lane < t.count[top] && lane * span < ihi && (lane + 1) * span > ilo) {
                    const float4 lo = t.lo[t.off[top] + lane], hi = t.hi[t.off[top] + lane];
                    const float dx = iv_gap(lo.x, hi.x, blo[0], bhi[0], g.Lf[0], g.periodic);
                    const float dy = iv_gap(lo.y, hi.y, blo[1], bhi[1], g.Lf[1], g.periodic);
                    const float dz = iv_gap(lo.z, hi.z, blo[2], bhi[2], g.Lf[2], g.periodic);
                    hit = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, dx * dx)) < g2hi * 1.0001f + 1e-30f;
                }
                float gap2 = -1.f;
                if (hit) {
                    const float4 lo = t.lo[t.off[top] + lane], hi = t.hi[t.off[top] + lane];
                    const float dx = iv_gap(lo.x, hi.x, blo[0], bhi[0], g.Lf[0], g.periodic);
                    const float dy = iv_gap(lo.y, hi.y, blo[1], bhi[1], g.Lf[1], g.periodic);
                    const float dz = iv_gap(lo.z, hi.z, blo[2], bhi[2], g.Lf[2], g.periodic);
                    gap2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, dx * dx));
                }
                const int nh = __popc(__ballot_sync(0xffffffffu, hit));
                uint32_t val = hit ? (((uint32_t)top << 27) | lane) : 0xffffffffu;
                warp_sort_desc(gap2, val);
                if ((int)lane < nh) S.stack[lane] = val;
                sp = nh;
                __syncwarp();
            }
            bool ovf = false;
            while (sp > 0) {
                const int cnt = walk(S, sp, 0, (const float4*)A.spos, A.spos, f64, A.tree, g, blo, bhi, g2prev, g2hi,
                                     ilo, ihi, ovf);
                streamed += cnt;
                if (lane == 0) tc.collected += cnt;
                if (ovf || streamed > TMAXPTS) { ovf = true; break; }
                if (cnt == 0) continue;
                // nearest first (to the bucket's box centre)
                {
                    const float cx = 0.5f * (blo[0] + bhi[0]), cy = 0.5f * (blo[1] + bhi[1]), cz = 0.5f * (blo[2] + bhi[2]);
                    for (int k = (int)lane; k < cnt; k += 32) {
                        const float4 q = S.chunk[k];
                        float dx = fabsf(q.x - cx), dy = fabsf(q.y - cy), dz = fabsf(q.z - cz);
                        if (g.periodic) {
                            dx = fminf(dx, g.Lf[0] - dx); dy = fminf(dy, g.Lf[1] - dy); dz = fminf(dz, g.Lf[2] - dz);
                        }
                        const float d2 = dx * dx + dy * dy + dz * dz;
                        S.key[k] = (__float_as_uint(d2) & ~255u) | (uint32_t)k;
                    }
                    __syncwarp();
                    sort_keys(S, cnt);
                }
                const bool act = alive && !done && !fail;
                const int f = clip_chunk<P>(S, cnt, C, spos, g, pi, self, slo, shi, act, near2, slack, tc);
                if (act && f) fail = f;
                __syncwarp();
            }
            if (ovf) {
                if (alive && !done && !fail) fail = TF_RADIUS;
                break;
            }
            g2prev = g2hi;
            // certified: every point within rho of the site has been examined
            if (alive && !done && !fail && 4.f * C.R2 <= rho * rho * (1.f - 8.f * u)) done = true;
            // next radius: what the unfinished cells need, between 1.25 and 2 times the current one
            float need = (alive && !done && !fail) ? 2.f * sqrtf(C.R2) * 1.001f : 0.f;
            need = warp_max<float>(need);
            if (need == 0.f) break;
            float nxt = fminf(fmaxf(need, 1.25f * rho), 2.f * rho);
            if (rho >= rho_cap) break;
            rho = fminf(nxt, rho_cap);
        }
        if (alive && !done && !fail) fail = TF_RADIUS;
        // ---------------- emission
        int nf = 0;
        uint64_t present = 0ull;
        if (alive && !fail) {
            nf = count_faces(C, &present);
            if (nf < 0) fail = TF_WALL;
        }
        if (!(alive && !fail)) nf = 0;
        // reserve the warp's facet records at once
        int incl = nf;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if ((int)lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long base = 0ull;
        if (lane == 0 && total > 0) base = atomicAdd(&A.st->face_next, (unsigned long long)total);
        base = __shfl_sync(0xffffffffu, base, 0);
        const bool pool_ok = base + (unsigned long long)total <= A.face_cap;
        if (!pool_ok) {
            if (lane == 0) atomicCAS(&A.st->error, 0, RC_POOL);
            if (alive && !fail) fail = TF_CAP;
        } else if (alive && !fail) {
            const uint32_t start = (uint32_t)(base + (unsigned long long)(incl - nf));
            float vol, mzx, mzy, mzz, m2;
            if (!emit_faces(C, present, A.faces + start, vol, mzx, mzy, mzz, m2)) {
                fail = TF_CAP_PLANES;  // its records are left unused; the warp kernel writes new ones
            } else {
                CellOut co;
                co.vol = (double)vol;
                co.zx = mzx / vol;
                co.zy = mzy / vol;
                co.zz = mzz / vol;
                co.mom2 = m2;
                A.cell[self] = co;
                A.face_start[self] = start;
                A.face_count[self] = (uint16_t)nf;
                A.cstat[self] = (uint8_t)(CS_DONE | (tc.fp64 != f64_before ? CS_FP64 : 0));
                if (A.rad) A.rad[self] = sqrtf(C.R2) * (1.f + 1e-6f);
                atomicMax(&A.st->max_faces, (unsigned)nf);
            }
        }
        const bool emit = alive && !fail;
        // hand the unfinished cells to the warp kernel
        const bool hand = alive && !emit;
        if (hand && fail != TF_SKIP) atomicAdd(&A.st->n_tfail[fail > 0 && fail < 8 ? fail : 0], 1ull);  // 0: plane capacity
        const unsigned hm = __ballot_sync(0xffffffffu, hand);
        if (hm) {
            unsigned slot0 = 0;
            if (lane == 0) slot0 = atomicAdd(&A.st->n_warp_cells, (unsigned)__popc(hm));
            slot0 = __shfl_sync(0xffffffffu, slot0, 0);
            if (hand) A.warp_list[slot0 + __popc(hm & lt)] = self;
        }
        // facet records of the cells finished here
        int nfe = emit ? nf : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) nfe += __shfl_xor_sync(0xffffffffu, nfe, o);
        if (lane == 0 && nfe > 0) atomicAdd(&A.st->n_faces, (unsigned long long)nfe);
    }
    // counters
    unsigned long long v[5] = {tc.tested, tc.cut, tc.fp64, tc.passes, tc.collected};
#pragma unroll
    for (int k = 0; k < 5; k++)
#pragma unroll
        for (int o = 16; o; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0) {
        atomicAdd(&A.st->n_tested, v[0]);
        atomicAdd(&A.st->n_cut, v[1]);
        atomicAdd(&A.st->n_fp64, v[2]);
        atomicAdd(&A.st->n_t_tested, v[0]);
        atomicAdd(&A.st->n_t_cut, v[1]);
        atomicAdd(&A.st->n_t_fp64, v[2]);
        atomicAdd(&A.st->n_t_collected, v[4]);
        atomicAdd(&A.st->n_bucket_passes, v[3]);
        atomicAdd(&A.st->n_collected, v[4]);
    }
}

// ------------------------------------------------------------------ G lanes per cell (G = 4 or 8)
// The lane-group kernels: G lanes share one cell and a warp holds 32/G cells (consecutive particles in Morton
// order, a part of one tree bucket).  The warp streams the points near its cells through shared memory as the
// thread-per-cell kernel does.  Each cell lives in shared memory: its G lanes filter a chunk's points in turn,
// split every candidate's side tests (and their FP64 re-tests) by vertex, and combine the results with group
// reductions; the group's first lane applies the cuts and keeps the cell's bounds.  The predicates, cuts,
// certificate and emitted records are those of the thread-per-cell kernel, and so are the failure codes of the
// cells handed to the warp kernel.
constexpr int GWARPS = 2;  // warps per block

struct GCell {
    TCell C;
    uint8_t pend[TCH];  // the chunk's points that survive the filter, in chunk order
};

// lanes of the G-lane group holding this lane
template <int G>
__device__ __forceinline__ unsigned group_mask() {
    return ((1u << G) - 1u) << (lane_id() & ~(unsigned)(G - 1));
}

// Filter the chunk for the group's cell (lanes take points in turn, survivors kept in chunk order), then test the
// survivors one after the other: side tests split by vertex, the cut by the group's first lane.  active, the
// result and every branch are uniform over the group.  Returns 0 or a failure code.
template <typename P, int G>
__device__ int clip_chunk_group(const TSmem& S, int cnt, GCell& GC, const P* spos, const Geometry& g, const P& pi,
                                uint32_t self, int64_t slo, int64_t shi, bool active, float slack, TCount& tc) {
    TCell& C = GC.C;
    const float u = Prec<float>::u();
    const unsigned gmask = group_mask<G>();
    const unsigned glt = gmask & lanemask_lt();
    const int r = (int)(lane_id() & (unsigned)(G - 1));
    const int leader = __ffs(gmask) - 1;
    if (!active) return 0;
    int np = 0;
    {
        const float qx = (float)pi.x, qy = (float)pi.y, qz = (float)pi.z;
        const float iLx = 1.f / g.Lf[0], iLy = 1.f / g.Lf[1], iLz = 1.f / g.Lf[2];
        const float bext = fmaxf(fmaxf(fmaxf(-C.bmin[0], C.bmax[0]), fmaxf(-C.bmin[1], C.bmax[1])),
                                 fmaxf(-C.bmin[2], C.bmax[2]));
        const float rad = 2.f * sqrtf(C.R2);
        const float rskip = rad * (1.f + 1e-5f) + 4.f * slack;
        const float rskip2 = rskip * rskip;
        const float stol = 1e-5f * (4.f * bext * rad + rad * rad) + 8.f * slack * (bext + rad) + 1e-30f;
        for (int k0 = 0; k0 < cnt; k0 += G) {
            const int k = k0 + r;
            bool keep = false;
            uint32_t e = 0u;
            if (k < cnt) {
                e = S.key[k] & 255u;
                const float4 q = S.chunk[e];
                const uint32_t j = __float_as_uint(q.w);
                float dx = q.x - qx, dy = q.y - qy, dz = q.z - qz;
                if (g.periodic) {
                    dx -= g.Lf[0] * rintf(dx * iLx);
                    dy -= g.Lf[1] * rintf(dy * iLy);
                    dz -= g.Lf[2] * rintf(dz * iLz);
                }
                const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, dx * dx));
                keep = d2 <= rskip2 && j != self && (int64_t)j >= slo && (int64_t)j < shi;
                if (keep) {
                    const float sg = supp_g(dx, C.bmin[0], C.bmax[0]) + supp_g(dy, C.bmin[1], C.bmax[1]) +
                                     supp_g(dz, C.bmin[2], C.bmax[2]);
                    keep = !(sg < -stol);
                }
            }
            const unsigned km = __ballot_sync(gmask, keep);
            if (keep) GC.pend[np + __popc(km & glt)] = (uint8_t)e;
            np += __popc(km);
        }
        __syncwarp(gmask);
    }
    for (int k = 0; k < np; k++) {
        const float4 q = S.chunk[GC.pend[k]];
        const uint32_t j = __float_as_uint(q.w);
        float dx, dy, dz;
        int code;
        DispF<P, float>::get(spos[j], pi, g, dx, dy, dz, code);
        const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, dx * dx));
        if (d2 == 0.f) return TF_DUP;
        if (d2 * (1.f - 8.f * u) > 4.f * C.R2) continue;
        {
            // the cell's box has shrunk since the filter
            const float bext = fmaxf(fmaxf(fmaxf(-C.bmin[0], C.bmax[0]), fmaxf(-C.bmin[1], C.bmax[1])),
                                     fmaxf(-C.bmin[2], C.bmax[2]));
            const float rad2 = 4.f * C.R2;
            const float stol = 1e-5f * (4.f * bext * sqrtf(rad2) + rad2) + 1e-30f;
            const float sg = supp_g(dx, C.bmin[0], C.bmax[0]) + supp_g(dy, C.bmin[1], C.bmax[1]) +
                             supp_g(dz, C.bmin[2], C.bmax[2]);
            if (sg < -stol) continue;
        }
        const float h = 0.5f * d2;
        const float nrm = sqrtf(d2);
        const float hb = 16.f * u * h;
        // the lane's vertices r, r + G, ...: beyond -> bm, undecided -> FP64 from the inputs
        unsigned bm[TT / 32];
#pragma unroll
        for (int w = 0; w < TT / 32; w++) bm[w] = 0u;
        int f = 0;
        const int nT = C.nT;
        for (int t = r; t < nT; t += G) {
            const float4 v = C.V[t];
            const float sv = __fmaf_rn(dx, v.x, __fmaf_rn(dy, v.y, __fmaf_rn(dz, v.z, -h)));
            const float bound = __fmaf_rn(nrm, v.w, hb);
            int sd = sv > bound ? 1 : (sv < -bound ? -1 : 0);
            if (sd == 0 && !f) {
                uint32_t a, b, c;
                tri_ids(C.Tr[t], a, b, c);
                const PRef ra = {C.Ps[a], C.Pc[a]}, rb = {C.Ps[b], C.Pc[b]}, rc = {C.Ps[c], C.Pc[c]};
                const PRef rj = {j, (uint8_t)code};
                sd = side64<P>(spos, g, self, ra, rb, rc, rj);
                tc.fp64++;
                if (sd == 0) f = TF_UNDECIDED;
            }
            if (sd > 0) bm[t >> 5] |= 1u << (t & 31);
        }
        if (r == 0) tc.tested++;
        f = (int)__reduce_max_sync(gmask, (unsigned)f);
        if (f) return f;
        unsigned any = 0u;
#pragma unroll
        for (int w = 0; w < TT / 32; w++) {
            bm[w] = __reduce_or_sync(gmask, bm[w]);
            any |= bm[w];
        }
        if (!any) continue;
        int cf = 0;
        if (r == 0) {
            cf = cut_cell(C, bm, dx, dy, dz, h, nrm, j, code);
            if (!cf) {
                tc.cut++;
                bound_cell(C);
            }
        }
        __syncwarp(gmask);
        cf = __shfl_sync(gmask, cf, leader);
        if (cf) return cf;
    }
    return 0;
}

template <typename P, int G>
__global__ void __launch_bounds__(GWARPS * 32) k_clip_group(ClipArgs A) {
    constexpr int W = 32 / G;            // cells per warp
    constexpr int MODE = G == 4 ? 2 : 3;  // the threads-per-cell mode of this kernel's cells
    extern __shared__ __align__(16) unsigned char gsmem[];
    const int wib = (int)(threadIdx.x >> 5);
    TSmem& S = reinterpret_cast<TSmem*>(gsmem)[wib];
    const unsigned lane = lane_id(), lt = lanemask_lt();
    const int gi = (int)(lane / G);       // the lane's cell within the warp
    const int r = (int)(lane % G);        // its rank in the cell's group
    const unsigned gmask = group_mask<G>();
    GCell& GC = reinterpret_cast<GCell*>(gsmem + GWARPS * sizeof(TSmem))[wib * W + gi];
    TCell& C = GC.C;
    if (*((volatile unsigned*)&A.st->invalid_input)) return;
    const P* spos = (const P*)A.spos;
    const bool f64 = sizeof(P) != 16;
    const float u = Prec<float>::u();
    const int64_t nunits = (A.N + W - 1) / W;
    TCount tc = {0ull, 0ull, 0ull, 0ull, 0ull};
    for (;;) {
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(&A.st->work_next_group[G == 4 ? 0 : 1], 1ull);
        b = __shfl_sync(0xffffffffu, b, 0);
        if ((int64_t)b >= nunits) break;
        const int64_t self64 = (int64_t)b * W + gi;
        bool alive = self64 < A.N;
        const uint32_t self = alive ? (uint32_t)self64 : 0u;
        Geometry g = A.geo;
        int64_t slo = 0, shi = A.N;
        int mode = A.tpc_mode;
        if (A.sset && alive) {
            const uint32_t s = A.sset[self];
            g = A.sgeo[s];
            slo = A.soff[s];
            shi = A.soff[s + 1];
            if (A.set_cfg) mode = (A.set_cfg[s] >> 16) & 3;
        }
        if (mode != MODE) alive = false;  // another kernel's cell
        if (!__any_sync(0xffffffffu, alive)) continue;
        const P pi = spos[self];
        const float qx = (float)pi.x, qy = (float)pi.y, qz = (float)pi.z;
        // the box of the warp's live cells and their index range
        float blo[3] = {alive ? qx : INFINITY, alive ? qy : INFINITY, alive ? qz : INFINITY};
        float bhi[3] = {alive ? qx : -INFINITY, alive ? qy : -INFINITY, alive ? qz : -INFINITY};
        int64_t ilo = alive ? slo : INT64_MAX, ihi = alive ? shi : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
#pragma unroll
            for (int a = 0; a < 3; a++) {
                blo[a] = fminf(blo[a], __shfl_xor_sync(0xffffffffu, blo[a], o));
                bhi[a] = fmaxf(bhi[a], __shfl_xor_sync(0xffffffffu, bhi[a], o));
            }
            ilo = min(ilo, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)ilo, o));
            ihi = max(ihi, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)ihi, o));
        }
        // each cell's distance to its 4th nearest mate in its tree bucket (32 consecutive particles): lane l
        // takes mate l, the warp sorts the distances once per cell
        float near2 = INFINITY;
        {
            const int64_t jm = ((int64_t)b * W / 32) * 32 + lane;
            float mx = 0.f, my = 0.f, mz = 0.f;
            const bool mv = jm < A.N;
            if (mv) {
                const P pm = spos[jm];
                mx = (float)pm.x; my = (float)pm.y; mz = (float)pm.z;
            }
            const bool per = A.sset == nullptr && A.geo.periodic;
            for (int w = 0; w < W; w++) {
                const float sx = __shfl_sync(0xffffffffu, qx, w * G), sy = __shfl_sync(0xffffffffu, qy, w * G),
                            sz = __shfl_sync(0xffffffffu, qz, w * G);
                const long long wlo = __shfl_sync(0xffffffffu, (long long)slo, w * G),
                                whi = __shfl_sync(0xffffffffu, (long long)shi, w * G);
                const int64_t sw = (int64_t)b * W + w;
                float d2 = INFINITY;
                if (mv && jm != sw && jm >= wlo && jm < whi) {
                    float dx = fabsf(mx - sx), dy = fabsf(my - sy), dz = fabsf(mz - sz);
                    if (per) {
                        dx = fminf(dx, A.geo.Lf[0] - dx); dy = fminf(dy, A.geo.Lf[1] - dy); dz = fminf(dz, A.geo.Lf[2] - dz);
                    }
                    d2 = dx * dx + dy * dy + dz * dz;
                }
                for (int k = 2; k <= 32; k <<= 1)
                    for (int jj = k >> 1; jj > 0; jj >>= 1) {
                        const float o = __shfl_xor_sync(0xffffffffu, d2, jj);
                        const bool up = ((lane & k) == 0), lower = (lane & jj) == 0;
                        const float mn = fminf(d2, o), mx2 = fmaxf(d2, o);
                        d2 = (lower == up) ? mn : mx2;
                    }
                const float d4w = __shfl_sync(0xffffffffu, d2, 3);
                if (gi == w) near2 = d4w;
            }
        }
        // the warp's first radius: 1.6 x the median over its live cells of that distance
        float rho;
        {
            float d4 = alive ? near2 : INFINITY;
            for (int k = 2; k <= 32; k <<= 1)
                for (int jj = k >> 1; jj > 0; jj >>= 1) {
                    const float o = __shfl_xor_sync(0xffffffffu, d4, jj);
                    const bool up = ((lane & k) == 0), lower = (lane & jj) == 0;
                    const float mn = fminf(d4, o), mx = fmaxf(d4, o);
                    d4 = (lower == up) ? mn : mx;
                }
            const int n_alive = __popc(__ballot_sync(0xffffffffu, alive));
            d4 = __shfl_sync(0xffffffffu, d4, n_alive / 2);
            if (d4 < INFINITY && d4 > 0.f) rho = 1.6f * sqrtf(d4);
            else rho = (float)(2.0 * cbrt(g.L[0] * g.L[1] * g.L[2] / (double)max((int64_t)1, shi - slo)));
            rho = __shfl_sync(0xffffffffu, rho, 0);
        }
        const double lmin = fmin(g.L[0], fmin(g.L[1], g.L[2]));
        const float rho_cap = g.periodic ? (float)(0.24 * lmin) : INFINITY;
        if (rho > rho_cap) rho = rho_cap;
        if (!(near2 < INFINITY) || near2 <= 0.f) near2 = rho * rho * (1.f / 16.f);
        float slack = 16.f * u * fmaxf(fmaxf(fmaxf(fabsf(g.hif[0]), fabsf(g.lof[0])), fmaxf(fabsf(g.hif[1]), fabsf(g.lof[1]))),
                                        fmaxf(fmaxf(fabsf(g.hif[2]), fabsf(g.lof[2])), fmaxf(g.Lf[0], fmaxf(g.Lf[1], g.Lf[2])))) + 1e-30f;
        slack = warp_max<float>(alive ? slack : 0.f);
        // start box on the scale of the cell's own neighbourhood, set up by the group's first lane
        int fail = 0;
        {
            const float Bown = fminf(4.f * rho, 3.f * sqrtf(near2));
            if (alive && r == 0) fail = init_cell<P>(C, g, pi, self, Bown);
            __syncwarp();
            fail = __shfl_sync(0xffffffffu, fail, (int)(lane & ~(unsigned)(G - 1)));
        }
        const unsigned long long f64_before = tc.fp64;
        bool done = !alive;
        float g2prev = -1.f;
        int streamed = 0;
        for (int pass = 0; pass < TPASSES; pass++) {
            const bool want = alive && !done && !fail;
            if (!__any_sync(0xffffffffu, want)) break;
            if (lane == 0) tc.passes++;
            const float gr = rho * (1.f + 4.f * u) + slack;
            const float g2hi = gr * gr * (1.f + 4.f * u);
            int sp = 0;
            {
                const Tree& t = A.tree;
                const int top = t.levels;
                const int64_t span = (int64_t)1 << (5 * top);
                bool hit = false;
                float gap2 = -1.f;
                if ((int64_t)lane < t.count[top] && lane * span < ihi && (lane + 1) * span > ilo) {
                    const float4 lo = t.lo[t.off[top] + lane], hi = t.hi[t.off[top] + lane];
                    const float dx = iv_gap(lo.x, hi.x, blo[0], bhi[0], g.Lf[0], g.periodic);
                    const float dy = iv_gap(lo.y, hi.y, blo[1], bhi[1], g.Lf[1], g.periodic);
                    const float dz = iv_gap(lo.z, hi.z, blo[2], bhi[2], g.Lf[2], g.periodic);
                    gap2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, dx * dx));
                    hit = gap2 < g2hi * 1.0001f + 1e-30f;
                }
                if (!hit) gap2 = -1.f;
                const int nh = __popc(__ballot_sync(0xffffffffu, hit));
                uint32_t val = hit ? (((uint32_t)top << 27) | lane) : 0xffffffffu;
                warp_sort_desc(gap2, val);
                if ((int)lane < nh) S.stack[lane] = val;
                sp = nh;
                __syncwarp();
            }
            bool ovf = false;
            while (sp > 0) {
                const int cnt = walk(S, sp, 0, (const float4*)A.spos, A.spos, f64, A.tree, g, blo, bhi, g2prev, g2hi,
                                     ilo, ihi, ovf);
                streamed += cnt;
                if (lane == 0) tc.collected += cnt;
                if (ovf || streamed > TMAXPTS) { ovf = true; break; }
                if (cnt == 0) continue;
                {
                    const float cx = 0.5f * (blo[0] + bhi[0]), cy = 0.5f * (blo[1] + bhi[1]), cz = 0.5f * (blo[2] + bhi[2]);
                    for (int k = (int)lane; k < cnt; k += 32) {
                        const float4 q = S.chunk[k];
                        float dx = fabsf(q.x - cx), dy = fabsf(q.y - cy), dz = fabsf(q.z - cz);
                        if (g.periodic) {
                            dx = fminf(dx, g.Lf[0] - dx); dy = fminf(dy, g.Lf[1] - dy); dz = fminf(dz, g.Lf[2] - dz);
                        }
                        const float d2 = dx * dx + dy * dy + dz * dz;
                        S.key[k] = (__float_as_uint(d2) & ~255u) | (uint32_t)k;
                    }
                    __syncwarp();
                    sort_keys(S, cnt);
                }
                const bool act = alive && !done && !fail;
                const int f = clip_chunk_group<P, G>(S, cnt, GC, spos, g, pi, self, slo, shi, act, slack, tc);
                if (act && f) fail = f;
                __syncwarp();
            }
            if (ovf) {
                if (alive && !done && !fail) fail = TF_RADIUS;
                break;
            }
            g2prev = g2hi;
            if (alive && !done && !fail && 4.f * C.R2 <= rho * rho * (1.f - 8.f * u)) done = true;
            float need = (alive && !done && !fail) ? 2.f * sqrtf(C.R2) * 1.001f : 0.f;
            need = warp_max<float>(need);
            if (need == 0.f) break;
            float nxt = fminf(fmaxf(need, 1.25f * rho), 2.f * rho);
            if (rho >= rho_cap) break;
            rho = fminf(nxt, rho_cap);
        }
        if (alive && !done && !fail) fail = TF_RADIUS;
        // ---------------- emission by the group's first lane (any lane of the group may have re-tested in FP64)
        const bool used64 = (__ballot_sync(0xffffffffu, tc.fp64 != f64_before) & gmask) != 0u;
        const bool lead = alive && r == 0;
        int nf = 0;
        uint64_t present = 0ull;
        if (lead && !fail) {
            nf = count_faces(C, &present);
            if (nf < 0) fail = TF_WALL;
        }
        if (!(lead && !fail)) nf = 0;
        int incl = nf;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if ((int)lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long base = 0ull;
        if (lane == 0 && total > 0) base = atomicAdd(&A.st->face_next, (unsigned long long)total);
        base = __shfl_sync(0xffffffffu, base, 0);
        const bool pool_ok = base + (unsigned long long)total <= A.face_cap;
        if (!pool_ok) {
            if (lane == 0) atomicCAS(&A.st->error, 0, RC_POOL);
            if (lead && !fail) fail = TF_CAP;
        } else if (lead && !fail) {
            const uint32_t start = (uint32_t)(base + (unsigned long long)(incl - nf));
            float vol, mzx, mzy, mzz, m2;
            if (!emit_faces(C, present, A.faces + start, vol, mzx, mzy, mzz, m2)) {
                fail = TF_CAP_PLANES;
            } else {
                CellOut co;
                co.vol = (double)vol;
                co.zx = mzx / vol;
                co.zy = mzy / vol;
                co.zz = mzz / vol;
                co.mom2 = m2;
                A.cell[self] = co;
                A.face_start[self] = start;
                A.face_count[self] = (uint16_t)nf;
                A.cstat[self] = (uint8_t)(CS_DONE | (used64 ? CS_FP64 : 0));
                if (A.rad) A.rad[self] = sqrtf(C.R2) * (1.f + 1e-6f);
                atomicMax(&A.st->max_faces, (unsigned)nf);
            }
        }
        const bool emit = lead && !fail;
        const bool hand = lead && !emit;
        if (hand) atomicAdd(&A.st->n_tfail[fail > 0 && fail < 8 ? fail : 0], 1ull);
        const unsigned hm = __ballot_sync(0xffffffffu, hand);
        if (hm) {
            unsigned slot0 = 0;
            if (lane == 0) slot0 = atomicAdd(&A.st->n_warp_cells, (unsigned)__popc(hm));
            slot0 = __shfl_sync(0xffffffffu, slot0, 0);
            if (hand) A.warp_list[slot0 + __popc(hm & lt)] = self;
        }
        int nfe = emit ? nf : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) nfe += __shfl_xor_sync(0xffffffffu, nfe, o);
        if (lane == 0 && nfe > 0) atomicAdd(&A.st->n_faces, (unsigned long long)nfe);
        __syncwarp();
    }
    unsigned long long v[5] = {tc.tested, tc.cut, tc.fp64, tc.passes, tc.collected};
#pragma unroll
    for (int k = 0; k < 5; k++)
#pragma unroll
        for (int o = 16; o; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0) {
        atomicAdd(&A.st->n_tested, v[0]);
        atomicAdd(&A.st->n_cut, v[1]);
        atomicAdd(&A.st->n_fp64, v[2]);
        atomicAdd(&A.st->n_collected, v[4]);
    }
}

// ------------------------------------------------------------------ volume-averaged grid densities
// Volume of a (closed, convex) lane-local polytope, by the divergence theorem from the site (which need not lie
// inside): sum over planes of (signed offset / |n|) x area / 3.  A face is convex, so its vertices (the triangles
// that list the plane) are ordered by angle about their mean in the plane's own basis; the polygon area then
// needs nothing from the triangulation's adjacency, which a near-degenerate cut can leave inconsistent.
template <class CL>
__device__ float cell_volume(const CL& C) {
    float vol = 0.f;
    for (int p = 0; p < C.nP; p++) {
        float ang[CL::MT];
        uint8_t ft[CL::MT];
        int m = 0;
        float cx = 0.f, cy = 0.f, cz = 0.f;
        for (int t = 0; t < C.nT; t++) {
            uint32_t a, b, c;
            tri_ids(C.Tr[t], a, b, c);
            if (a != (uint32_t)p && b != (uint32_t)p && c != (uint32_t)p) continue;
            ft[m++] = (uint8_t)t;
            cx += C.V[t].x; cy += C.V[t].y; cz += C.V[t].z;
        }
        if (m < 3) continue;  // a plane that only touches the polytope: no area
        const float im = 1.f / (float)m;
        cx *= im; cy *= im; cz *= im;
        const float4 pl = C.Pl[p];
        const float inrm = 1.f / C.Pn[p];
        const float nx = pl.x * inrm, ny = pl.y * inrm, nz = pl.z * inrm;
        // u perpendicular to n, w = n x u
        float ux, uy, uz;
        if (fabsf(nx) < 0.9f) { ux = 0.f; uy = nz; uz = -ny; }
        else { ux = -nz; uy = 0.f; uz = nx; }
        const float iu = rsqrtf(ux * ux + uy * uy + uz * uz);
        ux *= iu; uy *= iu; uz *= iu;
        const float wx = ny * uz - nz * uy, wy = nz * ux - nx * uz, wz = nx * uy - ny * ux;
        for (int k = 0; k < m; k++) {
            const float4 v = C.V[ft[k]];
            const float dx = v.x - cx, dy = v.y - cy, dz = v.z - cz;
            ang[k] = atan2f(dx * wx + dy * wy + dz * wz, dx * ux + dy * uy + dz * uz);
        }
        for (int k = 1; k < m; k++) {  // insertion sort by angle
            const float a = ang[k];
            const uint8_t t = ft[k];
            int q = k - 1;
            while (q >= 0 && ang[q] > a) { ang[q + 1] = ang[q]; ft[q + 1] = ft[q]; q--; }
            ang[q + 1] = a;
            ft[q + 1] = t;
        }
        float area = 0.f;
        for (int k = 0; k < m; k++) {
            const float4 v1 = C.V[ft[k]], v2 = C.V[ft[k + 1 < m ? k + 1 : 0]];
            const float ax = v1.x - cx, ay = v1.y - cy, az = v1.z - cz;
            const float bx = v2.x - cx, by = v2.y - cy, bz = v2.z - cz;
            area += 0.5f * ((ay * bz - az * by) * nx + (az * bx - ax * bz) * ny + (ax * by - ay * bx) * nz);
        }
        vol += pl.w * inrm * area * (float)(1.0 / 3.0);
    }
    return vol;
}

// Cut C by n.y <= h for a volume: a vertex is removed when n.v - h > 0 in FP32 (no error bound: an
// ill-conditioned vertex has a wide bound that would keep a part the plane should remove, while a wrong sign on
// a vertex within rounding of the plane changes the volume by a rounding-sized sliver).  Returns 1 if C became
// empty, 0 otherwise, or a failure code (negative).
template <class CL>
__device__ int cut_plain(CL& C, float nx, float ny, float nz, float h, float nrm, uint32_t src = 0u,
                         int code = CODE_ART) {
    const float u = Prec<float>::u();
    unsigned bm[CL::MT / 32], um[CL::MT / 32];
    (void)u;
    test_plane(C, nx, ny, nz, h, 0.f, 0.f, bm, um);
    int nb = 0;
    for (int w = 0; w < CL::MT / 32; w++) nb += __popc(bm[w]);
    if (nb == 0) return 0;
    if (nb == C.nT) return 1;
    const int f = cut_cell(C, bm, nx, ny, nz, h, nrm, src, code);
    return f ? -f : 0;
}

struct GridArgs {
    const void* spos;
    int64_t N;
    Geometry geo;
    const Face* faces;
    const uint32_t* face_start;
    const uint16_t* face_count;
    const double* dens;  // sorted order
    int G;
    double h[3];         // voxel side L / G
    double* acc;         // [G^3] sum of rho |cell & voxel|
    int4* retry;         // (cell, voxel x, y, z unwrapped; x = INT_MIN: every voxel) for the larger cell type
    unsigned retry_cap;
    unsigned* n_retry;
    unsigned* n_fail;
};

// The cell of sorted particle k from its facet planes (start: a cube of half-side lmin/4, which holds every cell
// the build accepted, or the box walls).  Returns 0 or a failure code.
template <typename P, class CL>
__device__ int grid_cell(CL& C, const GridArgs& A, int64_t k, const P& pi) {
    const Geometry& g = A.geo;
    const double lmin = fmin(g.L[0], fmin(g.L[1], g.L[2]));
    const float B = g.periodic ? (float)(0.25 * lmin) : (float)(2.0 * fmax(g.L[0], fmax(g.L[1], g.L[2])));
    int f = init_cell<P>(C, g, pi, (uint32_t)k, B);
    const uint32_t st = A.face_start[k];
    const int cnt = A.face_count[k];
    for (int q = 0; q < cnt && !f; q++) {
        const Face fc = A.faces[st + q];
        const float d2 = __fmaf_rn(fc.dz, fc.dz, __fmaf_rn(fc.dy, fc.dy, fc.dx * fc.dx));
        // the plane keeps its neighbour's sorted index (code 0: a plane between particles)
        const int r = cut_plain(C, fc.dx, fc.dy, fc.dz, 0.5f * d2, sqrtf(d2), fc.nbr, 0);
        if (r) f = r < 0 ? -r : TF_CAP;  // a facet plane never empties its own cell
    }
    if (!f) bound_cell(C);
    return f;
}

// Volume of cell C inside voxel (ax, ay, az) (unwrapped indices; periodic boxes wrap them), translated by `shift`
// along every axis, into *vol; the voxel's linear index into *vi.  Returns 0, or a failure code; *vol = 0 when they
// do not meet.
template <class CL>
__device__ int voxel_part(const CL& C, CL& D, const GridArgs& A, const double* xi, int64_t ax, int64_t ay, int64_t az,
                          double shift, float* vol, int64_t* vi) {
    const Geometry& g = A.geo;
    const int64_t ia[3] = {ax, ay, az};
    int64_t v[3];
    double lo_[3], hi_[3];
    for (int c = 0; c < 3; c++) {
        int64_t q = ia[c] % A.G;
        if (q < 0) q += A.G;
        v[c] = q;
        const double sl = (double)((ia[c] - q) / A.G) * g.L[c];
        lo_[c] = g.lo[c] + (double)q * A.h[c] + sl - xi[c] + shift;
        hi_[c] = g.lo[c] + (double)(q + 1) * A.h[c] + sl - xi[c] + shift;
    }
    *vi = (v[2] * A.G + v[1]) * A.G + v[0];
    *vol = 0.f;
    if (lo_[0] > C.bmax[0] || hi_[0] < C.bmin[0] || lo_[1] > C.bmax[1] || hi_[1] < C.bmin[1] || lo_[2] > C.bmax[2] ||
        hi_[2] < C.bmin[2])
        return 0;
    D.nT = C.nT;
    D.nP = C.nP;
    for (int t = 0; t < C.nT; t++) { D.V[t] = C.V[t]; D.Tr[t] = C.Tr[t]; }
    for (int p = 0; p < C.nP; p++) { D.Pl[p] = C.Pl[p]; D.Pn[p] = C.Pn[p]; D.Ps[p] = C.Ps[p]; D.Pc[p] = C.Pc[p]; }
    for (int w = 0; w < 6; w++) {
        const int axis = w >> 1;
        const bool upper = (w & 1) == 0;
        const float sg = upper ? 1.f : -1.f;
        const float hh = upper ? (float)hi_[axis] : (float)(-lo_[axis]);
        const int r = cut_plain(D, axis == 0 ? sg : 0.f, axis == 1 ? sg : 0.f, axis == 2 ? sg : 0.f, hh, 1.f);
        if (r < 0) return -r;
        if (r) return 0;  // empty
    }
    const float vv = cell_volume(D);
    // a sliver's FP32 volume may come out slightly below zero; anything beyond 1e-5 of the voxel is a failure
    if (vv < -1e-5f * (float)(A.h[0] * A.h[1] * A.h[2])) return 10;
    *vol = fmaxf(vv, 0.f);
    return 0;
}

// The retry pass's part: unshifted first; a voxel wall that passes within the rounding bound of a cell vertex
// can make the kept and removed vertices of a cut inconsistent (the face splits), so the voxel is then
// translated by 1e-5 and 4e-5 of its side (the part's volume moves by at most that slab: far below FP32
// tolerance on the average) before giving up.
template <class CL>
__device__ int voxel_part_retry(const CL& C, CL& D, const GridArgs& A, const double* xi, int64_t ax, int64_t ay,
                                int64_t az, float* vol, int64_t* vi) {
    const double hmin = fmin(A.h[0], fmin(A.h[1], A.h[2]));
    int e = voxel_part(C, D, A, xi, ax, ay, az, 0.0, vol, vi);
    if (e) e = voxel_part(C, D, A, xi, ax, ay, az, 1e-5 * hmin, vol, vi);
    if (e) e = voxel_part(C, D, A, xi, ax, ay, az, -4e-5 * hmin, vol, vi);
    return e;
}

// a part that cannot be computed: counted in total and by reason (counters[4 + code])
__device__ __forceinline__ void grid_fail(const GridArgs& A, int code) {
    atomicAdd(A.n_fail, 1u);
    atomicAdd(A.n_fail + 3 + (code > 0 && code < 12 ? code : 0), 1u);
}

__device__ __forceinline__ void push_retry(const GridArgs& A, int64_t k, int ax, int ay, int az) {
    const unsigned slot = atomicAdd(A.n_retry, 1u);
    if (slot < A.retry_cap) A.retry[slot] = make_int4((int)k, ax, ay, az);
    else grid_fail(A, 11);
}

// One thread per cell (RETRY = false) or per retry entry (RETRY = true, the larger cell type): rho times the
// volume of the cell inside each voxel its box meets is added to that voxel.  A pair the small cell type
// cannot hold goes to the retry list, so that no voxel receives a part twice.
template <typename P, class CL, bool RETRY>
__global__ void __launch_bounds__(128) k_grid_volume(GridArgs A) {
    const int64_t n = RETRY ? (int64_t)min(*((volatile unsigned*)A.n_retry), A.retry_cap) : A.N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        int4 ent = make_int4(0, INT_MIN, 0, 0);
        if (RETRY) ent = A.retry[e];
        const int64_t k = RETRY ? (int64_t)ent.x : e;
        const P pi = ((const P*)A.spos)[k];
        CL C, D;
        int f = grid_cell<P, CL>(C, A, k, pi);
        if (f) {
            if (!RETRY) push_retry(A, k, INT_MIN, 0, 0);
            else grid_fail(A, f);
            continue;
        }
        const double xi[3] = {(double)pi.x, (double)pi.y, (double)pi.z};
        const double rho = A.dens[k];
        if (RETRY && ent.y != INT_MIN) {
            float vol;
            int64_t vi;
            const int e2 = voxel_part_retry(C, D, A, xi, ent.y, ent.z, ent.w, &vol, &vi);
            if (e2) grid_fail(A, e2);
            else if (vol > 0.f) atomicAdd(&A.acc[vi], rho * (double)vol);
            continue;
        }
        const Geometry& g = A.geo;
        int64_t a0[3], a1[3];
        for (int c = 0; c < 3; c++) {
            a0[c] = (int64_t)floor((xi[c] + (double)C.bmin[c] - g.lo[c]) / A.h[c]) - 1;
            a1[c] = (int64_t)floor((xi[c] + (double)C.bmax[c] - g.lo[c]) / A.h[c]) + 1;
            if (!g.periodic) {
                a0[c] = a0[c] < 0 ? 0 : a0[c];
                a1[c] = a1[c] > A.G - 1 ? A.G - 1 : a1[c];
            }
        }
        for (int64_t az = a0[2]; az <= a1[2]; az++)
            for (int64_t ay = a0[1]; ay <= a1[1]; ay++)
                for (int64_t ax = a0[0]; ax <= a1[0]; ax++) {
                    float vol;
                    int64_t vi;
                    const int e2 = RETRY ? voxel_part_retry(C, D, A, xi, ax, ay, az, &vol, &vi)
                                         : voxel_part(C, D, A, xi, ax, ay, az, 0.0, &vol, &vi);
                    if (e2) {
                        if (!RETRY) push_retry(A, k, (int)ax, (int)ay, (int)az);
                        else grid_fail(A, e2);
                    } else if (vol > 0.f) {
                        atomicAdd(&A.acc[vi], rho * (double)vol);
                    }
                }
    }
}

// ------------------------------------------------------------------ weighted centroidal energy gradient
// integral of |y|^2 y over the triangle (a, b, c) divided by its area: the degree-3 rule of Strang and Fix
// (weight -27/48 at the centroid, 25/48 at barycentric (3/5, 1/5, 1/5) and its permutations), exact for cubics
__device__ __forceinline__ void tri_m3(float4 a, float4 b, float4 c, float* out) {
    const float w0 = -27.f / 48.f, w1 = 25.f / 48.f;
    float px[4], py[4], pz[4];
    px[0] = (a.x + b.x + c.x) * (1.f / 3.f); py[0] = (a.y + b.y + c.y) * (1.f / 3.f); pz[0] = (a.z + b.z + c.z) * (1.f / 3.f);
    px[1] = 0.6f * a.x + 0.2f * b.x + 0.2f * c.x; py[1] = 0.6f * a.y + 0.2f * b.y + 0.2f * c.y; pz[1] = 0.6f * a.z + 0.2f * b.z + 0.2f * c.z;
    px[2] = 0.2f * a.x + 0.6f * b.x + 0.2f * c.x; py[2] = 0.2f * a.y + 0.6f * b.y + 0.2f * c.y; pz[2] = 0.2f * a.z + 0.6f * b.z + 0.2f * c.z;
    px[3] = 0.2f * a.x + 0.2f * b.x + 0.6f * c.x; py[3] = 0.2f * a.y + 0.2f * b.y + 0.6f * c.y; pz[3] = 0.2f * a.z + 0.2f * b.z + 0.6f * c.z;
    out[0] = out[1] = out[2] = 0.f;
    for (int k = 0; k < 4; k++) {
        const float w = (k == 0 ? w0 : w1) * (px[k] * px[k] + py[k] * py[k] + pz[k] * pz[k]);
        out[0] += w * px[k]; out[1] += w * py[k]; out[2] += w * pz[k];
    }
}

struct CvtArgs {
    const void* spos;
    int64_t N;
    Geometry geo;
    const Face* faces;
    const uint32_t* face_start;
    const uint16_t* face_count;
    const CellOut* cell;
    const uint32_t* perm;
    const void* w;        // weights, input order, dtype of pos
    int dtype;
    void* out;            // dE_w / dx, input order [N][3]
    int4* retry;
    unsigned retry_cap;
    unsigned* n_retry;
    unsigned* n_fail;
};

// dE_w/dx_k = 2 w_k V_k (x_k - z_k) + sum over facets (w_k - w_j) / |d| integral_f |y - x_k|^2 (y - x_k) dA, one
// thread per cell (RETRY: per listed cell, larger cell type); the facet integral over the facet polygon of the cell
// rebuilt from its facet planes, vertices ordered by angle in the facet plane and fanned.
template <typename P, class CL, bool RETRY>
__global__ void __launch_bounds__(128) k_cvt_weighted(CvtArgs A) {
    const int64_t n = RETRY ? (int64_t)min(*((volatile unsigned*)A.n_retry), A.retry_cap) : A.N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = RETRY ? (int64_t)A.retry[e].x : e;
        const P pi = ((const P*)A.spos)[k];
        GridArgs ga;
        ga.geo = A.geo; ga.faces = A.faces; ga.face_start = A.face_start; ga.face_count = A.face_count;
        CL C;
        const int f = grid_cell<P, CL>(C, ga, k, pi);
        if (f) {
            if (!RETRY) {
                const unsigned slot = atomicAdd(A.n_retry, 1u);
                if (slot < A.retry_cap) A.retry[slot] = make_int4((int)k, 0, 0, 0);
                else atomicAdd(A.n_fail, 1u);
            } else {
                atomicAdd(A.n_fail, 1u);
            }
            continue;
        }
        const uint32_t ik = A.perm[k];
        const double wk = A.dtype == VT_F32 ? (double)((const float*)A.w)[ik] : ((const double*)A.w)[ik];
        const CellOut co = A.cell[k];
        double gx = -2.0 * wk * co.vol * co.zx, gy = -2.0 * wk * co.vol * co.zy, gz = -2.0 * wk * co.vol * co.zz;
        for (int p = 6; p < C.nP; p++) {
            if (C.Pc[p] >= 27) continue;
            float ang[CL::MT];
            uint8_t ft[CL::MT];
            int m = 0;
            float cx = 0.f, cy = 0.f, cz = 0.f;
            for (int t = 0; t < C.nT; t++) {
                uint32_t a, b, c;
                tri_ids(C.Tr[t], a, b, c);
                if (a != (uint32_t)p && b != (uint32_t)p && c != (uint32_t)p) continue;
                ft[m++] = (uint8_t)t;
                cx += C.V[t].x; cy += C.V[t].y; cz += C.V[t].z;
            }
            if (m < 3) continue;
            const float im = 1.f / (float)m;
            cx *= im; cy *= im; cz *= im;
            const float4 pl = C.Pl[p];
            const float inrm = 1.f / C.Pn[p];
            const float nx = pl.x * inrm, ny = pl.y * inrm, nz = pl.z * inrm;
            float ux, uy, uz;
            if (fabsf(nx) < 0.9f) { ux = 0.f; uy = nz; uz = -ny; }
            else { ux = -nz; uy = 0.f; uz = nx; }
            const float iu = rsqrtf(ux * ux + uy * uy + uz * uz);
            ux *= iu; uy *= iu; uz *= iu;
            const float wx = ny * uz - nz * uy, wy = nz * ux - nx * uz, wz = nx * uy - ny * ux;
            for (int q = 0; q < m; q++) {
                const float4 v = C.V[ft[q]];
                const float dx = v.x - cx, dy = v.y - cy, dz = v.z - cz;
                ang[q] = atan2f(dx * wx + dy * wy + dz * wz, dx * ux + dy * uy + dz * uz);
            }
            for (int q = 1; q < m; q++) {
                const float a = ang[q];
                const uint8_t t = ft[q];
                int r = q - 1;
                while (r >= 0 && ang[r] > a) { ang[r + 1] = ang[r]; ft[r + 1] = ft[r]; r--; }
                ang[r + 1] = a;
                ft[r + 1] = t;
            }
            // fan from the first vertex: area along the outward normal times the rule's mean of |y|^2 y
            double mx = 0.0, my = 0.0, mz = 0.0;
            const float4 v0 = C.V[ft[0]];
            for (int q = 1; q + 1 < m; q++) {
                const float4 v1 = C.V[ft[q]], v2 = C.V[ft[q + 1]];
                const float e1x = v1.x - v0.x, e1y = v1.y - v0.y, e1z = v1.z - v0.z;
                const float e2x = v2.x - v0.x, e2y = v2.y - v0.y, e2z = v2.z - v0.z;
                const float at = 0.5f * ((e1y * e2z - e1z * e2y) * nx + (e1z * e2x - e1x * e2z) * ny +
                                         (e1x * e2y - e1y * e2x) * nz);
                float t3[3];
                tri_m3(v0, v1, v2, t3);
                mx += (double)at * t3[0]; my += (double)at * t3[1]; mz += (double)at * t3[2];
            }
            const uint32_t ij = A.perm[C.Ps[p]];
            const double wj = A.dtype == VT_F32 ? (double)((const float*)A.w)[ij] : ((const double*)A.w)[ij];
            const double cf = (wk - wj) * (double)inrm;
            gx += cf * mx; gy += cf * my; gz += cf * mz;
        }
        if (A.dtype == VT_F32) {
            float* o = (float*)A.out + 3 * (int64_t)ik;
            o[0] = (float)gx; o[1] = (float)gy; o[2] = (float)gz;
        } else {
            double* o = (double*)A.out + 3 * (int64_t)ik;
            o[0] = gx; o[1] = gy; o[2] = gz;
        }
    }
}

template <typename T>
__global__ void k_grid_finish(const double* __restrict__ acc, int64_t n, double inv_vox, T* __restrict__ out) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) out[v] = (T)(acc[v] * inv_vox);
}


template <typename P, int G>
int launch_group_t(const ClipArgs& a, int sm_count, cudaStream_t s) {
    constexpr int W = 32 / G;
    const size_t smem = GWARPS * (sizeof(TSmem) + W * sizeof(GCell));
    static int per_sm_dev[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    int per_sm = (dev >= 0 && dev < 64) ? per_sm_dev[dev] : 0;
    if (per_sm == 0) {
        cudaFuncSetAttribute(k_clip_group<P, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_clip_group<P, G>, GWARPS * 32, smem);
        if (per_sm < 1) per_sm = 1;
        if (dev >= 0 && dev < 64) per_sm_dev[dev] = per_sm;
    }
    k_clip_group<P, G><<<sm_count * per_sm, GWARPS * 32, smem, s>>>(a);
    return 1;
}
}  // namespace

int launch_grid_volume(const void* spos, int dtype, int64_t N, const Geometry& g, const Face* faces,
                       const uint32_t* face_start, const uint16_t* face_count, const double* dens_sorted, int G,
                       double* acc, int4* retry, unsigned retry_cap, unsigned* counters, void* out, int sm_count,
                       cudaStream_t s) {
    GridArgs a;
    a.spos = spos; a.N = N; a.geo = g; a.faces = faces; a.face_start = face_start; a.face_count = face_count;
    a.dens = dens_sorted; a.G = G; a.acc = acc; a.retry = retry; a.retry_cap = retry_cap;
    a.n_retry = counters; a.n_fail = counters + 1;
    for (int c = 0; c < 3; c++) a.h[c] = g.L[c] / G;
    const int64_t n = (int64_t)G * G * G;
    cudaMemsetAsync(acc, 0, n * sizeof(double), s);
    cudaMemsetAsync(counters, 0, 16 * sizeof(unsigned), s);
    const unsigned nb = (unsigned)((N + 127) / 128);
    const unsigned rb = (unsigned)(sm_count * 4);
    if (dtype == VT_F32) {
        k_grid_volume<float4, TCell, false><<<nb, 128, 0, s>>>(a);
        k_grid_volume<float4, TCellBig, true><<<rb, 128, 0, s>>>(a);
    } else {
        k_grid_volume<dpt4, TCell, false><<<nb, 128, 0, s>>>(a);
        k_grid_volume<dpt4, TCellBig, true><<<rb, 128, 0, s>>>(a);
    }
    const double inv = 1.0 / (a.h[0] * a.h[1] * a.h[2]);
    const unsigned gb = (unsigned)((n + 255) / 256);
    if (dtype == VT_F32) k_grid_finish<float><<<gb, 256, 0, s>>>(acc, n, inv, (float*)out);
    else k_grid_finish<double><<<gb, 256, 0, s>>>(acc, n, inv, (double*)out);
    return 3;
}

int launch_cvt_weighted(const void* spos, int dtype, int64_t N, const Geometry& g, const Face* faces,
                        const uint32_t* face_start, const uint16_t* face_count, const CellOut* cell,
                        const uint32_t* perm, const void* w, void* out, int4* retry, unsigned retry_cap,
                        unsigned* counters, int sm_count, cudaStream_t s) {
    CvtArgs a;
    a.spos = spos; a.N = N; a.geo = g; a.faces = faces; a.face_start = face_start; a.face_count = face_count;
    a.cell = cell; a.perm = perm; a.w = w; a.dtype = dtype; a.out = out; a.retry = retry; a.retry_cap = retry_cap;
    a.n_retry = counters; a.n_fail = counters + 1;
    cudaMemsetAsync(counters, 0, 16 * sizeof(unsigned), s);
    const unsigned nb = (unsigned)((N + 127) / 128);
    const unsigned rb = (unsigned)(sm_count * 4);
    if (dtype == VT_F32) {
        k_cvt_weighted<float4, TCell, false><<<nb, 128, 0, s>>>(a);
        k_cvt_weighted<float4, TCellBig, true><<<rb, 128, 0, s>>>(a);
    } else {
        k_cvt_weighted<dpt4, TCell, false><<<nb, 128, 0, s>>>(a);
        k_cvt_weighted<dpt4, TCellBig, true><<<rb, 128, 0, s>>>(a);
    }
    return 2;
}

int launch_clip_group(const ClipArgs& a, int dtype, int lanes, int sm_count, cudaStream_t s) {
    if (dtype == VT_F32) return lanes == 4 ? launch_group_t<float4, 4>(a, sm_count, s) : launch_group_t<float4, 8>(a, sm_count, s);
    return lanes == 4 ? launch_group_t<dpt4, 4>(a, sm_count, s) : launch_group_t<dpt4, 8>(a, sm_count, s);
}

int launch_clip_thread(const ClipArgs& a, int dtype, int sm_count, cudaStream_t s) {
    static int per_sm_dev[2][64] = {{0}};
    int dev = 0;
    cudaGetDevice(&dev);
    const int k = dtype == VT_F32 ? 0 : 1;
    int per_sm = (dev >= 0 && dev < 64) ? per_sm_dev[k][dev] : 0;
    if (per_sm == 0) {
        if (dtype == VT_F32)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_clip_thread<float4>, TWARPS * 32, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_clip_thread<dpt4>, TWARPS * 32, 0);
        if (per_sm < 1) per_sm = 1;
        if (dev >= 0 && dev < 64) per_sm_dev[k][dev] = per_sm;
    }
    const int blocks = sm_count * per_sm;
    if (dtype == VT_F32) k_clip_thread<float4><<<blocks, TWARPS * 32, 0, s>>>(a);
    else k_clip_thread<dpt4><<<blocks, TWARPS * 32, 0, s>>>(a);
    return 1;
}

}  // namespace vt
