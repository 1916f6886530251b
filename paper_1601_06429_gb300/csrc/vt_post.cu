// vt_post.cu -- per-particle products of the cells (hot-path steps A5-A9):
// volumes and densities in input order, the neighbour lists (CSR, real indices,
// ascending), the least-squares density gradient, the grid densities and the
// volume adjoint.  All gathers go through the facet records written by the
// clipping kernel; the particles are in Morton order, so neighbour gathers hit L2.
#include <cuda_runtime.h>
#include <stdint.h>

#include "vt_internal.cuh"
#include "vt_kernels.cuh"

namespace vt {

template <typename P> struct PT;
template <> struct PT<float4> { typedef float T; };
template <> struct PT<dpt4> { typedef double T; };

// ------------------------------------------------------------------ volume / density
template <typename T>
__global__ void k_out_vol(const CellOut* __restrict__ cell, const uint32_t* __restrict__ perm, int64_t N,
                          T* __restrict__ vol) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N) vol[perm[k]] = (T)cell[k].vol;
}

void launch_out_vol(const CellOut* cell, const uint32_t* perm, int64_t N, void* vol, int dtype, cudaStream_t s) {
    unsigned nb = (unsigned)((N + 255) / 256);
    if (dtype == VT_F32) k_out_vol<float><<<nb, 256, 0, s>>>(cell, perm, N, (float*)vol);
    else k_out_vol<double><<<nb, 256, 0, s>>>(cell, perm, N, (double*)vol);
}

// Implementation section: density = particle mass / cell volume
template <typename P, typename T>
__global__ void k_density(const CellOut* __restrict__ cell, const P* __restrict__ spos,
                          const uint32_t* __restrict__ perm, int64_t N, double* __restrict__ dens_sorted,
                          T* __restrict__ dens) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    double d = (double)spos[k].w / cell[k].vol;
    dens_sorted[k] = d;
    if (dens) dens[perm[k]] = (T)d;
}

void launch_density(const CellOut* cell, const void* spos, int dtype, const uint32_t* perm, int64_t N,
                    double* dens_sorted, void* dens, cudaStream_t s) {
    unsigned nb = (unsigned)((N + 255) / 256);
    if (dtype == VT_F32)
        k_density<float4, float><<<nb, 256, 0, s>>>(cell, (const float4*)spos, perm, N, dens_sorted,
                                                     (float*)dens);
    else
        k_density<dpt4, double><<<nb, 256, 0, s>>>(cell, (const dpt4*)spos, perm, N, dens_sorted,
                                                    (double*)dens);
}

// ------------------------------------------------------------------ neighbour lists
__global__ void k_nbr_count(const uint16_t* __restrict__ face_count, const uint32_t* __restrict__ inv, int64_t N,
                            uint16_t* __restrict__ cnt_in) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) cnt_in[i] = face_count[inv[i]];
}

void launch_nbr_count(const uint16_t* face_count, const uint32_t* inv, int64_t N, uint16_t* cnt_in, cudaStream_t s) {
    k_nbr_count<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(face_count, inv, N, cnt_in);
}

// one warp per particle (input order): its facets' neighbours mapped to input indices, sorted ascending
constexpr int EMIT_WARPS = 8;
__global__ void __launch_bounds__(EMIT_WARPS * 32) k_nbr_emit(const Face* __restrict__ faces,
                                                              const uint32_t* __restrict__ face_start,
                                                              const uint16_t* __restrict__ face_count,
                                                              const uint32_t* __restrict__ perm,
                                                              const uint32_t* __restrict__ inv,
                                                              const int64_t* __restrict__ nbr_off, int64_t N,
                                                              int32_t* __restrict__ nbr_id) {
    __shared__ uint32_t buf[EMIT_WARPS][MAXP];
    const int w = threadIdx.x >> 5;
    const unsigned lane = threadIdx.x & 31;
    int64_t i = (int64_t)blockIdx.x * EMIT_WARPS + w;
    if (i >= N) return;
    uint32_t k = inv[i];
    uint32_t st = face_start[k];
    int cnt = face_count[k];
    int64_t o = nbr_off[i];
    if (cnt <= 32) {
        uint32_t v = 0xffffffffu;
        if ((int)lane < cnt) v = perm[faces[st + lane].nbr];
        for (int kk = 2; kk <= 32; kk <<= 1)
            for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                uint32_t q = __shfl_xor_sync(0xffffffffu, v, jj);
                bool up = (lane & kk) == 0, lower = (lane & jj) == 0;
                uint32_t mn = min(v, q), mx = max(v, q);
                v = (lower == up) ? mn : mx;
            }
        if ((int)lane < cnt) nbr_id[o + lane] = (int32_t)v;
        return;
    }
    int m = 64;
    while (m < cnt) m <<= 1;
    for (int q = lane; q < m; q += 32) buf[w][q] = q < cnt ? perm[faces[st + q].nbr] : 0xffffffffu;
    __syncwarp();
    for (int kk = 2; kk <= m; kk <<= 1)
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int q = lane; q < m; q += 32) {
                int x = q ^ jj;
                if (x > q) {
                    uint32_t a = buf[w][q], b = buf[w][x];
                    bool asc = (q & kk) == 0;
                    if ((a > b) == asc) { buf[w][q] = b; buf[w][x] = a; }
                }
            }
            __syncwarp();
        }
    for (int q = lane; q < cnt; q += 32) nbr_id[o + q] = (int32_t)buf[w][q];
}

void launch_nbr_emit(const Face* faces, const uint32_t* face_start, const uint16_t* face_count, const uint32_t* perm,
                     const uint32_t* inv, const int64_t* nbr_off, int64_t N, int32_t* nbr_id, cudaStream_t s) {
    unsigned nb = (unsigned)((N + EMIT_WARPS - 1) / EMIT_WARPS);
    k_nbr_emit<<<nb, EMIT_WARPS * 32, 0, s>>>(faces, face_start, face_count, perm, inv, nbr_off, N, nbr_id);
}

// ------------------------------------------------------------------ density gradient
// Implementation section ("density gradient ... using density and neighboring information"); reading:
// least squares over the Voronoi neighbours, (sum d d^T) g = sum d (rho_j - rho_i), solved by Cramer's rule.
template <typename T>
__global__ void k_gradient(const Face* __restrict__ faces, const uint32_t* __restrict__ face_start,
                           const uint16_t* __restrict__ face_count, const double* __restrict__ dens,
                           const uint32_t* __restrict__ perm, int64_t N, T* __restrict__ grad) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    uint32_t st = face_start[k];
    int cnt = face_count[k];
    double ri = dens[k];
    float mxx = 0.f, mxy = 0.f, mxz = 0.f, myy = 0.f, myz = 0.f, mzz = 0.f;
    double bx = 0.0, by = 0.0, bz = 0.0;
    for (int q = 0; q < cnt; q++) {
        Face f = faces[st + q];
        double dr = dens[f.nbr] - ri;
        mxx = fmaf(f.dx, f.dx, mxx); mxy = fmaf(f.dx, f.dy, mxy); mxz = fmaf(f.dx, f.dz, mxz);
        myy = fmaf(f.dy, f.dy, myy); myz = fmaf(f.dy, f.dz, myz); mzz = fmaf(f.dz, f.dz, mzz);
        bx = fma((double)f.dx, dr, bx); by = fma((double)f.dy, dr, by); bz = fma((double)f.dz, dr, bz);
    }
    double a = mxx, b = mxy, c = mxz, d = myy, e = myz, ff = mzz;
    double c00 = d * ff - e * e, c01 = c * e - b * ff, c02 = b * e - c * d;
    double c11 = a * ff - c * c, c12 = b * c - a * e, c22 = a * d - b * b;
    double det = a * c00 + b * c01 + c * c02;
    double gx = 0, gy = 0, gz = 0;
    if (det != 0.0) {
        double id = 1.0 / det;
        gx = (c00 * bx + c01 * by + c02 * bz) * id;
        gy = (c01 * bx + c11 * by + c12 * bz) * id;
        gz = (c02 * bx + c12 * by + c22 * bz) * id;
    }
    uint32_t i = perm[k];
    grad[3 * (int64_t)i + 0] = (T)gx;
    grad[3 * (int64_t)i + 1] = (T)gy;
    grad[3 * (int64_t)i + 2] = (T)gz;
}

void launch_gradient(const Face* faces, const uint32_t* face_start, const uint16_t* face_count, const double* dens_sorted,
                     const uint32_t* perm, int64_t N, void* grad, int dtype, cudaStream_t s) {
    unsigned nb = (unsigned)((N + 255) / 256);
    if (dtype == VT_F32)
        k_gradient<float><<<nb, 256, 0, s>>>(faces, face_start, face_count, dens_sorted, perm, N,
                                             (float*)grad);
    else
        k_gradient<double><<<nb, 256, 0, s>>>(faces, face_start, face_count, dens_sorted, perm, N,
                                              (double*)grad);
}

// ------------------------------------------------------------------ grid densities
// Implementation section ("average Voronoi densities on a regular grid"); reading: the density of the cell
// containing each of the node's S^3 sub-points (its nearest particle), averaged.  The nearest particle is
// decided in FP64 with the fixed evaluation order fma(dz,dz, fma(dy,dy, dx*dx)) on minimum-image dx, ties to
// the lower input index; FP32 is only used to prune.
__device__ __forceinline__ float gap1(float q, float lo, float hi, float L, int periodic) {
    float d = fmaxf(fmaxf(lo - q, q - hi), 0.f);
    if (periodic) {
        d = fminf(d, fmaxf(lo + L - q, 0.f));
        d = fminf(d, fmaxf(q + L - hi, 0.f));
    }
    return d;
}
__device__ __forceinline__ double wrap_d(double t, double L, int periodic) {
    if (periodic) {
        if (t > 0.5 * L) t = __dsub_rn(t, L);
        else if (t < -0.5 * L) t = __dadd_rn(t, L);
    }
    return t;
}

constexpr int GRID_WARPS = 4;
constexpr int GSTACK = 192;

template <typename P>
__global__ void __launch_bounds__(GRID_WARPS * 32) k_grid(const P* __restrict__ spos, int64_t N, Geometry g, Tree t,
                                                           const double* __restrict__ dens,
                                                           const uint32_t* __restrict__ perm, int G, int S,
                                                           void* __restrict__ out, int dtype, DevStatus* st) {
    __shared__ uint32_t stack[GRID_WARPS][GSTACK];
    const int w = threadIdx.x >> 5;
    const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
    const int S3 = S * S * S;
    const int64_t gw = (int64_t)blockIdx.x * GRID_WARPS + w, nw = (int64_t)gridDim.x * GRID_WARPS;
    const float slack = 4.0f * 1.2e-7f *
                        fmaxf(fmaxf(fabsf(g.hif[0]), fabsf(g.lof[0])),
                              fmaxf(fmaxf(fabsf(g.hif[1]), fabsf(g.lof[1])), fmaxf(fabsf(g.hif[2]), fabsf(g.lof[2]))));
    uint32_t guess = 0;  // sorted index of the last answer (spatial coherence along rows)
    // each warp takes whole rows of G nodes along x
    for (int64_t row = gw; row < (int64_t)G * G; row += nw) {
        for (int a = 0; a < G; a++) {
            int64_t node = row * G + a;
            int b = (int)(row % G), c = (int)(row / G);
            double acc = 0.0;
            for (int sp = 0; sp < S3; sp++) {
                int uu = sp % S, vv = (sp / S) % S, ww = sp / (S * S);
                double qd[3];
                qd[0] = __dadd_rn(g.lo[0], __dmul_rn(__dadd_rn((double)a, __ddiv_rn(__dadd_rn((double)uu, 0.5), (double)S)),
                                                     __ddiv_rn(g.L[0], (double)G)));
                qd[1] = __dadd_rn(g.lo[1], __dmul_rn(__dadd_rn((double)b, __ddiv_rn(__dadd_rn((double)vv, 0.5), (double)S)),
                                                     __ddiv_rn(g.L[1], (double)G)));
                qd[2] = __dadd_rn(g.lo[2], __dmul_rn(__dadd_rn((double)c, __ddiv_rn(__dadd_rn((double)ww, 0.5), (double)S)),
                                                     __ddiv_rn(g.L[2], (double)G)));
                float qx = (float)qd[0], qy = (float)qd[1], qz = (float)qd[2];
                // initial bound from the previous answer
                double best;
                uint32_t bj = guess, bi;
                {
                    P pj = spos[bj];
                    double dx = wrap_d(__dsub_rn((double)pj.x, qd[0]), g.L[0], g.periodic);
                    double dy = wrap_d(__dsub_rn((double)pj.y, qd[1]), g.L[1], g.periodic);
                    double dz = wrap_d(__dsub_rn((double)pj.z, qd[2]), g.L[2], g.periodic);
                    best = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
                    bi = perm[bj];
                }
                float bestf = (float)best * 1.0001f + 1e-30f;
                int top = t.levels;
                int spn = 0;
                {
                    bool hit = false;
                    if ((int64_t)lane < t.count[top]) {
                        float4 lo = t.lo[t.off[top] + lane], hi = t.hi[t.off[top] + lane];
                        float dx = fmaxf(gap1(qx, lo.x, hi.x, g.Lf[0], g.periodic) - slack, 0.f);
                        float dy = fmaxf(gap1(qy, lo.y, hi.y, g.Lf[1], g.periodic) - slack, 0.f);
                        float dz = fmaxf(gap1(qz, lo.z, hi.z, g.Lf[2], g.periodic) - slack, 0.f);
                        hit = dx * dx + dy * dy + dz * dz <= bestf;
                    }
                    unsigned m = __ballot_sync(0xffffffffu, hit);
                    if (hit) stack[w][__popc(m & lt)] = ((uint32_t)top << 27) | lane;
                    spn = __popc(m);
                }
                __syncwarp();
                while (spn > 0) {
                    uint32_t ent = stack[w][spn - 1];
                    spn--;
                    __syncwarp();
                    int lvl = ent >> 27;
                    int64_t nd = ent & ((1u << 27) - 1);
                    if (lvl == 1) {
                        int64_t j = nd * 32 + lane;
                        double d2 = INFINITY;
                        uint32_t ji = 0xffffffffu;
                        if (j < N) {
                            P pj = spos[j];
                            float fx = fabsf((float)pj.x - qx), fy = fabsf((float)pj.y - qy), fz = fabsf((float)pj.z - qz);
                            if (g.periodic) {
                                fx = fminf(fx, g.Lf[0] - fx); fy = fminf(fy, g.Lf[1] - fy); fz = fminf(fz, g.Lf[2] - fz);
                            }
                            // each float component is within `slack` of its FP64 value
                            float df = sqrtf(fx * fx + fy * fy + fz * fz);
                            if (df <= sqrtf(bestf) + 4.f * slack) {
                                double dx = wrap_d(__dsub_rn((double)pj.x, qd[0]), g.L[0], g.periodic);
                                double dy = wrap_d(__dsub_rn((double)pj.y, qd[1]), g.L[1], g.periodic);
                                double dz = wrap_d(__dsub_rn((double)pj.z, qd[2]), g.L[2], g.periodic);
                                d2 = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
                                ji = perm[j];
                            }
                        }
                        // warp argmin over (d2, input index)
                        double md = d2;
                        uint32_t mi = ji, ms = (uint32_t)j;
#pragma unroll
                        for (int o = 16; o; o >>= 1) {
                            double od = __shfl_xor_sync(0xffffffffu, md, o);
                            uint32_t oi = __shfl_xor_sync(0xffffffffu, mi, o);
                            uint32_t os = __shfl_xor_sync(0xffffffffu, ms, o);
                            if (od < md || (od == md && oi < mi)) { md = od; mi = oi; ms = os; }
                        }
                        if (md < best || (md == best && mi < bi)) {
                            best = md; bi = mi; bj = ms;
                            bestf = (float)best * 1.0001f + 1e-30f;
                        }
                    } else {
                        int cl = lvl - 1;
                        int64_t ch = nd * 32 + lane;
                        bool hit = false;
                        if (ch < t.count[cl]) {
                            float4 lo = t.lo[t.off[cl] + ch], hi = t.hi[t.off[cl] + ch];
                            float dx = fmaxf(gap1(qx, lo.x, hi.x, g.Lf[0], g.periodic) - slack, 0.f);
                            float dy = fmaxf(gap1(qy, lo.y, hi.y, g.Lf[1], g.periodic) - slack, 0.f);
                            float dz = fmaxf(gap1(qz, lo.z, hi.z, g.Lf[2], g.periodic) - slack, 0.f);
                            hit = dx * dx + dy * dy + dz * dz <= bestf;
                        }
                        unsigned m = __ballot_sync(0xffffffffu, hit);
                        if (spn + __popc(m) > GSTACK) {
                            if (lane == 0) atomicCAS(&st->error, 0, VT_ERR_CAPACITY);
                            break;
                        }
                        if (hit) stack[w][spn + __popc(m & lt)] = ((uint32_t)cl << 27) | (uint32_t)ch;
                        spn += __popc(m);
                        __syncwarp();
                    }
                }
                guess = bj;
                acc += dens[bj];
            }
            if (lane == 0) {
                double v = acc / S3;
                if (dtype == VT_F32) ((float*)out)[node] = (float)v;
                else ((double*)out)[node] = v;
            }
        }
    }
}

void launch_grid(const void* spos, int dtype, int64_t N, const Geometry& g, const Tree& t, const double* dens_sorted,
                 const uint32_t* perm, int G, int S, void* grid, DevStatus* st, int sm_count, cudaStream_t s) {
    int blocks = sm_count * 8;
    if (dtype == VT_F32)
        k_grid<float4><<<blocks, GRID_WARPS * 32, 0, s>>>((const float4*)spos, N, g, t, dens_sorted,
                                                          perm, G, S, grid, dtype, st);
    else
        k_grid<dpt4><<<blocks, GRID_WARPS * 32, 0, s>>>((const dpt4*)spos, N, g, t, dens_sorted, perm,
                                                        G, S, grid, dtype, st);
}

// ------------------------------------------------------------------ backward
// dL/dx_k = sum_j (A_kj/|r_kj|)(g_k - g_j)(c_kj - x_k) + dL_dE * 2 V_k (x_k - z_k); one thread per cell,
// a gather over the cell's own facets (each facet is stored from both sides, so no atomics are needed).
template <typename T>
__global__ void k_backward(const Face* __restrict__ faces, const uint32_t* __restrict__ face_start,
                           const uint16_t* __restrict__ face_count, const CellOut* __restrict__ cell,
                           const uint32_t* __restrict__ perm, int64_t N, const T* __restrict__ dLdV, double dLdE,
                           T* __restrict__ out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    uint32_t i = perm[k];
    T ax = 0, ay = 0, az = 0;
    if (dLdV) {
        T gk = dLdV[i];
        uint32_t st = face_start[k];
        int cnt = face_count[k];
        for (int q = 0; q < cnt; q++) {
            Face f = faces[st + q];
            T gj = dLdV[perm[f.nbr]];
            T r = sqrt((T)f.dx * f.dx + (T)f.dy * f.dy + (T)f.dz * f.dz);
            T wgt = (T)f.area / r * (gk - gj);
            ax += wgt * (T)f.cx; ay += wgt * (T)f.cy; az += wgt * (T)f.cz;
        }
    }
    if (dLdE != 0.0) {
        CellOut co = cell[k];
        T s = (T)(-2.0 * dLdE * co.vol);
        ax += s * (T)co.zx; ay += s * (T)co.zy; az += s * (T)co.zz;
    }
    out[3 * (int64_t)i + 0] = ax;
    out[3 * (int64_t)i + 1] = ay;
    out[3 * (int64_t)i + 2] = az;
}

void launch_backward(const Face* faces, const uint32_t* face_start, const uint16_t* face_count, const CellOut* cell,
                     const void* spos, int dtype, const uint32_t* perm, const uint32_t* inv, int64_t N,
                     const void* dLdV, double dLdE, void* out, cudaStream_t s) {
    (void)spos; (void)inv;
    unsigned nb = (unsigned)((N + 255) / 256);
    if (dtype == VT_F32)
        k_backward<float><<<nb, 256, 0, s>>>(faces, face_start, face_count, cell, perm, N, (const float*)dLdV, dLdE,
                                             (float*)out);
    else
        k_backward<double><<<nb, 256, 0, s>>>(faces, face_start, face_count, cell, perm, N, (const double*)dLdV, dLdE,
                                              (double*)out);
}

}  // namespace vt
