// vt_sort.cu -- wrap/validate + Morton key, LSD radix sort, gather into sorted order,
// and the bucket tree used for candidate search (hot-path steps A1-A2).
//
// The paper distributes particles over MPI tasks by a spatial decomposition and
// exchanges boundary particles (Implementation section); on one GPU the same
// locality comes from sorting the particles along a Morton curve: cells that
// are processed together are near each other, and the sorted order defines a
// 32-ary tree of bounding boxes (buckets of 32 consecutive particles) that
// answers "all particles within radius r" for any local density.
#include <cuda_runtime.h>
#include <stdint.h>

#include "vt_internal.cuh"
#include "vt_kernels.cuh"

namespace vt {

// ---------------------------------------------------------------- keys
__device__ __forceinline__ uint64_t spread3_16(uint32_t v) {
    uint64_t x = v & 0xFFFFu;
    x = (x | (x << 16)) & 0x0000FF0000FFull;
    x = (x | (x << 8)) & 0x00F00F00F00Full;
    x = (x | (x << 4)) & 0x0C30C30C30C3ull;
    x = (x | (x << 2)) & 0x249249249249ull;
    return x;
}

// x in the box: periodic [lo, hi), bounded [lo, hi]; false for NaN.  FP32 inputs against a box whose ends are
// FP32 numbers compare exactly in FP32 (no FP64 on the path, which runs at 1/64 of the FP32 rate).
template <typename T>
__device__ __forceinline__ bool in_box(T x, const Geometry& g, int c) {
    if (sizeof(T) == 4 && g.box_f32) {
        const float xf = (float)x;
        return g.periodic ? (xf >= g.lof[c] && xf < g.hif[c]) : (xf >= g.lof[c] && xf <= g.hif[c]);
    }
    const double xd = (double)x;
    return g.periodic ? (xd >= g.lo[c] && xd < g.hi[c]) : (xd >= g.lo[c] && xd <= g.hi[c]);
}

template <typename T>
__global__ void k_key(const T* __restrict__ pos, int64_t N, Geometry g, uint64_t* __restrict__ key,
                      uint32_t* __restrict__ idx, DevStatus* st) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    uint32_t q[3];
    bool bad = false;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const T x = pos[3 * i + c];
        const bool ok = in_box<T>(x, g, c);
        if (!ok) bad = true;  // also catches NaN
        // the key only orders the particles: FP32 suffices (the index is clamped below)
        const float t = ((float)x - g.lof[c]) * g.qs[c];
        int qi = ok ? (int)t : 0;
        q[c] = (uint32_t)min(max(qi, 0), 65535);
    }
    if (bad) {
        atomicAdd(&st->invalid_input, 1u);
        atomicCAS(&st->error, 0, VT_ERR_INVALID);
    }
    key[i] = spread3_16(q[0]) | (spread3_16(q[1]) << 1) | (spread3_16(q[2]) << 2);
    idx[i] = (uint32_t)i;
}

// batched sets: key = set << 48 | Morton code of the position quantised in the set's own box
template <typename T>
__global__ void k_key_batched(const T* __restrict__ pos, int64_t N, const Geometry* __restrict__ sgeo,
                              const uint32_t* __restrict__ setid, uint64_t* __restrict__ key,
                              uint32_t* __restrict__ idx, DevStatus* st) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint32_t s = setid[i];
    const Geometry& g = sgeo[s];
    uint32_t q[3];
    bool bad = false;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const T x = pos[3 * i + c];
        const bool ok = in_box<T>(x, g, c);
        if (!ok) bad = true;
        // the key only orders the particles: FP32 suffices (the index is clamped below)
        const float t = ((float)x - g.lof[c]) * g.qs[c];
        int qi = ok ? (int)t : 0;
        q[c] = (uint32_t)min(max(qi, 0), 65535);
    }
    if (bad) {
        atomicAdd(&st->invalid_input, 1u);
        atomicCAS(&st->error, 0, VT_ERR_INVALID);
    }
    key[i] = ((uint64_t)s << 48) | spread3_16(q[0]) | (spread3_16(q[1]) << 1) | (spread3_16(q[2]) << 2);
    idx[i] = (uint32_t)i;
}

// set of every particle from the set offsets (binary search)
__global__ void k_set_ids(const int64_t* __restrict__ soff, int n_sets, int64_t N, uint32_t* __restrict__ setid) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int lo = 0, hi = n_sets;  // soff[lo] <= i < soff[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (soff[mid] <= i) lo = mid;
        else hi = mid;
    }
    setid[i] = (uint32_t)lo;
}

__global__ void k_gather_u32(const uint32_t* __restrict__ src, const uint32_t* __restrict__ perm, int64_t N,
                             uint32_t* __restrict__ dst) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N) dst[k] = src[perm[k]];
}

int launch_key_batched(const void* pos, int dtype, int64_t N, const Geometry* sgeo, const uint32_t* setid,
                       uint64_t* key, uint32_t* idx, DevStatus* st, cudaStream_t s) {
    unsigned nb = (unsigned)((N + 255) / 256);
    if (dtype == VT_F32)
        k_key_batched<float><<<nb, 256, 0, s>>>((const float*)pos, N, sgeo, setid, key, idx, st);
    else
        k_key_batched<double><<<nb, 256, 0, s>>>((const double*)pos, N, sgeo, setid, key, idx, st);
    return 1;
}
int launch_set_ids(const int64_t* soff, int n_sets, int64_t N, uint32_t* setid, cudaStream_t s) {
    k_set_ids<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(soff, n_sets, N, setid);
    return 1;
}
int launch_gather_u32(const uint32_t* src, const uint32_t* perm, int64_t N, uint32_t* dst, cudaStream_t s) {
    k_gather_u32<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(src, perm, N, dst);
    return 1;
}

// the sorted indices of the owned particles (input rows 0 .. n_owned-1) as the clipping kernel's cell list, and
// its length
__global__ void k_owned_list(const uint32_t* __restrict__ inv, int64_t n_owned, uint32_t* __restrict__ list,
                             DevStatus* st) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n_owned) list[k] = inv[k];
    if (k == 0) st->n_warp_cells = (unsigned)n_owned;
}
int launch_owned_list(const uint32_t* inv, int64_t n_owned, uint32_t* list, DevStatus* st, cudaStream_t s) {
    k_owned_list<<<(unsigned)((n_owned + 255) / 256), 256, 0, s>>>(inv, n_owned, list, st);
    return 1;
}

// ---------------------------------------------------------------- scan
// exclusive scan, blocks of 1024 threads x 4 items, recursive over block sums
template <typename TI, typename TO>
__global__ void k_scan_block(const TI* __restrict__ in, TO* __restrict__ out, int64_t n, TO* __restrict__ partial) {
    __shared__ TO wsum[32];
    int64_t base = (int64_t)blockIdx.x * 4096 + threadIdx.x * 4;
    TO v[4];
    TO s = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        v[k] = (base + k < n) ? (TO)in[base + k] : (TO)0;
        s += v[k];
    }
    // inclusive warp scan of s
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    TO x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        TO y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        TO t = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            TO y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wsum[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    TO excl = x - s + (w > 0 ? wsum[w - 1] : (TO)0);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if (base + k < n) out[base + k] = excl;
        excl += v[k];
    }
    if (threadIdx.x == 1023 && partial) partial[blockIdx.x] = wsum[31];
}

template <typename TO>
__global__ void k_scan_add(TO* __restrict__ out, int64_t n, const TO* __restrict__ partial_scanned) {
    int64_t i = (int64_t)blockIdx.x * 4096 + threadIdx.x * 4;
    TO a = partial_scanned[blockIdx.x];
#pragma unroll
    for (int k = 0; k < 4; k++)
        if (i + k < n) out[i + k] += a;
}

size_t scan_tmp_bytes(int64_t n) {
    size_t b = 0;
    while (n > 4096) {
        n = (n + 4095) / 4096;
        b += (size_t)(n + 1) * 8;
    }
    return b + 64;
}

template <typename TI, typename TO>
static int scan_rec(const TI* in, TO* out, int64_t n, char* tmp, cudaStream_t s) {
    int64_t nb = (n + 4095) / 4096;
    if (nb <= 1) {
        k_scan_block<TI, TO><<<1, 1024, 0, s>>>(in, out, n, (TO*)nullptr);
        return 1;
    }
    TO* part = (TO*)tmp;
    char* rest = tmp + ((nb + 1) * sizeof(TO) + 15) / 16 * 16;
    k_scan_block<TI, TO><<<(unsigned)nb, 1024, 0, s>>>(in, out, n, part);
    int k = scan_rec<TO, TO>(part, part, nb, rest, s);
    k_scan_add<TO><<<(unsigned)nb, 1024, 0, s>>>(out, n, part);
    return k + 2;
}

int scan_u32_u32(const uint32_t* in, uint32_t* out, int64_t n, void* tmp, cudaStream_t s) {
    return scan_rec<uint32_t, uint32_t>(in, out, n, (char*)tmp, s);
}
int scan_u16_i64(const uint16_t* in, int64_t* out, int64_t n, void* tmp, cudaStream_t s) {
    return scan_rec<uint16_t, int64_t>(in, out, n, (char*)tmp, s);
}

// ---------------------------------------------------------------- radix sort
constexpr int RS_WARPS = 8;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_WARPS * RS_ROUNDS * 32;  // 4096
constexpr int RS_SMEM = RS_TILE * (8 + 4);             // staged tile: keys and values

__global__ void __launch_bounds__(256) k_radix_hist(const uint64_t* __restrict__ key, int64_t N, int shift,
                                                    uint32_t* __restrict__ hist, int nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int k = threadIdx.x; k < RS_TILE; k += 256) {
        int64_t i = base + k;
        if (i < N) atomicAdd(&h[(key[i] >> shift) & 255], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Scatter of one tile: every key's rank within its digit (per warp, then over the warps) gives its position in
// the tile reordered by digit; the tile is staged in that order in shared memory and written out position by
// position, so that consecutive threads write consecutive addresses of one digit's run (coalesced stores)
// instead of up to 32 digit buckets per warp.  Dynamic shared memory: RS_TILE keys and values.
__global__ void __launch_bounds__(256) k_radix_scatter(const uint64_t* __restrict__ key, const uint32_t* __restrict__ val,
                                                       uint64_t* __restrict__ key_out, uint32_t* __restrict__ val_out,
                                                       int64_t N, int shift, const uint32_t* __restrict__ goff,
                                                       int nblocks) {
    extern __shared__ __align__(16) unsigned char rs_smem[];
    uint64_t* skey = reinterpret_cast<uint64_t*>(rs_smem);
    uint32_t* sval = reinterpret_cast<uint32_t*>(skey + RS_TILE);
    __shared__ uint32_t cnt[RS_WARPS][256];
    __shared__ uint32_t boff[256];   // start of each digit in the reordered tile
    __shared__ uint32_t wsum[RS_WARPS];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < RS_WARPS * 256; k += 256) (&cnt[0][0])[k] = 0;
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * RS_TILE;
    int64_t base = tile0 + (int64_t)w * RS_ROUNDS * 32;
    uint64_t kk[RS_ROUNDS];
    uint32_t vv[RS_ROUNDS];
    uint32_t rk[RS_ROUNDS];
    unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; r++) {
        int64_t i = base + r * 32 + lane;
        bool valid = i < N;
        kk[r] = valid ? key[i] : 0ull;
        vv[r] = valid ? val[i] : 0u;
        uint32_t d = valid ? (uint32_t)((kk[r] >> shift) & 255) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = (d < 256) ? cnt[w][d] : 0u;
        rk[r] = before + __popc(peers & lt);
        __syncwarp();
        int leader = __ffs(peers) - 1;
        if (lane == leader && d < 256) cnt[w][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over the warps, and the digit's total in the tile
    uint32_t total = 0;
    {
        int d = threadIdx.x;
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ww++) {
            uint32_t c = cnt[ww][d];
            cnt[ww][d] = total;
            total += c;
        }
    }
    // exclusive scan of the digit totals over the block (thread d holds digit d)
    {
        uint32_t x = total;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        uint32_t add = 0;
        for (int ww = 0; ww < w; ww++) add += wsum[ww];
        boff[threadIdx.x] = add + x - total;
    }
    __syncthreads();
    // stage the tile in digit order
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; r++) {
        int64_t i = base + r * 32 + lane;
        if (i < N) {
            uint32_t d = (uint32_t)((kk[r] >> shift) & 255);
            uint32_t lp = boff[d] + cnt[w][d] + rk[r];
            skey[lp] = kk[r];
            sval[lp] = vv[r];
        }
    }
    __syncthreads();
    // write out: position t of the reordered tile goes to its digit's run in the global order
    const int n = (int)min((int64_t)RS_TILE, N - tile0);
    for (int t = threadIdx.x; t < n; t += 256) {
        const uint64_t k2 = skey[t];
        const uint32_t d = (uint32_t)((k2 >> shift) & 255);
        const uint32_t p = goff[(int64_t)d * nblocks + blockIdx.x] + ((uint32_t)t - boff[d]);
        key_out[p] = k2;
        val_out[p] = sval[t];
    }
}

size_t radix_tmp_bytes(int64_t N) {
    int64_t nb = (N + RS_TILE - 1) / RS_TILE;
    size_t h = (size_t)nb * 256;
    return 2 * h * sizeof(uint32_t) + scan_tmp_bytes((int64_t)h) + 256;
}

// sorts (key, val) by the low `bits` bits of key; the result ends in key/val
int radix_sort(uint64_t* key, uint32_t* val, uint64_t* key_alt, uint32_t* val_alt, int64_t N, int bits, void* tmp,
               cudaStream_t s) {
    int nb = (int)((N + RS_TILE - 1) / RS_TILE);
    if (nb == 0) return 0;
    int launches = 0;
    // the staged scatter uses more than the default 48 KB of dynamic shared memory (set once per device)
    static int smem_set[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !smem_set[dev]) {
        cudaFuncSetAttribute(k_radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, RS_SMEM);
        smem_set[dev] = 1;
    }
    uint32_t* hist = (uint32_t*)tmp;
    uint32_t* goff = hist + (size_t)nb * 256;
    void* stmp = goff + (size_t)nb * 256;
    uint64_t* ka = key;
    uint32_t* va = val;
    uint64_t* kb = key_alt;
    uint32_t* vb = val_alt;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        k_radix_hist<<<nb, 256, 0, s>>>(ka, N, shift, hist, nb);
        launches += 2 + scan_u32_u32(hist, goff, (int64_t)nb * 256, stmp, s);
        k_radix_scatter<<<nb, 256, RS_SMEM, s>>>(ka, va, kb, vb, N, shift, goff, nb);
        uint64_t* tk = ka; ka = kb; kb = tk;
        uint32_t* tv = va; va = vb; vb = tv;
    }
    if (ka != key) {
        cudaMemcpyAsync(key, ka, N * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(val, va, N * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    }
    return launches;
}

// ---------------------------------------------------------------- gather
template <typename T, typename P>
__global__ void k_gather(const T* __restrict__ pos, const T* __restrict__ mass, const uint32_t* __restrict__ perm,
                         int64_t N, P* __restrict__ spos, uint32_t* __restrict__ inv) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    uint32_t i = perm[k];
    P p;
    p.x = pos[3 * (int64_t)i + 0];
    p.y = pos[3 * (int64_t)i + 1];
    p.z = pos[3 * (int64_t)i + 2];
    p.w = mass ? mass[i] : (T)1;
    spos[k] = p;
    inv[i] = (uint32_t)k;
}

template __global__ void k_key<float>(const float*, int64_t, Geometry, uint64_t*, uint32_t*, DevStatus*);
template __global__ void k_key<double>(const double*, int64_t, Geometry, uint64_t*, uint32_t*, DevStatus*);

int launch_key(const void* pos, int dtype, int64_t N, const Geometry& g, uint64_t* key, uint32_t* idx, DevStatus* st,
               cudaStream_t s) {
    unsigned nb = (unsigned)((N + 255) / 256);
    if (dtype == VT_F32)
        k_key<float><<<nb, 256, 0, s>>>((const float*)pos, N, g, key, idx, st);
    else
        k_key<double><<<nb, 256, 0, s>>>((const double*)pos, N, g, key, idx, st);
    return 1;
}

int launch_gather(const void* pos, const void* mass, int dtype, const uint32_t* perm, int64_t N, void* spos,
                  uint32_t* inv, cudaStream_t s) {
    unsigned nb = (unsigned)((N + 255) / 256);
    if (dtype == VT_F32)
        k_gather<float, float4><<<nb, 256, 0, s>>>((const float*)pos, (const float*)mass, perm, N, (float4*)spos, inv);
    else
        k_gather<double, dpt4><<<nb, 256, 0, s>>>((const double*)pos, (const double*)mass, perm, N, (dpt4*)spos, inv);
    return 1;
}

// ---------------------------------------------------------------- tree
__device__ __forceinline__ float f_dn(double x) { return __double2float_rd(x); }
__device__ __forceinline__ float f_up(double x) { return __double2float_ru(x); }

template <typename P>
__global__ void k_tree_buckets(const P* __restrict__ spos, int64_t N, float4* __restrict__ lo, float4* __restrict__ hi,
                               int64_t nbuck) {
    int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (b >= nbuck) return;
    int64_t i = b * 32 + lane;
    float l0 = INFINITY, l1 = INFINITY, l2 = INFINITY, h0 = -INFINITY, h1 = -INFINITY, h2 = -INFINITY;
    if (i < N) {
        P p = spos[i];
        l0 = f_dn(p.x); l1 = f_dn(p.y); l2 = f_dn(p.z);
        h0 = f_up(p.x); h1 = f_up(p.y); h2 = f_up(p.z);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        l0 = fminf(l0, __shfl_xor_sync(0xffffffffu, l0, o));
        l1 = fminf(l1, __shfl_xor_sync(0xffffffffu, l1, o));
        l2 = fminf(l2, __shfl_xor_sync(0xffffffffu, l2, o));
        h0 = fmaxf(h0, __shfl_xor_sync(0xffffffffu, h0, o));
        h1 = fmaxf(h1, __shfl_xor_sync(0xffffffffu, h1, o));
        h2 = fmaxf(h2, __shfl_xor_sync(0xffffffffu, h2, o));
    }
    if (lane == 0) {
        lo[b] = make_float4(l0, l1, l2, 0.f);
        hi[b] = make_float4(h0, h1, h2, 0.f);
    }
}

__global__ void k_tree_level(const float4* __restrict__ clo, const float4* __restrict__ chi, int64_t nchild,
                             float4* __restrict__ lo, float4* __restrict__ hi, int64_t nnode) {
    int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (b >= nnode) return;
    int64_t c = b * 32 + lane;
    float4 l = make_float4(INFINITY, INFINITY, INFINITY, 0.f), h = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
    if (c < nchild) { l = clo[c]; h = chi[c]; }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        l.x = fminf(l.x, __shfl_xor_sync(0xffffffffu, l.x, o));
        l.y = fminf(l.y, __shfl_xor_sync(0xffffffffu, l.y, o));
        l.z = fminf(l.z, __shfl_xor_sync(0xffffffffu, l.z, o));
        h.x = fmaxf(h.x, __shfl_xor_sync(0xffffffffu, h.x, o));
        h.y = fmaxf(h.y, __shfl_xor_sync(0xffffffffu, h.y, o));
        h.z = fmaxf(h.z, __shfl_xor_sync(0xffffffffu, h.z, o));
    }
    if (lane == 0) { lo[b] = l; hi[b] = h; }
}

void tree_layout(int64_t N, Tree& t) {
    int64_t n = (N + 31) / 32;
    int64_t off = 0;
    t.levels = 0;
    for (int l = 1; l <= MAX_LEVELS; l++) {
        t.count[l] = n;
        t.off[l] = off;
        off += n;
        t.levels = l;
        if (n <= 32) break;
        n = (n + 31) / 32;
    }
    t.count[0] = N;
    t.off[0] = off;  // total node count
}

int launch_tree(const void* spos, int dtype, int64_t N, Tree& t, cudaStream_t s) {
    int64_t nb = t.count[1];
    unsigned g = (unsigned)((nb * 32 + 255) / 256);
    if (dtype == VT_F32)
        k_tree_buckets<float4><<<g, 256, 0, s>>>((const float4*)spos, N, t.lo + t.off[1], t.hi + t.off[1], nb);
    else
        k_tree_buckets<dpt4><<<g, 256, 0, s>>>((const dpt4*)spos, N, t.lo + t.off[1], t.hi + t.off[1], nb);
    for (int l = 2; l <= t.levels; l++) {
        int64_t nn = t.count[l];
        unsigned gg = (unsigned)((nn * 32 + 255) / 256);
        k_tree_level<<<gg, 256, 0, s>>>(t.lo + t.off[l - 1], t.hi + t.off[l - 1], t.count[l - 1], t.lo + t.off[l],
                                        t.hi + t.off[l], nn);
    }
    return t.levels;
}

}  // namespace vt
