// vt_api.cu -- the C ABI (see include/vt_gb300.h): handle, workspace, launch order, error reporting.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "vt_internal.cuh"
#include "vt_kernels.cuh"

using namespace vt;

namespace {

constexpr int RC_POOL_HOST = 1001;  // device code for "facet pool too small" (the host grows it)
constexpr unsigned GRID_RETRY_CAP = 1u << 20;  // (cell, voxel) pairs of the volume-averaged grid's second pass

// internal detail of the last failed vt_build on this thread (diagnostics)
thread_local int g_last_detail = 0;
thread_local int g_last_particle = -1;

// fault injection (vt_debug_fail_alloc): the number of handle allocations still to succeed before one fails
// (0: disarmed)
std::atomic<int> g_fail_alloc{0};

bool injected_failure() {
    int n = g_fail_alloc.load();
    while (n > 0) {
        if (g_fail_alloc.compare_exchange_weak(n, n - 1)) return n == 1;
    }
    return false;
}

// Handle workspaces come from a stream-ordered memory pool per device that the library owns: allocations and
// frees are ordered on the handle's stream (a free does not synchronise the device, so work of other streams,
// e.g. copies of a previous step's outputs, keeps running), and freed memory stays in the pool for the next
// build until vt_release_memory returns it.
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};

cudaMemPool_t device_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = ~0ull;  // keep freed memory for reuse
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = pool;
    }
    return g_pool[dev];
}

// one workspace allocation on the handle's stream from the device's pool (nullptr on failure)
void* pool_alloc(size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool = device_pool();
    void* p = nullptr;
    if (!pool || cudaMallocFromPoolAsync(&p, bytes, pool, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void pool_free(void* p, cudaStream_t s) {
    if (p && cudaFreeAsync(p, s) != cudaSuccess) cudaGetLastError();
}

struct Alloc {
    cudaStream_t s = nullptr;
    bool failed = false;
    template <typename T>
    T* get(size_t count) {
        if (count == 0) count = 1;
        if (injected_failure()) {
            failed = true;
            return nullptr;
        }
        void* p = pool_alloc(count * sizeof(T), s);
        if (!p) failed = true;
        return (T*)p;
    }
};

// Mapped pinned blocks for the status reads, one per live handle, kept for reuse (never returned to the system:
// a build does not pay for a pinned allocation).
std::mutex g_map_mu;
std::vector<DevStatus*> g_map_free;

DevStatus* map_take() {
    {
        std::lock_guard<std::mutex> lk(g_map_mu);
        if (!g_map_free.empty()) {
            DevStatus* p = g_map_free.back();
            g_map_free.pop_back();
            return p;
        }
    }
    void* p = nullptr;
    if (cudaHostAlloc(&p, sizeof(DevStatus), cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (DevStatus*)p;
}

void map_give(DevStatus* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_map_mu);
    g_map_free.push_back(p);
}

// give the kept blocks back to the system (those of live handles stay theirs)
void map_release() {
    std::lock_guard<std::mutex> lk(g_map_mu);
    for (DevStatus* p : g_map_free)
        if (cudaFreeHost(p) != cudaSuccess) cudaGetLastError();
    g_map_free.clear();
}

void free_handle(vt_handle h) {
    if (!h) return;
    for (int k = 0; k < 4; k++)
        if (h->ev[k]) cudaEventDestroy(h->ev[k]);
    void* ptrs[] = {h->spos, h->perm, h->inv, h->tree_mem, h->cell, h->face_start, h->face_count, h->cstat, h->rad,
                    h->exact_list, h->dens_sorted, h->faces, h->xws, h->tmp, h->nbr_off_cache, h->dstat,
                    h->keys, h->keys_alt, h->vals_alt, h->cnt_in, h->sset, h->sgeo, h->soff, h->set_in, h->warp_list,
                    h->set_cfg, h->gacc, h->gretry, h->gcnt};
    for (void* p : ptrs)
        if (p) pool_free(p, h->stream);
    map_give(h->smap);
    delete h;
}

// threads per cell -> the clipping kernels' mode (ClipArgs): 32 -> 0, 1 -> 1, 4 -> 2, 8 -> 3; -1 if unsupported
int tpc_mode_of(int tpc) {
    return tpc == 32 ? 0 : tpc == 1 ? 1 : tpc == 4 ? 2 : tpc == 8 ? 3 : -1;
}

int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return VT_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? VT_ERR_OOM : VT_ERR_CUDA;
}

// Status words reach the host through mapped pinned memory: one small block copies them there, and the host reads them
// after synchronising the handle's stream.  No copy engine takes part, so a status read never waits behind large
// copies that other streams have in flight (e.g. a previous step's outputs going to the host).
static_assert(sizeof(DevStatus) % 4 == 0, "status words are copied as 32-bit words");
__global__ void k_status_copy(const DevStatus* src, DevStatus* dst) {
    const unsigned* a = (const unsigned*)src;
    unsigned* b = (unsigned*)dst;
    for (int k = (int)threadIdx.x; k < (int)(sizeof(DevStatus) / 4); k += blockDim.x) b[k] = a[k];
}
// clear every status word, then set the input-validation count and the error to the given values
__global__ void k_status_reset(DevStatus* st, unsigned invalid_input, int error) {
    unsigned* w = (unsigned*)st;
    for (int k = (int)threadIdx.x; k < (int)(sizeof(DevStatus) / 4); k += blockDim.x) w[k] = 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
        st->invalid_input = invalid_input;
        st->error = error;
    }
}

// the handle's status words as they stand after its stream's work so far (synchronises the stream)
int read_status(vt_handle h, DevStatus* out) {
    DevStatus* dmap = nullptr;
    if (cudaHostGetDevicePointer((void**)&dmap, h->smap, 0) != cudaSuccess) {
        cudaGetLastError();
        return VT_ERR_CUDA;
    }
    k_status_copy<<<1, 128, 0, h->stream>>>(h->dstat, dmap);
    h->n_launches += 1;
    int rc = cuda_rc(cudaGetLastError());
    if (!rc) rc = cuda_rc(cudaStreamSynchronize(h->stream));
    if (!rc) memcpy(out, (const void*)h->smap, sizeof(DevStatus));
    return rc;
}

ClipArgs clip_args(vt_handle h) {
    ClipArgs a;
    a.spos = h->spos;
    a.N = h->N;
    a.geo = h->geo;
    a.tree = h->tree;
    a.k_target = h->prm.k_target;
    a.max_passes = h->prm.max_passes;
    a.radius_policy = h->prm.reserved[0];
    a.cell = h->cell;
    a.face_start = h->face_start;
    a.face_count = h->face_count;
    a.cstat = h->cstat;
    a.exact_list = h->exact_list;
    a.faces = h->faces;
    a.face_cap = h->face_cap;
    a.st = h->dstat;
    a.xws = h->xws;
    a.xws_warps = h->xws_warps;
    a.sset = h->sset;
    a.sgeo = h->sgeo;
    a.soff = h->soff;
    // another kernel first (thread per cell, or a lane group) when some cell takes a mode other than the warp's
    const bool thread_first = (h->modes & ~1) != 0;
    a.list_given = h->n_owned < h->N;
    a.warp_list = (thread_first || a.list_given) ? h->warp_list : nullptr;
    a.set_cfg = h->set_cfg;
    a.tpc_mode = h->prm.precision == VT_FILTER32 ? tpc_mode_of(h->prm.threads_per_cell) : 0;
    a.modes = h->modes;
    a.rad = h->rad;
    return a;
}

// a build over owned and ghost particles: the cells of the ghosts are not computed (volume 0, no facets), and
// the clipping kernel takes its cells from the list of the owned ones
int enqueue_owned(vt_handle h) {
    if (h->n_owned >= h->N) return VT_OK;
    cudaStream_t s = h->stream;
    int rc = cuda_rc(cudaMemsetAsync(h->cell, 0, (size_t)h->N * sizeof(CellOut), s));
    if (!rc) rc = cuda_rc(cudaMemsetAsync(h->face_count, 0, (size_t)h->N * sizeof(uint16_t), s));
    if (!rc) rc = cuda_rc(cudaMemsetAsync(h->rad, 0, (size_t)h->N * sizeof(float), s));
    if (!rc) h->n_launches += launch_owned_list(h->inv, h->n_owned, h->warp_list, h->dstat, s);
    return rc;
}

int run_clip(vt_handle h) {
    cudaStream_t s = h->stream;
    for (int attempt = 0; attempt < 4; attempt++) {
        // reset the clipping counters (the input-validation count and the error as last read are kept)
        k_status_reset<<<1, 128, 0, s>>>(h->dstat, h->hstat.invalid_input, h->hstat.error);
        h->n_launches += 1;
        int rc = enqueue_owned(h);
        if (rc) return rc;
        ClipArgs a = clip_args(h);
        cudaEventRecord(h->ev[2], s);
        h->n_launches += launch_clip(a, h->dtype, h->precision, h->sm_count, s);
        h->n_launches += launch_clip_exact(a, h->dtype, h->sm_count, s);
        cudaEventRecord(h->ev[3], s);
        rc = cuda_rc(cudaGetLastError());
        if (rc) return rc;
        rc = read_status(h, &h->hstat);
        if (rc) return rc;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]) == cudaSuccess) h->t_clip_ms = ms;
        if (h->hstat.error != RC_POOL_HOST) return h->hstat.error;
        // facet pool too small: grow it and redo the cells
        uint64_t need = h->hstat.face_next + (uint64_t)h->N * 4;
        uint64_t cap = h->face_cap * 2 > need ? h->face_cap * 2 : need;
        if (cap > 0xF0000000ull) return VT_ERR_CAPACITY;
        pool_free(h->faces, s);
        h->faces = (Face*)pool_alloc(cap * sizeof(Face), s);
        if (!h->faces) return VT_ERR_OOM;
        h->face_cap = cap;
        h->hstat.error = 0;
    }
    return VT_ERR_CAPACITY;
}

// the last neighbour offset = the facet count of the last clipping run
__global__ void k_off_tail(int64_t* p, const DevStatus* st) { *p = (int64_t)st->n_faces; }

int ensure_density(vt_handle h) {
    if (h->dens_ready) return VT_OK;
    h->n_launches += launch_density(h->cell, h->spos, h->dtype, h->perm, h->N, h->dens_sorted, nullptr, h->stream);
    h->dens_ready = 1;
    return cuda_rc(cudaGetLastError());
}

}  // namespace

extern "C" {

int vt_default_params(vt_params* p) {
    if (!p) return VT_ERR_INVALID;
    memset(p, 0, sizeof(*p));
    p->precision = VT_FILTER32;
    p->k_target = 24;
    p->reserved[0] = 1;
    p->max_passes = 1000;
    p->face_pool = 24;
    return VT_OK;
}

}  // extern "C"

namespace {

int check_params(const vt_params* p, vt_params& prm) {
    vt_default_params(&prm);
    if (p) prm = *p;
    if (prm.precision != VT_PLAIN64 && prm.precision != VT_FILTER32) return VT_ERR_INVALID;
    if (prm.reserved[0] < 0 || prm.reserved[0] > 1 || prm.reserved[1] || prm.reserved[2]) return VT_ERR_INVALID;
    if (prm.threads_per_cell == 0) prm.threads_per_cell = 32;
    if (tpc_mode_of(prm.threads_per_cell) < 0) return VT_ERR_INVALID;
    if (prm.k_target < 8 || prm.k_target > 120 || prm.max_passes < 1 || prm.max_passes > 100000 || prm.face_pool < 1 ||
        prm.face_pool > 128)
        return VT_ERR_INVALID;
    return VT_OK;
}

int make_geometry(const double* lo, const double* hi, int periodic, int precision, Geometry& geo) {
    memset(&geo, 0, sizeof(geo));
    for (int c = 0; c < 3; c++) {
        if (!(hi[c] > lo[c]) || !isfinite(lo[c]) || !isfinite(hi[c])) return VT_ERR_INVALID;
        geo.lo[c] = lo[c];
        geo.hi[c] = hi[c];
        geo.L[c] = hi[c] - lo[c];
        geo.qs[c] = (float)(65536.0 / geo.L[c]);
        geo.Lf[c] = (float)geo.L[c];
        geo.halfLf[c] = 0.5f * geo.Lf[c];
        geo.lof[c] = (float)lo[c];
        geo.hif[c] = (float)hi[c];
        if (precision == VT_FILTER32 && periodic && (double)geo.Lf[c] != geo.L[c]) return VT_ERR_UNSUPPORTED;
    }
    geo.periodic = periodic ? 1 : 0;
    geo.box_f32 = 1;
    for (int c = 0; c < 3; c++)
        if ((double)geo.lof[c] != geo.lo[c] || (double)geo.hif[c] != geo.hi[c]) geo.box_f32 = 0;
    return VT_OK;
}

// Key, sort, gather and tree of the positions `pos` into the handle's workspace (no allocation, no
// synchronisation).
void enqueue_sort_tree(vt_handle h, const void* pos, const void* mass) {
    cudaStream_t s = h->stream;
    const int64_t N = h->N;
    if (h->n_sets > 0) {
        // sort key = set id above the 48-bit Morton code of the set's own box: the sets stay contiguous
        // and in order, so set s occupies the same index range [set_off[s], set_off[s+1]) after sorting
        int sbits = 0;
        while ((1 << sbits) < h->n_sets) sbits++;
        h->n_launches += launch_key_batched(pos, h->dtype, N, h->sgeo, h->set_in, h->keys, h->perm, h->dstat, s);
        h->n_launches += radix_sort(h->keys, h->perm, h->keys_alt, h->vals_alt, N, 48 + sbits, h->tmp, s);
        h->n_launches += launch_gather_u32(h->set_in, h->perm, N, h->sset, s);
    } else {
        h->n_launches += launch_key(pos, h->dtype, N, h->geo, h->keys, h->perm, h->dstat, s);
        h->n_launches += radix_sort(h->keys, h->perm, h->keys_alt, h->vals_alt, N, 48, h->tmp, s);
    }
    h->n_launches += launch_gather(pos, mass, h->dtype, h->perm, N, h->spos, h->inv, s);
    h->n_launches += launch_tree(h->spos, h->dtype, N, h->tree, s);
}

// Shared by vt_build (n_sets == 0: one set, geometry `geo`) and vt_build_batched (n_sets >= 1: the host
// tables set_off [n_sets+1] and sgeo [n_sets]).
int build_impl(vt_handle* out, const void* pos, int dtype, const void* mass, int64_t N, const Geometry& geo,
               int n_sets, const int64_t* set_off, const Geometry* sgeo_host, const int32_t* cfg_host,
               const vt_params& prm, void* stream, int64_t n_owned = -1) {
    vt_handle h = new (std::nothrow) vt_handle_s;
    if (!h) return VT_ERR_OOM;
    memset(h, 0, sizeof(*h));
    h->N = N;
    h->n_owned = n_owned >= 0 && n_owned < N ? n_owned : N;
    h->dtype = dtype;
    h->precision = prm.precision;
    h->prm = prm;
    h->geo = geo;
    h->n_sets = n_sets;
    h->stream = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (h->sm_count <= 0) h->sm_count = 1;

    Alloc A;
    A.s = h->stream;
    size_t psz = dtype == VT_F32 ? sizeof(float4) : sizeof(dpt4);
    h->spos = A.get<unsigned char>(N * psz);
    h->keys = A.get<uint64_t>(N);
    h->keys_alt = A.get<uint64_t>(N);
    h->perm = A.get<uint32_t>(N);
    h->vals_alt = A.get<uint32_t>(N);
    h->inv = A.get<uint32_t>(N);
    tree_layout(N, h->tree);
    h->tree_mem = A.get<float4>(2 * h->tree.off[0]);
    h->tree.lo = h->tree_mem;
    h->tree.hi = h->tree_mem ? h->tree_mem + h->tree.off[0] : nullptr;
    h->cell = A.get<CellOut>(N);
    h->face_start = A.get<uint32_t>(N);
    h->face_count = A.get<uint16_t>(N);
    h->cnt_in = A.get<uint16_t>(N);
    h->cstat = A.get<uint8_t>(N);
    h->exact_list = A.get<uint32_t>(N);
    h->warp_list = A.get<uint32_t>(N);
    h->rad = A.get<float>(N);
    h->dens_sorted = A.get<double>(N);
    h->face_cap = (uint64_t)N * prm.face_pool;
    h->faces = A.get<Face>(h->face_cap);
    h->xws_warps = h->sm_count * 4;
    h->xws = A.get<double>((size_t)h->xws_warps * exact_ws_doubles_per_warp());
    size_t tb = radix_tmp_bytes(N);
    size_t sb = scan_tmp_bytes(N + 1);
    h->tmp_bytes = tb > sb ? tb : sb;
    h->tmp = A.get<unsigned char>(h->tmp_bytes);
    h->dstat = A.get<DevStatus>(1);
    h->smap = map_take();
    if (!h->smap) A.failed = true;
    if (n_sets > 0) {
        h->sset = A.get<uint32_t>(N);
        h->set_in = A.get<uint32_t>(N);
        h->sgeo = A.get<Geometry>(n_sets);
        h->soff = A.get<int64_t>(n_sets + 1);
        if (cfg_host) h->set_cfg = A.get<int32_t>(n_sets);
    }
    // the threads-per-cell modes present: each set's, or the handle's
    if (cfg_host) {
        for (int k = 0; k < n_sets; k++)
            if (set_off[k + 1] > set_off[k]) h->modes |= 1 << ((cfg_host[k] >> 16) & 3);
    } else {
        h->modes = 1 << (prm.precision == VT_FILTER32 ? tpc_mode_of(prm.threads_per_cell) : 0);
    }
    for (int k = 0; k < 4; k++)
        if (cudaEventCreate(&h->ev[k]) != cudaSuccess) {
            cudaGetLastError();
            h->ev[k] = nullptr;
            A.failed = true;
        }
    if (A.failed) {
        free_handle(h);
        return VT_ERR_OOM;
    }
    cudaStream_t s = h->stream;
    memset(&h->hstat, 0, sizeof(h->hstat));
    int rc = cuda_rc(cudaMemsetAsync(h->dstat, 0, sizeof(DevStatus), s));
    if (!rc && n_sets > 0) {
        rc = cuda_rc(cudaMemcpyAsync(h->sgeo, sgeo_host, n_sets * sizeof(Geometry), cudaMemcpyHostToDevice, s));
        if (!rc)
            rc = cuda_rc(cudaMemcpyAsync(h->soff, set_off, (n_sets + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        if (!rc && cfg_host)
            rc = cuda_rc(cudaMemcpyAsync(h->set_cfg, cfg_host, n_sets * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    }
    if (!rc) {
        cudaEventRecord(h->ev[0], s);
        if (n_sets > 0) h->n_launches += launch_set_ids(h->soff, n_sets, N, h->set_in, s);
        enqueue_sort_tree(h, pos, mass);
        cudaEventRecord(h->ev[1], s);
        rc = cuda_rc(cudaGetLastError());
    }
    if (!rc) rc = read_status(h, &h->hstat);
    if (!rc) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]) == cudaSuccess) h->t_sort_ms = ms;
    }
    if (!rc && h->hstat.invalid_input) rc = VT_ERR_INVALID;
    if (!rc) rc = run_clip(h);
    if (rc) {
        g_last_detail = h->hstat.error_detail;
        g_last_particle = -1;
        if (h->hstat.error && h->hstat.error_cell >= 0 && h->hstat.error_cell < N && h->perm) {
            uint32_t pi = 0;
            if (cudaMemcpy(&pi, h->perm + h->hstat.error_cell, sizeof(pi), cudaMemcpyDeviceToHost) == cudaSuccess)
                g_last_particle = (int)pi;
        }
        free_handle(h);
        return rc;
    }
    g_last_detail = 0;
    g_last_particle = -1;
    h->n_faces = (int64_t)h->hstat.n_faces;
    *out = h;
    return VT_OK;
}

}  // namespace

extern "C" {

int vt_build(vt_handle* out, const void* pos, int dtype, const void* mass, int64_t N, const double box_lo[3],
             const double box_hi[3], int periodic, const vt_params* p, void* stream) {
    if (!out) return VT_ERR_INVALID;
    *out = nullptr;
    if (!pos || !box_lo || !box_hi || N < 1 || N > 0x7FFFFFFF / 2) return VT_ERR_INVALID;
    if (dtype != VT_F32 && dtype != VT_F64) return VT_ERR_INVALID;
    vt_params prm;
    int rc = check_params(p, prm);
    if (rc) return rc;
    Geometry geo;
    rc = make_geometry(box_lo, box_hi, periodic, prm.precision, geo);
    if (rc) return rc;
    return build_impl(out, pos, dtype, mass, N, geo, 0, nullptr, nullptr, nullptr, prm, stream);
}

int vt_build_owned(vt_handle* out, const void* pos, int dtype, const void* mass, int64_t N, int64_t n_owned,
                   const double box_lo[3], const double box_hi[3], int periodic, const vt_params* p, void* stream) {
    if (!out) return VT_ERR_INVALID;
    *out = nullptr;
    if (!pos || !box_lo || !box_hi || N < 1 || N > 0x7FFFFFFF / 2 || n_owned < 1 || n_owned > N) return VT_ERR_INVALID;
    if (dtype != VT_F32 && dtype != VT_F64) return VT_ERR_INVALID;
    vt_params prm;
    int rc = check_params(p, prm);
    if (rc) return rc;
    prm.threads_per_cell = 32;  // the listed cells go to the warp kernel
    Geometry geo;
    rc = make_geometry(box_lo, box_hi, periodic, prm.precision, geo);
    if (rc) return rc;
    return build_impl(out, pos, dtype, mass, N, geo, 0, nullptr, nullptr, nullptr, prm, stream, n_owned);
}

int vt_build_batched(vt_handle* out, const void* pos, int dtype, const void* mass, const int64_t* set_off, int n_sets,
                     const double* boxes, const int32_t* set_k, const int32_t* set_tpc, const vt_params* p,
                     void* stream) {
    if (!out) return VT_ERR_INVALID;
    *out = nullptr;
    if (!pos || !set_off || !boxes || n_sets < 1 || n_sets > VT_MAX_SETS) return VT_ERR_INVALID;
    if (dtype != VT_F32 && dtype != VT_F64) return VT_ERR_INVALID;
    if (set_off[0] != 0) return VT_ERR_INVALID;
    for (int k = 0; k < n_sets; k++)
        if (set_off[k + 1] < set_off[k]) return VT_ERR_INVALID;
    const int64_t N = set_off[n_sets];
    if (N < 1 || N > 0x7FFFFFFF / 2) return VT_ERR_INVALID;
    vt_params prm;
    int rc = check_params(p, prm);
    if (rc) return rc;
    Geometry* sg = new (std::nothrow) Geometry[n_sets];
    int32_t* cfg = (set_k || set_tpc) ? new (std::nothrow) int32_t[n_sets] : nullptr;
    if (!sg || ((set_k || set_tpc) && !cfg)) {
        delete[] sg;
        delete[] cfg;
        return VT_ERR_OOM;
    }
    for (int k = 0; k < n_sets && !rc; k++) rc = make_geometry(boxes + 6 * k, boxes + 6 * k + 3, 0, prm.precision, sg[k]);
    for (int k = 0; cfg && k < n_sets && !rc; k++) {
        const int kt = set_k ? set_k[k] : prm.k_target;
        const int tpc = set_tpc ? (set_tpc[k] ? set_tpc[k] : 32) : prm.threads_per_cell;
        if (kt < 8 || kt > 120 || tpc_mode_of(tpc) < 0) rc = VT_ERR_INVALID;
        // the thread-per-cell and lane-group kernels exist for the FP32 filter only
        cfg[k] = kt | (prm.precision == VT_FILTER32 && tpc_mode_of(tpc) > 0 ? tpc_mode_of(tpc) << 16 : 0);
    }
    if (!rc) rc = build_impl(out, pos, dtype, mass, N, sg[0], n_sets, set_off, sg, cfg, prm, stream);
    delete[] sg;
    delete[] cfg;
    return rc;
}

int vt_autotune_batched(const void* pos, int dtype, const int64_t* set_off, int n_sets, const double* boxes,
                        const vt_params* p, int64_t sample, int32_t* k_out, int32_t* tpc_out, void* stream) {
    if (!pos || !set_off || !boxes || !k_out || !tpc_out || n_sets < 1 || n_sets > VT_MAX_SETS) return VT_ERR_INVALID;
    if (dtype != VT_F32 && dtype != VT_F64) return VT_ERR_INVALID;
    if (set_off[0] != 0) return VT_ERR_INVALID;
    for (int k = 0; k < n_sets; k++)
        if (set_off[k + 1] < set_off[k]) return VT_ERR_INVALID;
    if (set_off[n_sets] < 1 || set_off[n_sets] > 0x7FFFFFFF / 2) return VT_ERR_INVALID;
    vt_params prm;
    int rc = check_params(p, prm);
    if (rc) return rc;
    if (sample <= 0) sample = 262144;
    if (sample < 1024) sample = 1024;
    static const int ks[5] = {16, 24, 32, 48, 64};
    const int tpcs[4] = {32, 1, 4, 8};
    const int n_tpc = prm.precision == VT_FILTER32 ? 4 : 1;
    const size_t row = (dtype == VT_F32 ? sizeof(float) : sizeof(double)) * 3;
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < n_sets; k++) {
        k_out[k] = prm.k_target;
        tpc_out[k] = 32;
    }
    int* pick = new (std::nothrow) int[n_sets];
    int64_t* soff = new (std::nothrow) int64_t[n_sets + 1];
    double* sbox = new (std::nothrow) double[6 * (size_t)n_sets];
    Geometry* sg = new (std::nothrow) Geometry[n_sets];
    if (!pick || !soff || !sbox || !sg) rc = VT_ERR_OOM;
    // size classes [2^c, 2^(c+1))
    for (int c = 0; c < 31 && !rc; c++) {
        int64_t npts = 0;
        int nin = 0;
        for (int k = 0; k < n_sets; k++) {
            const int64_t n = set_off[k + 1] - set_off[k];
            if (n >= ((int64_t)1 << c) && n < ((int64_t)2 << c)) { npts += n; nin++; }
        }
        if (nin == 0) continue;
        // sample: whole sets spread evenly through the class, about `sample` points
        const int64_t stride = npts > sample ? (npts + sample - 1) / sample : 1;
        int np = 0, seen = 0;
        int64_t tot = 0;
        soff[0] = 0;
        for (int k = 0; k < n_sets; k++) {
            const int64_t n = set_off[k + 1] - set_off[k];
            if (!(n >= ((int64_t)1 << c) && n < ((int64_t)2 << c))) continue;
            if (seen++ % stride) continue;
            pick[np] = k;
            tot += n;
            soff[np + 1] = tot;
            for (int q = 0; q < 6; q++) sbox[6 * np + q] = boxes[6 * k + q];
            np++;
        }
        void* buf = nullptr;
        if (cudaMalloc(&buf, (size_t)tot * row) != cudaSuccess) {
            cudaGetLastError();
            rc = VT_ERR_OOM;
            break;
        }
        for (int q = 0; q < np && !rc; q++) {
            const int k = pick[q];
            rc = cuda_rc(cudaMemcpyAsync((char*)buf + soff[q] * row, (const char*)pos + set_off[k] * row,
                                         (size_t)(set_off[k + 1] - set_off[k]) * row, cudaMemcpyDeviceToDevice, s));
        }
        for (int q = 0; q < np && !rc; q++) rc = make_geometry(sbox + 6 * q, sbox + 6 * q + 3, 0, prm.precision, sg[q]);
        // one untimed build, then every configuration; the clipping time decides
        double best = 1e300;
        int bk = prm.k_target, bt = 32, last_err = VT_OK;
        for (int trial = -1; trial < 5 * n_tpc && !rc; trial++) {
            vt_params t = prm;
            if (trial >= 0) {
                t.k_target = ks[trial % 5];
                t.threads_per_cell = tpcs[trial / 5];
            }
            vt_handle h = nullptr;
            const int e = build_impl(&h, buf, dtype, nullptr, tot, sg[0], np, soff, sg, nullptr, t, stream);
            if (e) {
                last_err = e;
                continue;
            }
            const double ms = h->t_clip_ms;
            cudaStreamSynchronize(h->stream);
            free_handle(h);
            if (trial >= 0 && ms < best) {
                best = ms;
                bk = t.k_target;
                bt = t.threads_per_cell;
            }
        }
        cudaFree(buf);
        if (!rc && best == 1e300) rc = last_err ? last_err : VT_ERR_CUDA;
        for (int k = 0; k < n_sets && !rc; k++) {
            const int64_t n = set_off[k + 1] - set_off[k];
            if (n >= ((int64_t)1 << c) && n < ((int64_t)2 << c)) {
                k_out[k] = bk;
                tpc_out[k] = bt;
            }
        }
    }
    delete[] pick;
    delete[] soff;
    delete[] sbox;
    delete[] sg;
    return rc;
}

int vt_rebuild(vt_handle h, const void* pos, const void* mass) {
    if (!h || !pos) return VT_ERR_INVALID;
    cudaStream_t s = h->stream;
    // every counter, the work queues and the sticky error start at zero
    int rc = cuda_rc(cudaMemsetAsync(h->dstat, 0, sizeof(DevStatus), s));
    if (rc) return rc;
    enqueue_sort_tree(h, pos, mass);
    rc = enqueue_owned(h);
    if (rc) return rc;
    ClipArgs a = clip_args(h);
    h->n_launches += launch_clip(a, h->dtype, h->precision, h->sm_count, s);
    h->n_launches += launch_clip_exact(a, h->dtype, h->sm_count, s);
    h->dens_ready = 0;
    h->faces_on_device = 1;
    return cuda_rc(cudaGetLastError());
}

int vt_cells(vt_handle h, void* vol, int64_t* nbr_off, int32_t* nbr_id, int64_t* n_faces_out) {
    if (!h) return VT_ERR_INVALID;
    cudaStream_t s = h->stream;
    if (n_faces_out) {
        if (h->faces_on_device) {
            // once the handle has been rebuilt (perhaps by a replayed graph) the count is read from the device
            int rc = read_status(h, &h->hstat);
            if (rc) return rc;
            h->n_faces = (int64_t)h->hstat.n_faces;
        }
        *n_faces_out = h->n_faces;
    }
    if (vol) h->n_launches += launch_out_vol(h->cell, h->perm, h->N, vol, h->dtype, s);
    if (nbr_off || nbr_id) {
        int64_t* off = nbr_off;
        if (!off) {
            if (!h->nbr_off_cache) {
                h->nbr_off_cache = (int64_t*)pool_alloc((h->N + 1) * sizeof(int64_t), s);
                if (!h->nbr_off_cache) return VT_ERR_OOM;
            }
            off = h->nbr_off_cache;
        }
        h->n_launches += launch_nbr_count(h->face_count, h->inv, h->N, h->cnt_in, s);
        h->n_launches += scan_u16_i64(h->cnt_in, off, h->N, h->tmp, s);
        k_off_tail<<<1, 1, 0, s>>>(off + h->N, h->dstat);
        h->n_launches += 1;
        if (nbr_id)
            h->n_launches += launch_nbr_emit(h->faces, h->face_start, h->face_count, h->perm, h->inv, off, h->N, nbr_id, s);
    }
    return cuda_rc(cudaGetLastError());
}

int vt_cell_radius(vt_handle h, void* rad) {
    if (!h || !rad) return VT_ERR_INVALID;
    h->n_launches += launch_out_rad(h->rad, h->perm, h->N, rad, h->dtype, h->stream);
    return cuda_rc(cudaGetLastError());
}

int vt_cell_flags(vt_handle h, uint8_t* flags) {
    if (!h || !flags) return VT_ERR_INVALID;
    h->n_launches += launch_cell_flags(h->cstat, h->perm, h->N, flags, h->stream);
    return cuda_rc(cudaGetLastError());
}

int vt_density(vt_handle h, void* dens) {
    if (!h || !dens) return VT_ERR_INVALID;
    h->n_launches += launch_density(h->cell, h->spos, h->dtype, h->perm, h->N, h->dens_sorted, dens, h->stream);
    h->dens_ready = 1;
    return cuda_rc(cudaGetLastError());
}

int vt_gradient(vt_handle h, void* grad) {
    if (!h || !grad) return VT_ERR_INVALID;
    int rc = ensure_density(h);
    if (rc) return rc;
    h->n_launches += launch_gradient(h->faces, h->face_start, h->face_count, h->dens_sorted, h->perm, h->N, grad, h->dtype, h->stream);
    return cuda_rc(cudaGetLastError());
}

int vt_gradient_gg(vt_handle h, void* grad) {
    if (!h || !grad) return VT_ERR_INVALID;
    int rc = ensure_density(h);
    if (rc) return rc;
    h->n_launches += launch_gradient_gg(h->faces, h->face_start, h->face_count, h->cell, h->dens_sorted, h->perm, h->N,
                                        grad, h->dtype, h->stream);
    return cuda_rc(cudaGetLastError());
}

int vt_grid_density(vt_handle h, int G, int S, void* grid) {
    if (!h || !grid || G < 1 || G > 4096 || S < 1 || S > 8) return VT_ERR_INVALID;
    if ((int64_t)G * G * G > ((int64_t)1 << 34)) return VT_ERR_INVALID;
    if (h->n_sets > 0) return VT_ERR_UNSUPPORTED;  // a grid needs one box
    int rc = ensure_density(h);
    if (rc) return rc;
    h->n_launches += launch_grid(h->spos, h->dtype, h->N, h->geo, h->faces, h->face_start, h->face_count, h->keys,
                                 h->dens_sorted, h->perm, G, S, grid, h->dstat, h->stream);
    return cuda_rc(cudaGetLastError());
}

namespace {
int ensure_retry(vt_handle h) {
    if (h->gretry) return VT_OK;
    h->gretry = (int4*)pool_alloc((size_t)GRID_RETRY_CAP * sizeof(int4), h->stream);
    h->gcnt = (unsigned*)pool_alloc(16 * sizeof(unsigned), h->stream);
    if (!h->gretry || !h->gcnt) return VT_ERR_OOM;
    return VT_OK;
}
}  // namespace

int vt_backward_weighted(vt_handle h, const void* w, void* dE_dpos) {
    if (!h || !w || !dE_dpos) return VT_ERR_INVALID;
    int rc = ensure_retry(h);
    if (rc) return rc;
    h->n_launches += launch_cvt_weighted(h->spos, h->dtype, h->N, h->geo, h->faces, h->face_start, h->face_count,
                                         h->cell, h->perm, w, dE_dpos, h->gretry, GRID_RETRY_CAP, h->gcnt, h->sm_count,
                                         h->stream);
    return cuda_rc(cudaGetLastError());
}

int vt_grid_density_volume(vt_handle h, int G, void* grid) {
    if (!h || !grid || G < 1 || G > 1024) return VT_ERR_INVALID;
    if (h->n_sets > 0) return VT_ERR_UNSUPPORTED;  // a grid needs one box
    int rc = ensure_density(h);
    if (rc) return rc;
    const int64_t n = (int64_t)G * G * G;
    if (h->gacc_n < n) {
        pool_free(h->gacc, h->stream);
        h->gacc_n = 0;
        h->gacc = (double*)pool_alloc(n * sizeof(double), h->stream);
        if (!h->gacc) return VT_ERR_OOM;
        h->gacc_n = n;
    }
    rc = ensure_retry(h);
    if (rc) return rc;
    h->n_launches += launch_grid_volume(h->spos, h->dtype, h->N, h->geo, h->faces, h->face_start, h->face_count,
                                        h->dens_sorted, G, h->gacc, h->gretry, GRID_RETRY_CAP, h->gcnt, grid,
                                        h->sm_count, h->stream);
    return cuda_rc(cudaGetLastError());
}

int vt_moments(vt_handle h, void* centroid, void* energy) {
    if (!h || (!centroid && !energy)) return VT_ERR_INVALID;
    h->n_launches += launch_moments(h->cell, h->spos, h->dtype, h->perm, h->N, h->geo, centroid, energy, h->stream);
    return cuda_rc(cudaGetLastError());
}

int vt_backward(vt_handle h, const void* dL_dV, double dL_dE, void* dL_dpos) {
    if (!h || !dL_dpos || !isfinite(dL_dE)) return VT_ERR_INVALID;
    h->n_launches += launch_backward(h->faces, h->face_start, h->face_count, h->cell, h->spos, h->dtype, h->perm, h->inv, h->N, dL_dV,
                    dL_dE, dL_dpos, h->stream);
    return cuda_rc(cudaGetLastError());
}

int vt_status(vt_handle h, vt_stats* out) {
    if (!h || !out) return VT_ERR_INVALID;
    DevStatus d;
    int rc = read_status(h, &d);
    if (rc) return rc;
    memset(out, 0, sizeof(*out));
    out->n = h->N;
    out->n_faces = (int64_t)d.n_faces;
    out->n_cut = (int64_t)d.n_cut;
    out->n_tested = (int64_t)d.n_tested;
    out->n_passes = (int64_t)d.n_passes;
    out->n_fp64_fallbacks = (int64_t)d.n_fp64;
    out->n_exact_cells = (int64_t)d.n_exact_cells;
    out->n_exact_preds = (int64_t)d.n_exact_preds;
    out->n_exact_zero = (int64_t)d.n_exact_zero;
    out->max_faces = (int64_t)d.max_faces;
    if (d.error == RC_POOL_HOST) d.error = VT_ERR_CAPACITY;  // facet pool full in a vt_rebuild
    if (d.invalid_input && !d.error) d.error = VT_ERR_INVALID;
    out->device_error = d.error;
    out->n_launches = h->n_launches;
    out->t_sort_ms = h->t_sort_ms;
    out->t_clip_ms = h->t_clip_ms;
    out->reserved[0] = d.error_detail;
    out->reserved[1] = (int64_t)d.n_collect;
    out->reserved[2] = (int64_t)d.n_collected;
    out->n_handed_over = h->n_owned < h->N ? 0 : (int64_t)d.n_warp_cells;
    if (h->gcnt) {
        unsigned gc[2] = {0u, 0u};
        if (cudaMemcpy(gc, h->gcnt, sizeof(gc), cudaMemcpyDeviceToHost) == cudaSuccess) out->n_grid_failed = gc[1];
        else cudaGetLastError();
    }
    out->n_bucket_passes = (int64_t)d.n_bucket_passes;
    out->error_particle = -1;
    if (d.error && d.error_cell >= 0 && d.error_cell < h->N) {
        uint32_t pi = 0;
        if (cudaMemcpy(&pi, h->perm + d.error_cell, sizeof(pi), cudaMemcpyDeviceToHost) == cudaSuccess)
            out->error_particle = (int32_t)pi;
    }
    return d.error ? d.error : VT_OK;
}

}  // extern "C"

namespace {
// FMA throughput of every SM (TFLOP/s, 2 flops per FMA): best of three timed launches after one untimed
template <bool F64>
int probe_fma(double* tflops, void* stream) {
    if (!tflops) return VT_ERR_INVALID;
    *tflops = 0.0;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    void* sink = nullptr;
    if (cudaMalloc(&sink, 4096 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return VT_ERR_OOM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // the FP64 pipe is a small fraction of the FP32 one: fewer iterations keep the launch short
    const int blocks = sms * 8, iters = F64 ? 256 : 4096;
    double best = 0.0;
    int rc = VT_OK;
    for (int rep = 0; rep < 4 && !rc; rep++) {
        cudaEventRecord(e0, s);
        if (F64) launch_fma_probe64(blocks, iters, (double*)sink, s);
        else launch_fma_probe(blocks, iters, (float*)sink, s);
        cudaEventRecord(e1, s);
        rc = cuda_rc(cudaEventSynchronize(e1));
        float ms = 0.f;
        if (!rc && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f && rep > 0) {
            const double flops = 2.0 * 8.0 * 16.0 * iters * (double)blocks * 256.0;
            const double t = flops / (ms * 1e-3) / 1e12;
            if (t > best) best = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (!rc) rc = cuda_rc(cudaGetLastError());
    *tflops = best;
    return rc;
}
}  // namespace

extern "C" {

int vt_probe_fp32_tflops(double* tflops, void* stream) { return probe_fma<false>(tflops, stream); }

int vt_probe_fp64_tflops(double* tflops, void* stream) { return probe_fma<true>(tflops, stream); }

int vt_debug_fail_alloc(int nth) { return g_fail_alloc.exchange(nth > 0 ? nth : 0); }

#ifdef VT_PHASE_TIMERS
// builds with per-phase cycle counters only (not declared in the public header): the counters of the handle's
// last clipping launch (synchronises)
int vt_debug_phase_cycles(vt_handle h, unsigned long long* out10) {
    if (!h || !out10) return VT_ERR_INVALID;
    DevStatus d;
    int rc = read_status(h, &d);
    if (!rc) memcpy(out10, d.t_phase, sizeof(d.t_phase));
    return rc;
}
#endif

int vt_last_error_detail(int* particle) {
    if (particle) *particle = g_last_particle;
    return g_last_detail;
}

const char* vt_error_string(int code) {
    switch (code) {
        case VT_OK: return "ok";
        case VT_ERR_INVALID: return "invalid argument or input (NaN, out-of-box coordinate, bad handle)";
        case VT_ERR_OOM: return "device allocation failed";
        case VT_ERR_CUDA: return "CUDA runtime error";
        case VT_ERR_DUPLICATE: return "two particles at the same position";
        case VT_ERR_SECURITY: return "security-radius test did not pass within max_passes";
        case VT_ERR_UNSUPPORTED: return "unsupported configuration (periodic cell wider than a quarter box, or box length not representable in FP32 for the FP32 filter)";
        case VT_ERR_CAPACITY: return "per-cell capacity exceeded (planes, vertices, candidates or facet pool)";
        case VT_ERR_NUMERIC: return "exact-arithmetic workspace exceeded";
        default: return "unknown error code";
    }
}

void vt_destroy(vt_handle h) {
    if (!h) return;
    free_handle(h);  // frees ordered after the handle's pending work on its stream
}

int vt_release_memory(void) {
    cudaMemPool_t pool = device_pool();
    if (!pool) return VT_ERR_CUDA;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceSynchronize() != cudaSuccess) {  // frees still pending on a stream return after their work
        cudaGetLastError();
        return VT_ERR_CUDA;
    }
    map_release();
    return cuda_rc(cudaMemPoolTrimTo(pool, 0));
}

}  // extern "C"
