// vt_noalloc.cu -- cell volumes of a small point set without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside another library's
// memory pool, embedded or real-time hosts that forbid allocation after start-up,
// or callers that must not synchronise the device through the allocator.  For
// them this file runs the same key, sort, tree and clipping kernels as vt_build,
// with every piece of scratch memory carved out of one file-scope device array.
//
// Limits and rules (also stated in include/vt_gb300.h):
//  * at most VT_NOALLOC_MAX_N particles; larger sets get VT_ERR_CAPACITY;
//  * the array lives on every device that loads the library until the process
//    exits (about 8 MB);
//  * every call shares the array and it keeps the last call's contents; calls
//    whose work overlaps on the GPU (other streams, other host threads) race;
//  * the first call on a device looks up the array's device address with that
//    device current; make that first call before any stream capture.  The address
//    is kept for the life of the process: a cudaDeviceReset of that device loads
//    the module again elsewhere, so the entry point must not be used after one.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "vt_internal.cuh"
#include "vt_kernels.cuh"

namespace {

constexpr int64_t kMaxN = VT_NOALLOC_MAX_N;
constexpr int kFacePool = 24;   // facet records per particle
constexpr int kExactWarps = 8;  // warps of the exact-predicate kernel

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// sizes of the pieces, for kMaxN particles (FP64 positions take the larger record)
constexpr int64_t kTreeNodes = (kMaxN + 31) / 32 + (kMaxN + 1023) / 1024 + 64;
constexpr size_t kSpos = align256(kMaxN * 32);
constexpr size_t kKeys = align256(kMaxN * 8);
constexpr size_t kU32 = align256(kMaxN * 4);
constexpr size_t kU16 = align256(kMaxN * 2);
constexpr size_t kU8 = align256(kMaxN);
constexpr size_t kTree = align256(2 * kTreeNodes * 16);
constexpr size_t kCell = align256(kMaxN * sizeof(vt::CellOut));
constexpr size_t kFaces = align256((size_t)kMaxN * kFacePool * sizeof(vt::Face));
constexpr size_t kXws = align256((size_t)kExactWarps * vt::EXACT_WS * sizeof(double));
constexpr size_t kTmp = align256(64 * 1024);
constexpr size_t kStat = align256(sizeof(vt::DevStatus));
constexpr size_t kTotal = kSpos + 2 * kKeys + 4 * kU32 + kU16 + kU8 + kTree + kCell + kFaces + kXws + kTmp + kStat;

__device__ __align__(256) unsigned char g_scratch[kTotal];

std::mutex g_mu;
unsigned char* g_addr[64] = {nullptr};

// device address of g_scratch on the current device (looked up once per device and kept; not valid after a
// cudaDeviceReset of that device)
int scratch_address(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return VT_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return VT_ERR_CUDA;
        }
        g_addr[dev] = (unsigned char*)p;
    }
    *out = g_addr[dev];
    return VT_OK;
}

int rc_of(cudaError_t e) {
    if (e == cudaSuccess) return VT_OK;
    cudaGetLastError();
    return VT_ERR_CUDA;
}

}  // namespace

extern "C" int vt_volumes_noalloc(const void* pos, int dtype, int64_t N, const double box_lo[3],
                                  const double box_hi[3], int periodic, void* vol, void* stream) {
    using namespace vt;
    if (!pos || !vol || !box_lo || !box_hi || N < 1) return VT_ERR_INVALID;
    if (dtype != VT_F32 && dtype != VT_F64) return VT_ERR_INVALID;
    if (N > kMaxN) return VT_ERR_CAPACITY;
    Geometry geo;
    memset(&geo, 0, sizeof(geo));
    for (int c = 0; c < 3; c++) {
        if (!(box_hi[c] > box_lo[c])) return VT_ERR_INVALID;
        geo.lo[c] = box_lo[c];
        geo.hi[c] = box_hi[c];
        geo.L[c] = box_hi[c] - box_lo[c];
        geo.qs[c] = (float)(65536.0 / geo.L[c]);
        geo.Lf[c] = (float)geo.L[c];
        geo.halfLf[c] = 0.5f * geo.Lf[c];
        geo.lof[c] = (float)box_lo[c];
        geo.hif[c] = (float)box_hi[c];
        if (periodic && (double)geo.Lf[c] != geo.L[c]) return VT_ERR_UNSUPPORTED;
    }
    geo.periodic = periodic ? 1 : 0;
    geo.box_f32 = 1;
    for (int c = 0; c < 3; c++)
        if ((double)geo.lof[c] != geo.lo[c] || (double)geo.hif[c] != geo.hi[c]) geo.box_f32 = 0;
    unsigned char* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t s = (cudaStream_t)stream;

    // carve the array
    unsigned char* q = base;
    void* spos = q; q += kSpos;
    uint64_t* keys = (uint64_t*)q; q += kKeys;
    uint64_t* keys_alt = (uint64_t*)q; q += kKeys;
    uint32_t* perm = (uint32_t*)q; q += kU32;
    uint32_t* vals_alt = (uint32_t*)q; q += kU32;
    uint32_t* inv = (uint32_t*)q; q += kU32;
    uint32_t* face_start = (uint32_t*)q; q += kU32;
    uint16_t* face_count = (uint16_t*)q; q += kU16;
    uint8_t* cstat = (uint8_t*)q; q += kU8;
    float4* tree_mem = (float4*)q; q += kTree;
    CellOut* cell = (CellOut*)q; q += kCell;
    Face* faces = (Face*)q; q += kFaces;
    double* xws = (double*)q; q += kXws;
    void* tmp = q; q += kTmp;
    DevStatus* dstat = (DevStatus*)q; q += kStat;
    uint32_t* exact_list = vals_alt;  // free again once the sort is done

    Tree tree;
    tree_layout(N, tree);
    if (tree.off[0] > kTreeNodes || radix_tmp_bytes(N) > kTmp) return VT_ERR_CAPACITY;
    if (exact_ws_doubles_per_warp() != (size_t)EXACT_WS) return VT_ERR_CAPACITY;  // the kernel's stride per warp
    tree.lo = tree_mem;
    tree.hi = tree_mem + tree.off[0];

    // everything that must start at zero: the status words and counters
    rc = rc_of(cudaMemsetAsync(dstat, 0, sizeof(DevStatus), s));
    if (rc) return rc;
    launch_key(pos, dtype, N, geo, keys, perm, dstat, s);
    radix_sort(keys, perm, keys_alt, vals_alt, N, 48, tmp, s);
    launch_gather(pos, nullptr, dtype, perm, N, spos, inv, s);
    launch_tree(spos, dtype, N, tree, s);
    ClipArgs a;
    memset(&a, 0, sizeof(a));
    a.spos = spos;
    a.N = N;
    a.geo = geo;
    a.tree = tree;
    a.k_target = 24;
    a.max_passes = 1000;
    a.radius_policy = 1;
    a.cell = cell;
    a.face_start = face_start;
    a.face_count = face_count;
    a.cstat = cstat;
    a.exact_list = exact_list;
    a.faces = faces;
    a.face_cap = (uint64_t)N * kFacePool;
    a.st = dstat;
    a.xws = xws;
    a.xws_warps = kExactWarps;
    a.warp_list = nullptr;  // the warp-per-cell kernel on every cell, as vt_build's default
    launch_clip(a, dtype, VT_FILTER32, sms, s);
    launch_clip_exact(a, dtype, sms, s);
    rc = rc_of(cudaGetLastError());
    if (rc) return rc;
    DevStatus hs;
    rc = rc_of(cudaMemcpyAsync(&hs, dstat, sizeof(hs), cudaMemcpyDeviceToHost, s));
    if (!rc) rc = rc_of(cudaStreamSynchronize(s));
    if (rc) return rc;
    if (hs.invalid_input) return VT_ERR_INVALID;
    if (hs.error) return hs.error > 0 ? VT_ERR_CAPACITY : hs.error;  // a full facet pool cannot grow here
    launch_out_vol(cell, perm, N, vol, dtype, s);
    return rc_of(cudaGetLastError());
}
