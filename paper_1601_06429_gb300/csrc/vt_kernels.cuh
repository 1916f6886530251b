// vt_kernels.cuh -- host-side launch wrappers shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "vt_internal.cuh"

namespace vt {

// sorted FP64 particle record (x, y, z, mass)
struct __align__(32) dpt4 {
    double x, y, z, w;
};

size_t scan_tmp_bytes(int64_t n);
size_t radix_tmp_bytes(int64_t N);
int scan_u32_u32(const uint32_t* in, uint32_t* out, int64_t n, void* tmp, cudaStream_t s);
int scan_u16_i64(const uint16_t* in, int64_t* out, int64_t n, void* tmp, cudaStream_t s);
int radix_sort(uint64_t* key, uint32_t* val, uint64_t* key_alt, uint32_t* val_alt, int64_t N, int bits, void* tmp,
                cudaStream_t s);
int launch_key(const void* pos, int dtype, int64_t N, const Geometry& g, uint64_t* key, uint32_t* idx, DevStatus* st,
                cudaStream_t s);
int launch_gather(const void* pos, const void* mass, int dtype, const uint32_t* perm, int64_t N, void* spos,
                   uint32_t* inv, cudaStream_t s);
int launch_key_batched(const void* pos, int dtype, int64_t N, const Geometry* sgeo, const uint32_t* setid,
                       uint64_t* key, uint32_t* idx, DevStatus* st, cudaStream_t s);
int launch_set_ids(const int64_t* soff, int n_sets, int64_t N, uint32_t* setid, cudaStream_t s);
int launch_gather_u32(const uint32_t* src, const uint32_t* perm, int64_t N, uint32_t* dst, cudaStream_t s);
int launch_owned_list(const uint32_t* inv, int64_t n_owned, uint32_t* list, DevStatus* st, cudaStream_t s);
void tree_layout(int64_t N, Tree& t);
int launch_tree(const void* spos, int dtype, int64_t N, Tree& t, cudaStream_t s);

// clipping (vt_clip.cu)
struct ClipArgs {
    const void* spos;
    int64_t N;
    Geometry geo;
    Tree tree;
    int k_target;
    int max_passes;
    int radius_policy;  // 0: radius doubling; 1: next pass also limited by the density seen so far
    CellOut* cell;
    uint32_t* face_start;
    uint16_t* face_count;
    uint8_t* cstat;
    uint32_t* exact_list;
    Face* faces;
    uint64_t face_cap;
    DevStatus* st;
    double* xws;   // exact workspace, per warp
    int xws_warps;
    // batched independent sets (NULL for one set): set of each sorted particle, geometry of each set, and the
    // sorted index range [soff[s], soff[s+1]) of each set
    const uint32_t* sset;
    const Geometry* sgeo;
    const int64_t* soff;
    // FP32 filter: the thread-per-cell and lane-group kernels run first and list here (N entries) the cells the
    // warp kernel must take; NULL: the warp kernel takes every cell
    uint32_t* warp_list;
    // batched sets: per-set clipping configuration (k_target in the low 16 bits, bits 16-17: the threads-per-cell
    // mode below), or NULL for the handle's parameters
    const int32_t* set_cfg;
    // threads per cell as a mode: 0 one warp, 1 one thread, 2 four lanes, 3 eight lanes (the handle's; cells of
    // sets with a configuration take that set's), and the modes present among the cells (bit m: mode m)
    int tpc_mode;
    int modes;
    // list_given: warp_list already holds the cells to compute (st->n_warp_cells of them; the other particles
    // are candidates only) and no thread-per-cell kernel runs
    int list_given;
    // per-cell radius (sorted order): an upper bound of the largest vertex distance of the final cell, or NULL
    float* rad;
};
int launch_clip(const ClipArgs& a, int dtype, int precision, int sm_count, cudaStream_t s);
int launch_clip_exact(const ClipArgs& a, int dtype, int sm_count, cudaStream_t s);
int launch_clip_thread(const ClipArgs& a, int dtype, int sm_count, cudaStream_t s);
int launch_clip_group(const ClipArgs& a, int dtype, int lanes, int sm_count, cudaStream_t s);
int launch_fma_probe(int blocks, int iters, float* sink, cudaStream_t s);
int launch_fma_probe64(int blocks, int iters, double* sink, cudaStream_t s);
int launch_cvt_weighted(const void* spos, int dtype, int64_t N, const Geometry& g, const Face* faces,
                        const uint32_t* face_start, const uint16_t* face_count, const CellOut* cell,
                        const uint32_t* perm, const void* w, void* out, int4* retry, unsigned retry_cap,
                        unsigned* counters, int sm_count, cudaStream_t s);
int launch_grid_volume(const void* spos, int dtype, int64_t N, const Geometry& g, const Face* faces,
                       const uint32_t* face_start, const uint16_t* face_count, const double* dens_sorted, int G,
                       double* acc, int4* retry, unsigned retry_cap, unsigned* counters, void* out, int sm_count,
                       cudaStream_t s);
int launch_gradient_gg(const Face* faces, const uint32_t* face_start, const uint16_t* face_count, const CellOut* cell,
                       const double* dens_sorted, const uint32_t* perm, int64_t N, void* grad, int dtype,
                       cudaStream_t s);
size_t exact_ws_doubles_per_warp();

// post-processing (vt_post.cu)
int launch_out_vol(const CellOut* cell, const uint32_t* perm, int64_t N, void* vol, int dtype, cudaStream_t s);
int launch_out_rad(const float* rad, const uint32_t* perm, int64_t N, void* out, int dtype, cudaStream_t s);
int launch_cell_flags(const uint8_t* cstat, const uint32_t* perm, int64_t N, uint8_t* out, cudaStream_t s);
int launch_density(const CellOut* cell, const void* spos, int dtype, const uint32_t* perm, int64_t N,
                    double* dens_sorted, void* dens, cudaStream_t s);
int launch_nbr_count(const uint16_t* face_count, const uint32_t* inv, int64_t N, uint16_t* cnt_in, cudaStream_t s);
int launch_nbr_emit(const Face* faces, const uint32_t* face_start, const uint16_t* face_count, const uint32_t* perm,
                     const uint32_t* inv, const int64_t* nbr_off, int64_t N, int32_t* nbr_id, cudaStream_t s);
int launch_gradient(const Face* faces, const uint32_t* face_start, const uint16_t* face_count, const double* dens_sorted,
                     const uint32_t* perm, int64_t N, void* grad, int dtype, cudaStream_t s);
int launch_grid(const void* spos, int dtype, int64_t N, const Geometry& g, const Face* faces,
                const uint32_t* face_start, const uint16_t* face_count, const uint64_t* keys,
                const double* dens_sorted, const uint32_t* perm, int G, int S, void* grid, DevStatus* st,
                cudaStream_t s);
int launch_moments(const CellOut* cell, const void* spos, int dtype, const uint32_t* perm, int64_t N,
                   const Geometry& g, void* cen, void* energy, cudaStream_t s);
int launch_backward(const Face* faces, const uint32_t* face_start, const uint16_t* face_count, const CellOut* cell,
                     const void* spos, int dtype, const uint32_t* perm, const uint32_t* inv, int64_t N,
                     const void* dLdV, double dLdE, void* out, cudaStream_t s);

}  // namespace vt
