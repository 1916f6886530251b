// vt_internal.cuh -- shared declarations of the GB300 Voronoi library (device side + handle).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vt_gb300.h"

namespace vt {

constexpr int WARP = 32;
constexpr int STACK_CAP = 192;  // tree traversal stack per warp (fast clipping kernels)
constexpr int MAX_FACETS = 510; // facets of one cell (the exact kernel's plane capacity minus the initial six)
constexpr int BUCKET = 32;      // particles per leaf bucket of the search tree
constexpr int MAX_LEVELS = 8;
constexpr int EXACT_WS = 12288;  // doubles of expansion-arithmetic workspace per warp of the exact kernel

// cell status bits (per sorted cell)
constexpr uint8_t CS_DONE = 1;
constexpr uint8_t CS_NEED_EXACT = 2;
constexpr uint8_t CS_ERROR = 4;
constexpr uint8_t CS_FP64 = 8;    // FP32 geometry: a side test the FP32 filter left undecided was decided in FP64
constexpr uint8_t CS_EXACT = 16;  // finished by the exact-predicate kernel

// device-side counters (reset by vt_build, read back at its end)
struct DevStatus {
    unsigned long long n_faces;
    unsigned long long n_cut;
    unsigned long long n_tested;
    unsigned long long n_passes;
    unsigned long long n_fp64;
    unsigned long long n_exact_preds;
    unsigned long long n_exact_zero;
    unsigned long long face_next;    // next free facet record
    unsigned long long n_collect;    // candidate collections (tree traversals)
    unsigned long long n_collected;  // candidates collected
    unsigned long long t_phase[10];  // optional phase cycle counters (VT_PHASE_TIMERS builds)
    unsigned int n_exact_cells;      // length of the exact-recompute list
    unsigned int max_faces;
    int error;                       // first VT_ERR_* (atomicCAS from 0)
    int error_cell;                  // sorted index of that cell
    unsigned int work_next;          // dynamic cell scheduler
    unsigned int work_next_exact;
    unsigned int invalid_input;      // count of NaN / out-of-box coordinates
    int error_detail;                // internal reason of the first error (capacity: -101 planes, -102 triangles,
                                     // -103 boundary, -104 candidates, -105 search stack)
    unsigned long long work_next_bucket;  // bucket scheduler of the thread-per-cell kernel
    unsigned long long n_bucket_passes;   // its radius passes (per bucket)
    unsigned int n_warp_cells;            // cells it handed to the warp kernel (length of warp_list)
    unsigned long long n_tfail[8];        // ... by reason (capacity, ill-conditioned vertex, undecided in FP64,
                                          // duplicate, start box too small, security radius not reached)
    unsigned long long n_t_tested, n_t_cut, n_t_fp64, n_t_collected;  // its own counters
    unsigned long long work_next_group[2];  // unit schedulers of the four- and eight-lane kernels
};

// facet record (one per cell side of a facet between two particles)
struct __align__(16) Face {
    float dx, dy, dz;      // displacement x_j (image) - x_i
    float area;
    float cx, cy, cz;      // facet centroid relative to x_i
    uint32_t nbr;          // sorted index of the neighbour
};

// per-cell results in sorted order
struct CellOut {
    double vol;
    float zx, zy, zz;      // cell centroid relative to x_i
    float mom2;            // integral |y - x_i|^2 over the cell
};

struct Geometry {
    double lo[3], hi[3], L[3];
    float qs[3];            // 65536 / L per axis: the Morton key's quantisation (FP32: the key only orders)
    int box_f32;            // lo and hi are FP32 numbers: FP32 inputs can be checked against the box in FP32
    float Lf[3], halfLf[3], lof[3], hif[3];
    int periodic;
};

// search tree over sorted particles: level 1 = buckets of 32 particles, level l = 32 nodes of level l-1
struct Tree {
    int levels;                 // number of node levels (>= 1)
    int64_t count[MAX_LEVELS + 1];
    int64_t off[MAX_LEVELS + 1];  // offset of level l in the node arrays
    float4* lo;                 // [total nodes] (x,y,z,-)
    float4* hi;
};

}  // namespace vt

struct vt_handle_s {
    int64_t N;
    int dtype;  // VT_F32 / VT_F64
    int precision;
    vt_params prm;
    vt::Geometry geo;   // the box (batched handles: the first set's box, not periodic)
    cudaStream_t stream;
    // batched independent sets (n_sets == 0 for vt_build)
    int n_sets;
    uint32_t* sset;     // [N] set of each sorted particle
    uint32_t* set_in;   // [N] set of each input particle
    vt::Geometry* sgeo; // [n_sets]
    int64_t* soff;      // [n_sets+1] index range of each set (input and sorted order alike)
    int32_t* set_cfg;   // [n_sets] per-set k_target | thread-per-cell flag << 16, or NULL
    int modes;          // threads-per-cell modes present among the cells (bit m: mode m, see ClipArgs)
    // sorted particles
    void* spos;         // float4 (f32) or double4-like 4 doubles (f64): x,y,z,m
    uint32_t* perm;     // sorted -> input index
    uint32_t* inv;      // input -> sorted index
    // search tree
    vt::Tree tree;
    float4* tree_mem;
    // per-cell
    vt::CellOut* cell;      // [N] sorted order
    uint32_t* face_start;   // [N] sorted order
    uint16_t* face_count;   // [N] sorted order
    uint8_t* cstat;         // [N] sorted order
    uint32_t* exact_list;   // [N]
    uint32_t* warp_list;    // [N] cells the thread-per-cell kernel hands to the warp kernel (or the owned cells)
    int64_t n_owned;        // cells are computed for input rows [0, n_owned) only (N: all)
    float* rad;             // [N] sorted order: bound of each computed cell's largest vertex distance
    double* dens_sorted;    // [N] sorted order
    int dens_ready;
    uint64_t* keys;         // [N] Morton keys (sort)
    uint64_t* keys_alt;
    uint32_t* vals_alt;
    uint16_t* cnt_in;       // [N] facet counts in input order
    vt::Face* faces;        // [face_cap]
    uint64_t face_cap;
    // exact workspace (per warp of the exact kernel)
    double* xws;
    int xws_warps;
    // scratch for sort / scans
    void* tmp;
    size_t tmp_bytes;
    int64_t* nbr_off_cache;  // [N+1] input order offsets (device)
    int nbr_ready;
    vt::DevStatus* dstat;   // device
    vt::DevStatus hstat;    // host copy after build
    vt::DevStatus* smap;    // mapped pinned host block through which the status words are read
    int64_t n_faces;
    int faces_on_device;    // set by vt_rebuild: the facet count is read from the device from then on
    // volume-averaged grid: accumulator, retry list of the larger cell type, counters (retries, failures)
    double* gacc;
    int64_t gacc_n;
    int4* gretry;
    unsigned* gcnt;         // [16]: retries, failures, -, by reason (4 + code)
    int sm_count;
    int64_t n_launches;
    double t_sort_ms, t_clip_ms;
    cudaEvent_t ev[4];
};
