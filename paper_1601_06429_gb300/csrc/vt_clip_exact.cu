// vt_clip_exact.cu -- the exact-predicate clipping kernels (cells whose FP64 tests were undecided) and
// the launch entry points of the clipping stage.
#include "vt_clip_impl.cuh"

namespace vt {
void launch_clip_f32(const ClipArgs& a, int precision, int sm_count, cudaStream_t s);
void launch_clip_f64(const ClipArgs& a, int precision, int sm_count, cudaStream_t s);

size_t exact_ws_doubles_per_warp() { return EXACT_WS; }

// FP32 filter with a warp list: the thread-per-cell kernel, then the warp kernel on the cells it handed over.
// A given list (cells of owned particles only): the warp kernel on the listed cells.  Otherwise (plain FP64, or no
// list) the warp kernel on every cell.
int launch_clip(const ClipArgs& a, int dtype, int precision, int sm_count, cudaStream_t s) {
    int n = 0;
    ClipArgs b = a;
    if (a.list_given) {
        // the cells to compute are listed: the warp kernel takes exactly those
    } else if (precision == VT_FILTER32 && a.warp_list) {
        // the thread-per-cell kernel also lists the cells of the warp mode, so it runs whenever either is present
        if (a.modes & 3) n += launch_clip_thread(a, dtype, sm_count, s);
        if (a.modes & 4) n += launch_clip_group(a, dtype, 4, sm_count, s);
        if (a.modes & 8) n += launch_clip_group(a, dtype, 8, sm_count, s);
    } else {
        b.warp_list = nullptr;
    }
    if (dtype == VT_F32) launch_clip_f32(b, precision, sm_count, s);
    else launch_clip_f64(b, precision, sm_count, s);
    return n + 1;
}

int launch_clip_exact(const ClipArgs& a, int dtype, int sm_count, cudaStream_t s) {
    if (dtype == VT_F32) launch_one<float4, double, true>(a, sm_count, s);
    else launch_one<dpt4, double, true>(a, sm_count, s);
    return 1;
}
}  // namespace vt
