// vt_clip_f64.cu -- clipping kernels for FP64 particle storage (FP32-filtered and plain FP64 geometry).
#include "vt_clip_impl.cuh"

namespace vt {
void launch_clip_f64(const ClipArgs& a, int precision, int sm_count, cudaStream_t s) {
    if (precision == VT_FILTER32) launch_one<dpt4, float, false>(a, sm_count, s);
    else launch_one<dpt4, double, false>(a, sm_count, s);
}
}  // namespace vt
