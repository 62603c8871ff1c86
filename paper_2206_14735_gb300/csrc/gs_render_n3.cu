// Fused render kernel instantiated for rays of up to 96 samples.
#include "gs_render_kernel.cuh"

namespace gs {
template gs_status launch_n<3>(const gs_ctx*, RenderArgs&, int, cudaStream_t);
}  // namespace gs
