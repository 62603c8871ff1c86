// Fused render kernel (tcgen05 decoders, BF16 form) instantiated for rays of up to 160 samples.
#include "gs_render_tc.cuh"

namespace gs {
template gs_status launch_tc_n<PrecBF16, 5>(const gs_ctx*, RenderTcArgs&, int, cudaStream_t);
}  // namespace gs
