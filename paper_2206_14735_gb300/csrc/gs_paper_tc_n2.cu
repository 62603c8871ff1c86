// Tensor-core render kernel of the paper's architecture instantiated for rays of up to 64 samples.
#include "gs_paper_tc.cuh"

namespace gs {
namespace ptc {
template gs_status launch_paper_tc<2>(const PaperTcArgs&, int, int, cudaStream_t);
}  // namespace ptc
}  // namespace gs
