// Streamed line fill for k = 5.
#include "fill_lines_stream.cuh"

namespace msadp {

cudaError_t launch_fill_stream_k5(const LaunchDesc &L, int grid, cudaStream_t s) { return launch_stream<5>(L, grid, s); }
int fill_stream_ctas_k5() { return stream_ctas<5>(); }

}  // namespace msadp
