// Streamed line fill for k = 4.
#include "fill_lines_stream.cuh"

namespace msadp {

cudaError_t launch_fill_stream_k4(const LaunchDesc &L, int grid, cudaStream_t s) { return launch_stream<4>(L, grid, s); }
int fill_stream_ctas_k4() { return stream_ctas<4>(); }

}  // namespace msadp
