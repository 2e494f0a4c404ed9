// Streamed line fill for k = 6.
#include "fill_lines_stream.cuh"

namespace msadp {

cudaError_t launch_fill_stream_k6(const LaunchDesc &L, int grid, cudaStream_t s) { return launch_stream<6>(L, grid, s); }
int fill_stream_ctas_k6() { return stream_ctas<6>(); }

}  // namespace msadp
