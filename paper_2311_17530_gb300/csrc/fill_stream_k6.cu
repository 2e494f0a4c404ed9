// Streamed line fill for k = 6: the whole-column form (fill_lines_wide.cuh) when
// the last axis fits its box, the pipelined form otherwise.
#include "fill_lines_stream.cuh"
#include "fill_lines_wide.cuh"

namespace msadp {

cudaError_t launch_fill_stream_k6(const LaunchDesc &L, int grid, cudaStream_t s, int rho_s) {
    return rho_s <= kWideZ ? launch_wide<6>(L, grid, s) : launch_stream<6>(L, grid, s);
}
int fill_stream_ctas_k6() {
    const int a = wide_ctas<6>(), b = stream_ctas<6>();
    return a < b ? a : b;
}

}  // namespace msadp
