// Line-sweep fill for k = 6, instantiated for each compiled segment length.
#include "fill_lines.cuh"

namespace msadp {

cudaError_t launch_fill_lines_k6(int z, const LaunchDesc &L, int grid, cudaStream_t s) {
    return LinesK<6>::launch(z, L, grid, s);
}
int fill_lines_ctas_k6(int z) { return LinesK<6>::ctas(z); }
int fill_lines_warps_k6(int z) { return LinesK<6>::warps(z); }

}  // namespace msadp
