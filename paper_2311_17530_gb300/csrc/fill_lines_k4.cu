// Line-sweep fill for k = 4, instantiated for each compiled segment length.
#include "fill_lines.cuh"

namespace msadp {

cudaError_t launch_fill_lines_k4(int z, const LaunchDesc &L, int grid, cudaStream_t s) {
    return LinesK<4>::launch(z, L, grid, s);
}
int fill_lines_ctas_k4(int z) { return LinesK<4>::ctas(z); }
int fill_lines_warps_k4(int z) { return LinesK<4>::warps(z); }

}  // namespace msadp
