// Line-sweep fill for k = 5, instantiated for each compiled segment length.
#include "fill_lines.cuh"

namespace msadp {

cudaError_t launch_fill_lines_k5(int z, const LaunchDesc &L, int grid, cudaStream_t s) {
    return LinesK<5>::launch(z, L, grid, s);
}
int fill_lines_ctas_k5(int z) { return LinesK<5>::ctas(z); }
int fill_lines_warps_k5(int z) { return LinesK<5>::warps(z); }

}  // namespace msadp
