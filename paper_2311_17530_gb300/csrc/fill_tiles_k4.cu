// Generic tile fill for k = 4, instantiated for each candidate tile edge.
#include "fill_tiles.cuh"

namespace msadp {

cudaError_t launch_fill_tiles_k4(int edge, const LaunchDesc &L, int grid, cudaStream_t s) {
    return TilesK<4>::launch(edge, L, grid, s);
}
int fill_tiles_ctas_k4(int edge) { return TilesK<4>::ctas(edge); }
int fill_tiles_warps_k4(int edge) { return TilesK<4>::warps(edge); }

}  // namespace msadp
