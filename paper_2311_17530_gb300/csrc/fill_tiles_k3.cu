// Generic tile fill for k = 3, instantiated for each candidate tile edge.
#include "fill_tiles.cuh"

namespace msadp {

cudaError_t launch_fill_tiles_k3(int edge, const LaunchDesc &L, int grid, cudaStream_t s) {
    return TilesK<3>::launch(edge, L, grid, s);
}
int fill_tiles_ctas_k3(int edge) { return TilesK<3>::ctas(edge); }
int fill_tiles_warps_k3(int edge) { return TilesK<3>::warps(edge); }

}  // namespace msadp
