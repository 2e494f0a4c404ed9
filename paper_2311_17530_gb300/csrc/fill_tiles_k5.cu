// Generic tile fill for k = 5, instantiated for each candidate tile edge.
#include "fill_tiles.cuh"

namespace msadp {

cudaError_t launch_fill_tiles_k5(int edge, const LaunchDesc &L, int grid, cudaStream_t s) {
    return TilesK<5>::launch(edge, L, grid, s);
}
int fill_tiles_ctas_k5(int edge) { return TilesK<5>::ctas(edge); }
int fill_tiles_warps_k5(int edge) { return TilesK<5>::warps(edge); }

}  // namespace msadp
