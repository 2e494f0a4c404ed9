// Generic tile fill for k = 2, instantiated for each candidate tile edge.
#include "fill_tiles.cuh"

namespace msadp {

cudaError_t launch_fill_tiles_k2(int edge, const LaunchDesc &L, int grid, cudaStream_t s) {
    return TilesK<2>::launch(edge, L, grid, s);
}
int fill_tiles_ctas_k2(int edge) { return TilesK<2>::ctas(edge); }
int fill_tiles_warps_k2(int edge) { return TilesK<2>::warps(edge); }

}  // namespace msadp
