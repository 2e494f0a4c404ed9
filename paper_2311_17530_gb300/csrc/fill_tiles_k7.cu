// Generic tile fill for k = 7, instantiated for each candidate tile edge.
#include "fill_tiles.cuh"

namespace msadp {

cudaError_t launch_fill_tiles_k7(int edge, const LaunchDesc &L, int grid, cudaStream_t s) {
    return TilesK<7>::launch(edge, L, grid, s);
}
int fill_tiles_ctas_k7(int edge) { return TilesK<7>::ctas(edge); }
int fill_tiles_warps_k7(int edge) { return TilesK<7>::warps(edge); }

}  // namespace msadp
