// Generic tile fill for k = 6, instantiated for each candidate tile edge.
#include "fill_tiles.cuh"

namespace msadp {

cudaError_t launch_fill_tiles_k6(int edge, const LaunchDesc &L, int grid, cudaStream_t s) {
    return TilesK<6>::launch(edge, L, grid, s);
}
int fill_tiles_ctas_k6(int edge) { return TilesK<6>::ctas(edge); }
int fill_tiles_warps_k6(int edge) { return TilesK<6>::warps(edge); }

}  // namespace msadp
