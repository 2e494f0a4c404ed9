// Generic tile fill for k = 8, instantiated for each candidate tile edge.
#include "fill_tiles.cuh"

namespace msadp {

cudaError_t launch_fill_tiles_k8(int edge, const LaunchDesc &L, int grid, cudaStream_t s) {
    return TilesK<8>::launch(edge, L, grid, s);
}
int fill_tiles_ctas_k8(int edge) { return TilesK<8>::ctas(edge); }
int fill_tiles_warps_k8(int edge) { return TilesK<8>::warps(edge); }

}  // namespace msadp
