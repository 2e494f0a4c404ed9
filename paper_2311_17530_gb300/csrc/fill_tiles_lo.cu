// Generic tile fill, instantiated for k = 2, 3, 4.
#include "fill_tiles.cuh"

namespace msadp {

cudaError_t launch_fill_tiles_lo(int k, const LaunchDesc &L, int grid, cudaStream_t s) {
    switch (k) {
        case 2: return launch_tiles_k<2>(L, grid, s);
        case 3: return launch_tiles_k<3>(L, grid, s);
        case 4: return launch_tiles_k<4>(L, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

int fill_tiles_ctas_lo(int k) {
    switch (k) {
        case 2: return tiles_ctas_k<2>();
        case 3: return tiles_ctas_k<3>();
        case 4: return tiles_ctas_k<4>();
        default: return 0;
    }
}

}  // namespace msadp
