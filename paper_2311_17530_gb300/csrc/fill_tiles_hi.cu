// Generic tile fill, instantiated for k = 5, 6, 7, 8.
#include "fill_tiles.cuh"

namespace msadp {

cudaError_t launch_fill_tiles_hi(int k, const LaunchDesc &L, int grid, cudaStream_t s) {
    switch (k) {
        case 5: return launch_tiles_k<5>(L, grid, s);
        case 6: return launch_tiles_k<6>(L, grid, s);
        case 7: return launch_tiles_k<7>(L, grid, s);
        case 8: return launch_tiles_k<8>(L, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

int fill_tiles_ctas_hi(int k) {
    switch (k) {
        case 5: return tiles_ctas_k<5>();
        case 6: return tiles_ctas_k<6>();
        case 7: return tiles_ctas_k<7>();
        case 8: return tiles_ctas_k<8>();
        default: return 0;
    }
}

}  // namespace msadp
