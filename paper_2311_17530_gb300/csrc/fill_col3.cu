// k = 3 column kernel (placeholder until the specialised kernel lands).
#include "device_common.cuh"
#include "api_internal.h"

namespace msadp {

int col3_warps_per_cta() { return 8; }
int fill_col3_ctas_per_sm() { return 1; }
cudaError_t launch_fill_col3(const LaunchDesc &, int, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace msadp
