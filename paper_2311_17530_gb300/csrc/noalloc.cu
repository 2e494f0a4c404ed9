// msa_align_noalloc: one alignment that allocates no memory, device or host.
//
// Who needs it: callers that must not call cudaMalloc -- code running while
// another allocator owns the GPU's memory (a framework that reserved the device
// for its own pool), latency-critical loops where an allocation would stall or
// fragment, and callers whose error handling cannot recover from an allocation
// failure in the middle of a request. They pass device inputs and outputs; all
// working memory comes from the fixed array below.
//
// The array is a file-scope __device__ variable: every GPU that loads libmsadp
// holds MSA_NOALLOC_SCRATCH_BYTES of it until the process exits. Host code cannot
// use the name as a device address, so the first call on each device looks the
// address up with cudaGetSymbolAddress (with that device current) and caches it.
// That first call should come before any stream capture. All calls share the
// array and leave their contents behind: the parts that must start at zero are
// cleared on the stream at every call, and calls whose GPU work overlaps (two
// streams, or two host threads) race on the array and must be serialised by the
// caller.
#include <cstring>
#include <mutex>

#include "api_internal.h"
#include "device_common.cuh"

namespace msadp {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[MSA_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_na_mu;
void *g_na_ptr[kMaxDevices] = {};

// Wave order of the tiles, built on the device: count tiles per wave, prefix
// sums, then scatter (any order inside a wave keeps the order topological).
__global__ void noalloc_order_kernel(const ProblemDesc *prob, uint64_t *order, int32_t *wave_cnt, int nwaves) {
    const ProblemDesc &P = *prob;
    const int64_t nt = P.ntiles;
    for (int64_t t = threadIdx.x; t < nt; t += blockDim.x) {
        int64_t rem = t;
        int w = 0;
        for (int i = 0; i < P.k; ++i) {
            const int64_t c = rem / P.gstride[i];
            rem -= c * P.gstride[i];
            w += (int)c;
        }
        atomicAdd(&wave_cnt[w], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int w = 0; w < nwaves; ++w) {
            const int c = wave_cnt[w];
            wave_cnt[w] = acc;
            acc += c;
        }
    }
    __syncthreads();
    for (int64_t t = threadIdx.x; t < nt; t += blockDim.x) {
        int64_t rem = t;
        int w = 0;
        for (int i = 0; i < P.k; ++i) {
            const int64_t c = rem / P.gstride[i];
            rem -= c * P.gstride[i];
            w += (int)c;
        }
        order[atomicAdd(&wave_cnt[w], 1)] = (uint64_t)t;
    }
}

// The 256-entry character -> code map, passed by value to the set-up kernel.
struct AmapBytes {
    uint8_t m[256];
};

// Writes the problem descriptor and the character map into the scratch. Both
// travel as kernel parameters, so no host memory is read after the call returns
// (no copy from pageable memory, which would block and could not be captured).
__global__ void noalloc_setup_kernel(const ProblemDesc d, const AmapBytes a, ProblemDesc *prob, uint8_t *amap) {
    if (threadIdx.x == 0) *prob = d;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) amap[i] = a.m[i];
}

// Shape, strides and tile grid of the generic tile kernel: the planner's own
// plan_shape (the same limits and layouts as every plan), which needs no heap
// memory; the ticket order is built on the device instead.
int noalloc_plan(int k, const int32_t *lens, int A, HostPlan &hp) {
    long double cells = 1;
    for (int i = 0; i < k; ++i) {
        if (lens[i] < 0) return set_error(MSA_EINVAL, "lens[%d]=%d is negative", i, lens[i]);
        cells *= (long double)lens[i] + 1;
    }
    if (cells > (long double)MSA_NOALLOC_SCRATCH_BYTES)
        return set_error(MSA_ETOOBIG, "msa_align_noalloc: %.3Lg cells exceed the %u-byte static scratch", cells,
                         (unsigned)MSA_NOALLOC_SCRATCH_BYTES);
    std::string err;
    const int rc = plan_shape(k, lens, A, kKernelTiles, hp, err, tile_edge_for(k));
    if (rc) return set_error(rc, "msa_align_noalloc: %s", err.c_str());
    return MSA_OK;
}

}  // namespace
}  // namespace msadp

using namespace msadp;

extern "C" int msa_align_noalloc(int k, const int32_t *lens, const char *alphabet, const char *d_residues,
                                 const int32_t *d_subst, int32_t gap, msa_device_result *d_result,
                                 uint8_t *d_masks, void *stream) {
    if (k < 2 || k > MSA_MAX_K) return set_error(MSA_EINVAL, "k=%d outside [2,%d]", k, MSA_MAX_K);
    if (!lens || !d_subst || !d_result) return set_error(MSA_EINVAL, "NULL lens, table or result pointer");
    uint8_t amap[256];
    int rc = validate_alphabet(alphabet, amap);
    if (rc) return rc;
    const int A = (int)strlen(alphabet);
    HostPlan hp;
    rc = noalloc_plan(k, lens, A, hp);
    if (rc) return rc;
    if (hp.len_sum > 0 && (!d_residues || !d_masks)) return set_error(MSA_EINVAL, "NULL residues or masks");

    size_t reset_bytes = 0;
    const size_t layout = plan_layout(hp, nullptr, nullptr, &reset_bytes);
    const size_t wave_off = (layout + 255) & ~(size_t)255;
    const size_t need = wave_off + (size_t)hp.waves * 4;
    if (need > MSA_NOALLOC_SCRATCH_BYTES)
        return set_error(MSA_ETOOBIG, "msa_align_noalloc: this problem needs %zu bytes of scratch; the static "
                                      "array holds %u bytes",
                         need, (unsigned)MSA_NOALLOC_SCRATCH_BYTES);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(MSA_EINVAL, "device %d beyond the supported range", dev);
    char *base;
    {
        std::lock_guard<std::mutex> g(g_na_mu);
        if (!g_na_ptr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress of the static scratch");
            g_na_ptr[dev] = ptr;
        }
        base = static_cast<char *>(g_na_ptr[dev]);
    }

    PlanPointers pp;
    size_t rb = 0;
    plan_layout(hp, base, &pp, &rb);
    int32_t *wave_cnt = reinterpret_cast<int32_t *>(base + wave_off);
    ProblemDesc d;
    fill_problem_desc(hp, pp, 0, d);
    cudaStream_t s = (cudaStream_t)stream;
    int64_t spin_ms;
    {
        std::lock_guard<std::mutex> g(settings_mutex());
        spin_ms = settings().spin_ms;
    }
    // zero what the previous call left behind (launch state, tile flags, wave
    // counters), then the descriptor and character map by value
    e = cudaMemsetAsync(base, 0, reset_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(wave_cnt, 0, (size_t)hp.waves * 4, s);
    if (e != cudaSuccess) return cuda_error(e, "static scratch set-up");
    AmapBytes am;
    memcpy(am.m, amap, 256);
    noalloc_setup_kernel<<<1, 256, 0, s>>>(d, am, pp.prob, pp.amap);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "set-up kernel launch");
    noalloc_order_kernel<<<1, 1024, 0, s>>>(pp.prob, pp.order, wave_cnt, hp.waves);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "order kernel launch");
    IODesc io{d_residues, d_subst, d_result, d_masks, gap, 0};
    e = launch_encode(pp.prob, 1, hp.len_sum, nullptr, io, s);
    if (e != cudaSuccess) return cuda_error(e, "encode launch");
    LaunchDesc L;
    memset(&L, 0, sizeof L);
    L.probs = pp.prob;
    L.order = pp.order;
    L.ntickets = hp.ntiles;
    L.done = pp.done;
    L.ticket = &pp.state->ticket;
    L.err = &pp.state->err;
    L.spin_ns = spin_ms * 1000000LL;
    L.withhold = -1;
    L.nprob = 1;
    e = launch_fill_tiles(k, hp.edge, L, persistent_grid(k, kKernelTiles, hp.ntiles, A, hp.edge), s);
    if (e != cudaSuccess) return cuda_error(e, "fill launch");
    e = launch_traceback(pp.prob, 1, L.err, nullptr, io, s);
    if (e != cudaSuccess) return cuda_error(e, "traceback launch");
    return MSA_OK;
}
