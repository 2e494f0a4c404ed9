// Autotuner of the tile shape: the paper fixes its partition size S by hand
// (section 3.2's example uses S = 3); here each k has a few compiled tile edges
// (tile_edge_candidate) and, for k = 3, the column kernel (k = 2: the band
// kernel; k = 4 .. 6: the line kernel's compiled segment lengths, and at k = 4, 5
// its streamed form). msa_autotune times
// every candidate on a synthetic problem of the caller's shape -- plan creation,
// then repeated executions of encode, fill and traceback between CUDA events --
// and makes the fastest the choice for k in every later plan and serving batch.
#include <cstring>
#include <vector>

#include "api_internal.h"

using namespace msadp;

namespace {

struct DeviceBuffers {
    char *res = nullptr;
    int32_t *sub = nullptr;
    msa_device_result *out = nullptr;
    uint8_t *masks = nullptr;
    ~DeviceBuffers() {
        cudaFree(res);
        cudaFree(sub);
        cudaFree(out);
        cudaFree(masks);
    }
};

// Mean milliseconds of `repeats` executions of a plan (after one warm-up).
int time_candidate(int k, const int32_t *lens, const char *alphabet, int kernel, int edge, const DeviceBuffers &b,
                   int32_t gap, int repeats, cudaStream_t s, float *out_ms, int *out_kernel, int *out_edge) {
    msa_plan *plan = nullptr;
    int rc = plan_create(k, lens, alphabet, kernel, edge, &plan);
    if (rc) return rc;
    msa_plan_info info;
    msa_plan_get_info(plan, &info);
    *out_kernel = info.fill_kernel;
    *out_edge = info.fill_kernel == kKernelTiles || info.fill_kernel == kKernelLines ? edge : 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        rc = msa_plan_execute(plan, b.res, b.sub, gap, b.out, b.masks, s);
        if (!rc) e = cudaEventRecord(e0, s);
        for (int r = 0; r < repeats && !rc && e == cudaSuccess; ++r)
            rc = msa_plan_execute(plan, b.res, b.sub, gap, b.out, b.masks, s);
        if (!rc && e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (!rc && e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (!rc && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        *out_ms = ms / repeats;
        msa_device_result res;
        if (!rc && e == cudaSuccess) e = cudaMemcpy(&res, b.out, sizeof res, cudaMemcpyDeviceToHost);
        if (!rc && e == cudaSuccess && res.status != MSA_OK) rc = status_error(res.status);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    msa_plan_destroy(plan);
    if (!rc && e != cudaSuccess) rc = cuda_error(e, "autotune timing");
    return rc;
}

}  // namespace

extern "C" {

int msa_set_tile_edge(int k, int32_t edge) {
    if (set_tile_edge(k, edge) != MSA_OK)
        return set_error(MSA_EINVAL, "tile edge %d is not compiled for k=%d", edge, k);
    if (k == 3 && edge == 0) set_prefer_tiles_k3(false);  // defaults: the column kernel where it fits
    if (k == 2 && edge == 0) set_prefer_tiles_k2(false);  // defaults: the band kernel
    return MSA_OK;
}

int msa_get_tile_edge(int k, int32_t *out_edge) {
    if (k < 2 || k > MSA_MAX_K || !out_edge) return set_error(MSA_EINVAL, "bad arguments");
    *out_edge = tile_edge_for(k);
    return MSA_OK;
}

int msa_set_line_segment(int k, int32_t z) {
    if (set_line_z(k, z) != MSA_OK) return set_error(MSA_EINVAL, "line segment %d is not compiled for k=%d", z, k);
    if (z == 0) {  // defaults: the line kernel for k = 4 .. 6, streamed at k = 4, 5
        set_prefer_tiles_lines(k, false);
        reset_prefer_stream(k);
    }
    return MSA_OK;
}

int msa_get_line_segment(int k, int32_t *out_z) {
    if (k < 2 || k > MSA_MAX_K || !out_z) return set_error(MSA_EINVAL, "bad arguments");
    *out_z = line_z_for(k);
    return MSA_OK;
}

int msa_autotune(int k, const int32_t *lens, int alphabet_size, int32_t repeats, msa_tuning *out) {
    if (k < 2 || k > MSA_MAX_K || !lens || !out || repeats < 1)
        return set_error(MSA_EINVAL, "bad arguments");
    if (alphabet_size < 1 || alphabet_size > MSA_MAX_ALPHABET)
        return set_error(MSA_EINVAL, "alphabet size %d outside [1,%d]", alphabet_size, MSA_MAX_ALPHABET);
    int64_t total = 0;
    for (int i = 0; i < k; ++i) {
        if (lens[i] < 0) return set_error(MSA_EINVAL, "lens[%d]=%d is negative", i, lens[i]);
        total += lens[i];
    }
    // synthetic problem: letters A.., a linear congruential residue stream, and
    // a symmetric match/mismatch table (the fill's cost does not depend on values)
    const char *letters = "ABCDEFGHIJKLMNOPQRSTUVWXYZabcdef";
    char alphabet[MSA_MAX_ALPHABET + 1] = {};
    memcpy(alphabet, letters, (size_t)alphabet_size);
    std::vector<char> res((size_t)total + 1);
    uint32_t x = 2463534242u;
    for (int64_t i = 0; i < total; ++i) {
        x = x * 1664525u + 1013904223u;
        res[(size_t)i] = alphabet[(x >> 16) % (uint32_t)alphabet_size];
    }
    std::vector<int32_t> sub((size_t)alphabet_size * alphabet_size);
    for (int a = 0; a < alphabet_size; ++a)
        for (int b = 0; b < alphabet_size; ++b) sub[(size_t)a * alphabet_size + b] = a == b ? 5 : -4;
    int rc = MSA_OK;
    cudaStream_t s = library_stream(&rc);
    if (rc) return rc;
    DeviceBuffers b;
    cudaError_t e = cudaMalloc(&b.res, res.size());
    if (e == cudaSuccess) e = cudaMalloc(&b.sub, sub.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&b.out, sizeof(msa_device_result));
    if (e == cudaSuccess) e = cudaMalloc(&b.masks, (size_t)total + 16);
    if (e == cudaSuccess) e = cudaMemcpy(b.res, res.data(), res.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b.sub, sub.data(), sub.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(MSA_ENOMEM, "autotune buffers: %s", cudaGetErrorString(e));
    }
    memset(out, 0, sizeof *out);
    out->k = k;
    struct Cand {
        int kernel, edge;
    };
    std::vector<Cand> cands;
    for (int i = 0; i < kMaxTileEdges; ++i)
        if (tile_edge_candidate(k, i) > 0) cands.push_back({kKernelTiles, tile_edge_candidate(k, i)});
    if (k == 3 && choose_kernel(k, lens, alphabet_size, kKernelCol3) == kKernelCol3) cands.push_back({kKernelCol3, 0});
    if (k == 2) cands.push_back({kKernelBand2, 0});
    for (int i = 0; i < kMaxLineSegments; ++i)
        if (line_z_candidate(k, i) > 0) cands.push_back({kKernelLines, line_z_candidate(k, i)});
    if (k >= kStreamMinK && k <= kStreamMaxK && stream_fits(k, lens)) cands.push_back({kKernelStream, 0});
    int best = -1;
    for (const Cand &c : cands) {
        if (out->ncand >= MSA_MAX_TUNING_CANDIDATES) break;
        float ms = 0;
        int kern = 0, edge = 0;
        rc = time_candidate(k, lens, alphabet, c.kernel, c.kernel == kKernelTiles || c.kernel == kKernelLines ? c.edge : -1,
                            b, -8, repeats, s,
                            &ms, &kern, &edge);
        if (rc) return rc;
        const int i = out->ncand++;
        out->cand_kernel[i] = kern;
        out->cand_edge[i] = edge;
        out->cand_ms[i] = ms;
        if (best < 0 || ms < out->cand_ms[best]) best = i;
    }
    out->best = best;
    // the winner becomes the choice for k
    if (out->cand_kernel[best] == kKernelTiles) {
        set_tile_edge(k, out->cand_edge[best]);
        if (k == 3) set_prefer_tiles_k3(true);
        if (k == 2) set_prefer_tiles_k2(true);
        set_prefer_tiles_lines(k, true);
        set_prefer_stream(k, false);
    } else {
        if (k == 3) set_prefer_tiles_k3(false);
        if (k == 2) set_prefer_tiles_k2(false);
        if (out->cand_kernel[best] == kKernelLines) {
            set_line_z(k, out->cand_edge[best]);
            set_prefer_tiles_lines(k, false);
            set_prefer_stream(k, false);
        }
        if (out->cand_kernel[best] == kKernelStream) {
            set_prefer_tiles_lines(k, false);
            set_prefer_stream(k, true);
            // the best segmented candidate stays the choice where the streamed one cannot run (serving)
            int bl = -1;
            for (int i = 0; i < out->ncand; ++i)
                if (out->cand_kernel[i] == kKernelLines && (bl < 0 || out->cand_ms[i] < out->cand_ms[bl])) bl = i;
            if (bl >= 0) set_line_z(k, out->cand_edge[bl]);
        }
        // the best generic edge stays the fallback for shapes the column kernel cannot take
        int bt = -1;
        for (int i = 0; i < out->ncand; ++i)
            if (out->cand_kernel[i] == kKernelTiles && (bt < 0 || out->cand_ms[i] < out->cand_ms[bt])) bt = i;
        if (bt >= 0) set_tile_edge(k, out->cand_edge[bt]);
    }
    return MSA_OK;
}

}  // extern "C"
