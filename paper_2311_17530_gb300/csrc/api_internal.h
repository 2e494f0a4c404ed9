// Host-side helpers shared by api.cpp and serve.cpp.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "plan.h"

namespace msadp {

struct Settings {
    int64_t spin_ms = 5000;
    int64_t budget_mb = 16384;
    int64_t max_batch = 64;
    int64_t use_graphs = 1;
    int64_t batching = 1;
    int64_t fill_kernel = 0;
    int64_t withhold = -1;
    int64_t timing = 0;
    int64_t poison_tb = 0;
    int64_t verify_corner = 0;
};

// Header of a workspace; zeroed before every execution.
struct LaunchState {
    int32_t ticket;
    int32_t err;
    int32_t pad[2];
    msa_device_result istat;
};

struct PlanPointers {
    LaunchState *state = nullptr;
    int32_t *done = nullptr;
    uint64_t *order = nullptr;
    ProblemDesc *prob = nullptr;
    uint8_t *amap = nullptr;
    uint8_t *codes = nullptr;
    int32_t *tab = nullptr;
    int32_t *qcorner = nullptr;
    uint8_t *tb = nullptr;
    int32_t *Q = nullptr;
    int32_t *aux = nullptr;
};

int col3_warps_per_cta();

int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what);
Settings &settings();
std::mutex &settings_mutex();
cudaStream_t library_stream(int *rc);
int validate_alphabet(const char *alphabet, uint8_t amap[256]);
int validate_request(int k, const char *const *seqs, const int32_t *lens, const char *alphabet,
                     const int32_t *subst, uint8_t amap[256]);
int status_error(int status);
int persistent_grid(int k, int kernel, int64_t units, int A, int edge);
// msa_plan_create with an explicit kernel choice and tile edge (edge < 0: tuned).
int plan_create(int k, const int32_t *lens, const char *alphabet, int kernel_choice, int edge, msa_plan **out_plan);
size_t plan_layout(const HostPlan &hp, char *base, PlanPointers *pp, size_t *reset_bytes);
void fill_problem_desc(const HostPlan &hp, const PlanPointers &pp, int64_t tile_base, ProblemDesc &d);
int launch_fill(const HostPlan &hp, const LaunchDesc &L, int grid, cudaStream_t s);
cudaError_t clear_faces(const HostPlan &hp, const PlanPointers &pp, cudaStream_t s = nullptr);
// msa_plan_execute's steps, with the pruning kernels between encode and fill
// when `prune` is given (msa_align_pruned).
int run_plan(msa_plan *plan, const char *d_residues, const int32_t *d_subst, int32_t gap, msa_device_result *d_result,
             uint8_t *d_masks, void *stream, const PruneDesc *prune);
void expand_alignment(int k, const char *const *seqs, const int32_t *lens, const uint8_t *masks_rev,
                      int ncols, char *out);

}  // namespace msadp
