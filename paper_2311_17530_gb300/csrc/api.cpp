// libmsadp C-ABI: validation, plans, the synchronous msa_align, settings and
// the host-only planner queries.
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "api_internal.h"
#include "plan_hooks.h"

using namespace msadp;

namespace msadp {

thread_local std::string t_err;

int set_error(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return code;
}

int cuda_error(cudaError_t e, const char *what) {
    return set_error(MSA_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

Settings &settings() {
    static Settings s;
    return s;
}

std::mutex &settings_mutex() {
    static std::mutex m;
    return m;
}

static void *g_stream = nullptr;
static bool g_stream_set = false;
static cudaStream_t g_own_stream = nullptr;

cudaStream_t library_stream(int *rc) {
    *rc = MSA_OK;
    std::lock_guard<std::mutex> g(settings_mutex());  // msa_set_stream may run on another thread
    if (g_stream_set) return (cudaStream_t)g_stream;
    if (!g_own_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&g_own_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            *rc = cuda_error(e, "cudaStreamCreate");
            return nullptr;
        }
    }
    return g_own_stream;
}

int validate_alphabet(const char *alphabet, uint8_t amap[256]) {
    if (!alphabet) return set_error(MSA_EINVAL, "alphabet is NULL");
    const size_t A = strlen(alphabet);
    if (A < 1 || A > MSA_MAX_ALPHABET)
        return set_error(MSA_EINVAL, "alphabet size %zu outside [1,%d]", A, MSA_MAX_ALPHABET);
    memset(amap, 0xFF, 256);
    for (size_t i = 0; i < A; ++i) {
        const uint8_t c = (uint8_t)alphabet[i];
        if (amap[c] != 0xFF) return set_error(MSA_EINVAL, "alphabet repeats character '%c'", c);
        amap[c] = (uint8_t)i;
    }
    return MSA_OK;
}

int validate_request(int k, const char *const *seqs, const int32_t *lens, const char *alphabet,
                     const int32_t *subst, uint8_t amap[256]) {
    if (k < 2 || k > MSA_MAX_K) return set_error(MSA_EINVAL, "k=%d outside [2,%d]", k, MSA_MAX_K);
    if (!seqs || !lens || !subst) return set_error(MSA_EINVAL, "NULL seqs, lens or subst");
    int rc = validate_alphabet(alphabet, amap);
    if (rc) return rc;
    const int A = (int)strlen(alphabet);
    for (int i = 0; i < k; ++i) {
        if (lens[i] < 0) return set_error(MSA_EINVAL, "lens[%d]=%d is negative", i, lens[i]);
        if (lens[i] > 0 && !seqs[i]) return set_error(MSA_EINVAL, "seqs[%d] is NULL", i);
        for (int32_t t = 0; t < lens[i]; ++t)
            if (amap[(uint8_t)seqs[i][t]] == 0xFF)
                return set_error(MSA_EINVAL, "sequence %d position %d: residue '%c' not in alphabet", i,
                                 t, seqs[i][t]);
    }
    for (int a = 0; a < A; ++a)
        for (int b = a + 1; b < A; ++b)
            if (subst[a * A + b] != subst[b * A + a])
                return set_error(MSA_EINVAL, "substitution table not symmetric at (%d,%d)", a, b);
    return MSA_OK;
}

int status_error(int status) {
    switch (status) {
        case MSA_OK: return MSA_OK;
        case MSA_EINVAL: return set_error(MSA_EINVAL, "device check: residue outside the alphabet or non-symmetric table");
        case MSA_ETOOBIG: return set_error(MSA_ETOOBIG, "scores could leave the exact int32 range for this table and gap");
        case MSA_ETIMEOUT: return set_error(MSA_ETIMEOUT, "a device dependency wait exceeded its limit; the fill stopped");
        default: return set_error(MSA_ECUDA, "device traceback found an inconsistent traceback tensor (status %d)", status);
    }
}

int device_sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

int persistent_grid(int k, int kernel, int64_t units, int A, int edge) {
    // resident CTAs per SM, cached per (kernel, k, alphabet size or tile edge)
    static std::mutex mu;
    static int cache[kKernelCount][MSA_MAX_K + 1][MSA_MAX_ALPHABET + 1] = {};
    int c;
    {
        std::lock_guard<std::mutex> g(mu);
        const int sub = kernel == kKernelCol3    ? A
                      : kernel == kKernelLines ? (edge == line_z_candidate(k, 0) ? 1 : edge == line_z_candidate(k, 1) ? 2 : 3)
                                               : (edge & 31);
        int &slot = cache[kernel][k][sub];
        if (!slot) {
            slot = kernel == kKernelCol3    ? fill_col3_ctas_per_sm(col3_smem_bytes(A))
                   : kernel == kKernelBand2 ? fill_band2_ctas_per_sm()
                   : kernel == kKernelLines ? fill_lines_ctas_per_sm(k, edge)
                   : kernel == kKernelStream ? fill_stream_ctas_per_sm(k)
                                            : fill_tiles_ctas_per_sm(k, edge);
            if (slot <= 0) slot = 1;
        }
        c = slot;
    }
    // the tile, line and band kernels take one unit per warp, the column kernel
    // and the streamed line kernel one per CTA
    const int per_cta = kernel == kKernelCol3    ? 1
                      : kernel == kKernelBand2 ? fill_band2_warps_per_cta()
                      : kernel == kKernelLines ? std::max(1, fill_lines_warps_per_cta(k, edge))
                      : kernel == kKernelStream ? 1
                                               : std::max(1, fill_tiles_warps_per_cta(k, edge));
    int64_t need = (units + per_cta - 1) / per_cta;
    int64_t g = (int64_t)c * device_sm_count();
    if (need < g) g = need;
    return (int)(g < 1 ? 1 : g);
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Carve one workspace allocation; `base` may be nullptr to measure only.
size_t plan_layout(const HostPlan &hp, char *base, PlanPointers *pp, size_t *reset_bytes) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return base ? base + o : nullptr;
    };
    char *hdr = take(sizeof(LaunchState));
    char *done = take((size_t)hp.ntiles * 4);  // one completion counter per ticket
    *reset_bytes = off;
    char *order = take((size_t)hp.ntiles * 8);
    char *prob = take(sizeof(ProblemDesc));
    char *amap = take(256);
    char *codes = take((size_t)hp.len_sum + 16);
    char *tab = take((size_t)hp.A * hp.A * 4);
    char *qc = take(16);
    char *tb = take((size_t)hp.tb_dev_bytes + 16);
    char *Q = take((size_t)hp.qelems * 4 + 16);
    char *aux = take((size_t)hp.aux_elems * 4 + 16);
    if (pp && base) {
        LaunchState *ls = reinterpret_cast<LaunchState *>(hdr);
        pp->state = ls;
        pp->done = reinterpret_cast<int32_t *>(done);
        pp->order = reinterpret_cast<uint64_t *>(order);
        pp->prob = reinterpret_cast<ProblemDesc *>(prob);
        pp->amap = reinterpret_cast<uint8_t *>(amap);
        pp->codes = reinterpret_cast<uint8_t *>(codes);
        pp->tab = reinterpret_cast<int32_t *>(tab);
        pp->qcorner = reinterpret_cast<int32_t *>(qc);
        pp->tb = reinterpret_cast<uint8_t *>(tb);
        pp->Q = reinterpret_cast<int32_t *>(Q);
        pp->aux = reinterpret_cast<int32_t *>(aux);
    }
    return off;
}

void fill_problem_desc(const HostPlan &hp, const PlanPointers &pp, int64_t tile_base, ProblemDesc &d) {
    memset(&d, 0, sizeof d);
    d.k = hp.k;
    d.A = hp.A;
    d.B = hp.k;
    d.ncode = hp.len_sum;
    int32_t off = 0;
    for (int i = 0; i < hp.k; ++i) {
        d.rho[i] = hp.rho[i];
        d.len[i] = hp.lens[i];
        d.cofs[i] = off;
        off += hp.lens[i];
        d.G[i] = hp.G[i];
        d.E[i] = hp.E[i];
        d.gstride[i] = hp.gstride[i];
        d.sgstride[i] = hp.sgstride[i];
        d.qstride[i] = hp.qstride[i];
        d.tbstride[i] = hp.tbstride[i];
        d.lst[i] = hp.lst[i];
    }
    d.tb_block = hp.tb_block;
    d.lzq = hp.lzq;
    d.tile_base = tile_base;
    d.ntiles = hp.ntiles;
    d.has_qcorner = hp.check_corner;
    d.face0_stride = hp.face0_stride;
    d.face1_stride = hp.face1_stride;
    d.face0_rows = hp.face0_rows;
    d.face1_rows = hp.face1_rows;
    d.tb_layout = hp.tb_layout;
    d.pair_min_sum = hp.pair_min_sum;
    d.w_corner = hp.w_corner;
    d.len_sum = hp.len_sum;
    d.amap = pp.amap;
    d.codes = pp.codes;
    d.tab = pp.tab;
    d.Q = pp.Q;
    d.aux = pp.aux;
    d.tb = pp.tb;
    d.qcorner = pp.qcorner;
    d.istat = &pp.state->istat;
}

cudaError_t clear_faces(const HostPlan &hp, const PlanPointers &pp, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(pp.Q, 0, (size_t)hp.qelems * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(pp.aux, 0, (size_t)hp.aux_elems * 4, s);
    if (e == cudaSuccess && s == nullptr) e = cudaDeviceSynchronize();
    return e;
}

int launch_fill(const HostPlan &hp, const LaunchDesc &L, int grid, cudaStream_t s) {
    cudaError_t e = hp.kernel == kKernelCol3    ? launch_fill_col3(L, grid, col3_smem_bytes(hp.A), s)
                  : hp.kernel == kKernelBand2 ? launch_fill_band2(L, grid, s)
                  : hp.kernel == kKernelLines ? launch_fill_lines(hp.k, hp.edge, L, grid, s)
                  : hp.kernel == kKernelStream ? launch_fill_stream(hp.k, L, grid, s, hp.rho[hp.k - 1])
                                              : launch_fill_tiles(hp.k, hp.edge, L, grid, s);
    return e == cudaSuccess ? MSA_OK : cuda_error(e, "fill kernel launch");
}

}  // namespace msadp

struct msa_plan {
    HostPlan hp;
    char alphabet[MSA_MAX_ALPHABET + 1];
    char *ws = nullptr;
    size_t ws_bytes = 0;
    size_t reset_bytes = 0;
    PlanPointers pp;
    int grid = 1;
    cudaStream_t last_stream = nullptr;
    int32_t epoch = 0;  // tag of the last execution's face entries (column and streamed line kernels)
    // per-stage events of timed executions, a ring of kTimedRing executions
    static constexpr int kTimedRing = 256;
    std::vector<cudaEvent_t> ev;
    int timed = 0;  // executions recorded since the last msa_plan_timings
};

extern "C" {

const char *msa_last_error(void) { return t_err.c_str(); }

const char *msa_version(void) { return "libmsadp 0.1 (sm_103a)"; }

int msa_set_stream(void *stream) {
    std::lock_guard<std::mutex> g(settings_mutex());
    g_stream = stream;
    g_stream_set = true;
    return MSA_OK;
}

int msa_config(const char *key, int64_t value) {
    if (!key) return set_error(MSA_EINVAL, "NULL key");
    std::lock_guard<std::mutex> g(settings_mutex());
    Settings &s = settings();
    if (!strcmp(key, "spin_timeout_ms")) {
        if (value < 1) return set_error(MSA_EINVAL, "spin_timeout_ms must be >= 1");
        s.spin_ms = value;
    } else if (!strcmp(key, "device_budget_mb")) {
        if (value < 1) return set_error(MSA_EINVAL, "device_budget_mb must be >= 1");
        s.budget_mb = value;
    } else if (!strcmp(key, "max_batch")) {
        if (value < 1 || value > 4096) return set_error(MSA_EINVAL, "max_batch must be in [1,4096]");
        s.max_batch = value;
    } else if (!strcmp(key, "use_graphs")) {
        s.use_graphs = value ? 1 : 0;
    } else if (!strcmp(key, "batching")) {
        s.batching = value ? 1 : 0;
    } else if (!strcmp(key, "fill_kernel")) {
        if (value < 0 || value > 5) return set_error(MSA_EINVAL, "fill_kernel must be 0, 1, 2, 3, 4 or 5");
        s.fill_kernel = value;
    } else if (!strcmp(key, "timing")) {
        s.timing = value ? 1 : 0;
    } else if (!strcmp(key, "test_withhold_tile")) {
        s.withhold = value;
    } else if (!strcmp(key, "verify_corner")) {
        s.verify_corner = value ? 1 : 0;
    } else if (!strcmp(key, "test_poison_tb")) {
        s.poison_tb = value ? 1 : 0;
    } else if (!strcmp(key, "test_shuffle_waves")) {
        if (value < 0) return set_error(MSA_EINVAL, "test_shuffle_waves must be >= 0");
        set_wave_shuffle_seed((uint64_t)value);
    } else {
        return set_error(MSA_EINVAL, "unknown setting '%s'", key);
    }
    return MSA_OK;
}

int msa_plan_create(int k, const int32_t *lens, const char *alphabet, msa_plan **out_plan) {
    int kernel_choice;
    {
        std::lock_guard<std::mutex> g(settings_mutex());
        kernel_choice = (int)settings().fill_kernel;
    }
    return msadp::plan_create(k, lens, alphabet, kernel_choice, -1, out_plan);
}

}  // extern "C"

namespace msadp {

int plan_create(int k, const int32_t *lens, const char *alphabet, int kernel_choice, int edge, msa_plan **out_plan) {
    if (!out_plan) return set_error(MSA_EINVAL, "out_plan is NULL");
    *out_plan = nullptr;
    uint8_t amap[256];
    int rc = validate_alphabet(alphabet, amap);
    if (rc) return rc;
    const int A = (int)strlen(alphabet);
    msa_plan *p = new (std::nothrow) msa_plan();
    if (!p) return set_error(MSA_ENOMEM, "host allocation failed");
    std::string err;
    rc = make_plan(k, lens, A, kernel_choice, p->hp, err, edge);
    if (rc) {
        delete p;
        return set_error(rc, "%s", err.c_str());
    }
    {
        std::lock_guard<std::mutex> g(settings_mutex());
        p->hp.check_corner = p->hp.kernel != kKernelCol3 || settings().verify_corner ? 1 : 0;
    }
    strncpy(p->alphabet, alphabet, MSA_MAX_ALPHABET);
    p->ws_bytes = plan_layout(p->hp, nullptr, nullptr, &p->reset_bytes);
    cudaError_t e = cudaMalloc(&p->ws, p->ws_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        const size_t bytes = p->ws_bytes;
        delete p;
        return set_error(e == cudaErrorMemoryAllocation ? MSA_ENOMEM : MSA_ECUDA,
                         "cudaMalloc of %zu workspace bytes: %s", bytes, cudaGetErrorString(e));
    }
    size_t rb = 0;
    plan_layout(p->hp, p->ws, &p->pp, &rb);
    ProblemDesc d;
    fill_problem_desc(p->hp, p->pp, 0, d);
    e = cudaMemcpy(p->pp.prob, &d, sizeof d, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->pp.order, p->hp.order.data(), p->hp.order.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->pp.amap, amap, 256, cudaMemcpyHostToDevice);
    // tagged faces start with tag 0, which no execution uses
    if (e == cudaSuccess && tagged_faces(p->hp.kernel)) e = clear_faces(p->hp, p->pp);
    if (e != cudaSuccess) {
        cudaFree(p->ws);
        delete p;
        return cuda_error(e, "plan upload");
    }
    p->grid = persistent_grid(k, p->hp.kernel, p->hp.nunits, A, p->hp.edge);
    *out_plan = p;
    return MSA_OK;
}

}  // namespace msadp

extern "C" {

int msa_plan_execute(msa_plan *plan, const char *d_residues, const int32_t *d_subst, int32_t gap,
                     msa_device_result *d_result, uint8_t *d_masks, void *stream) {
    return msadp::run_plan(plan, d_residues, d_subst, gap, d_result, d_masks, stream, nullptr);
}

}  // extern "C"

namespace msadp {

// msa_plan_execute's steps; with `prune`, its kernels run between the encode
// step and the fill (the plan's problem descriptor then points at prune->skip).
int run_plan(msa_plan *plan, const char *d_residues, const int32_t *d_subst, int32_t gap, msa_device_result *d_result,
             uint8_t *d_masks, void *stream, const PruneDesc *prune) {
    if (!plan || !d_subst || !d_result || (plan->hp.len_sum > 0 && (!d_residues || !d_masks)))
        return set_error(MSA_EINVAL, "NULL plan or device pointer");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t spin_ms, withhold, timing, poison;
    {
        std::lock_guard<std::mutex> g(settings_mutex());
        spin_ms = settings().spin_ms;
        withhold = settings().withhold;
        timing = settings().timing;
        poison = settings().poison_tb;
    }
    plan->last_stream = s;
    cudaEvent_t *ev = nullptr;
    if (timing) {
        if (plan->ev.empty()) {
            plan->ev.assign(4 * msa_plan::kTimedRing, nullptr);
            for (auto &x : plan->ev)
                if (cudaEventCreate(&x) != cudaSuccess) return cuda_error(cudaGetLastError(), "cudaEventCreate");
        }
        ev = &plan->ev[4 * (plan->timed % msa_plan::kTimedRing)];
        cudaEventRecord(ev[0], s);
    }
    cudaError_t e = cudaMemsetAsync(plan->ws, 0, plan->reset_bytes, s);
    if (e == cudaSuccess && poison) e = cudaMemsetAsync(plan->pp.tb, 0xFF, (size_t)plan->hp.tb_dev_bytes, s);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync");
    IODesc io{d_residues, d_subst, d_result, d_masks, gap, 0};
    e = launch_encode(plan->pp.prob, 1, plan->hp.len_sum, nullptr, io, s);
    if (e != cudaSuccess) return cuda_error(e, "encode launch");
    if (prune) {
        e = launch_prune(*prune, prune->greedy != 0, s);
        if (e != cudaSuccess) return cuda_error(e, "pruning kernels");
    }
    LaunchDesc L;
    memset(&L, 0, sizeof L);
    L.probs = plan->pp.prob;
    L.order = plan->pp.order;
    L.ntickets = plan->hp.nunits;
    L.done = plan->pp.done;
    L.ticket = &plan->pp.state->ticket;
    L.err = &plan->pp.state->err;
    L.spin_ns = spin_ms * 1000000LL;
    L.withhold = withhold;
    L.nprob = 1;
    L.tab_ints = plan->hp.A * (plan->hp.A + 1) * 32;  // table plus the sentinel column
    L.corner = plan->hp.check_corner;
    if (tagged_faces(plan->hp.kernel)) {
        if (plan->epoch >= 32767) {  // column kernel tags (epoch << 16) + T would wrap: start over from cleared faces
            e = clear_faces(plan->hp, plan->pp, s);
            if (e != cudaSuccess) return cuda_error(e, "face reset");
            plan->epoch = 0;
        }
        L.epoch = ++plan->epoch;
    }
    if (ev) cudaEventRecord(ev[1], s);
    int rc = launch_fill(plan->hp, L, plan->grid, s);
    if (rc) return rc;
    if (ev) cudaEventRecord(ev[2], s);
    e = launch_traceback(plan->pp.prob, 1, L.err, nullptr, io, s);
    if (e != cudaSuccess) return cuda_error(e, "traceback launch");
    if (ev) {
        cudaEventRecord(ev[3], s);
        plan->timed++;
    }
    return MSA_OK;
}

}  // namespace msadp

extern "C" {

int msa_plan_timings(msa_plan *plan, float out_ms[3]) {
    if (!plan || !out_ms) return set_error(MSA_EINVAL, "NULL plan or output");
    if (!plan->timed) return set_error(MSA_EINVAL, "no timed execution (enable msa_config(\"timing\", 1))");
    const int n = plan->timed < msa_plan::kTimedRing ? plan->timed : msa_plan::kTimedRing;
    const int first = plan->timed - n;
    double acc[3] = {0, 0, 0};
    cudaError_t e = cudaSuccess;
    for (int r = first; r < plan->timed && e == cudaSuccess; ++r) {
        cudaEvent_t *ev = &plan->ev[4 * (r % msa_plan::kTimedRing)];
        e = cudaEventSynchronize(ev[3]);
        for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
            float ms = 0;
            e = cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
            acc[i] += ms;
        }
    }
    plan->timed = 0;
    if (e != cudaSuccess) return cuda_error(e, "event timing");
    for (int i = 0; i < 3; ++i) out_ms[i] = (float)(acc[i] / n);
    return MSA_OK;
}

int msa_plan_read_tb(msa_plan *plan, void *host_dst, int64_t bytes) {
    const HostPlan &hp = plan ? plan->hp : HostPlan();
    if (!plan || !host_dst || bytes < 0 || bytes > hp.tbbytes)
        return set_error(MSA_EINVAL, "bad plan, destination or size");
    cudaError_t e = cudaStreamSynchronize(plan->last_stream);
    if (e != cudaSuccess) return cuda_error(e, "traceback tensor copy");
    if (hp.tb_layout == 0) {
        e = cudaMemcpy(host_dst, plan->pp.tb, (size_t)bytes, cudaMemcpyDeviceToHost);
        return e == cudaSuccess ? MSA_OK : cuda_error(e, "traceback tensor copy");
    }
    std::vector<uint8_t> dev((size_t)hp.tb_dev_bytes);
    e = cudaMemcpy(dev.data(), plan->pp.tb, dev.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "traceback tensor copy");
    uint8_t *out = static_cast<uint8_t *>(host_dst);
    if (hp.tb_layout == 2 || hp.tb_layout == 3) {
        // tile-major device layouts -> row-major host copy, cell by cell: tile t's
        // block of tb_block bytes, the cell at sum_i (local coordinate i) * lst[i]
        const int k = hp.k;
        int x[MSA_MAX_K] = {};
        for (int64_t n = 0; n < hp.cells; ++n) {
            int64_t dst = 0, t = 0, loc = 0;
            for (int i = 0; i < k; ++i) {
                dst += x[i] * hp.tbstride[i];
                const int q = x[i] / hp.E[i];
                t += q * hp.gstride[i];
                loc += (int64_t)(x[i] - q * hp.E[i]) * hp.lst[i];
            }
            if (dst < bytes) out[dst] = dev[(size_t)(t * hp.tb_block + loc)];
            for (int i = k - 1; i >= 0; --i) {  // next cell in row-major order
                if (++x[i] < hp.rho[i]) break;
                x[i] = 0;
            }
        }
        return MSA_OK;
    }
    // column-blocked device layout -> row-major host copy
    const int rho2 = hp.rho[2];
    const int64_t colb = c3::tb_col_bytes(rho2);
    for (int x0 = 0; x0 < hp.rho[0]; ++x0) {
        const int A = x0 / c3::WR, rho = x0 % c3::WR, w = rho / c3::R, r = rho % c3::R;
        for (int x1 = 0; x1 < hp.rho[1]; ++x1) {
            const int B = x1 / 32, l = x1 % 32;
            const uint8_t *col = dev.data() + (int64_t)(A * hp.G[1] + B) * colb;
            const int64_t base = x0 * hp.tbstride[0] + x1 * hp.tbstride[1];
            for (int x2 = 0; x2 < rho2; ++x2) {
                const int64_t dst = base + x2;
                if (dst >= bytes) continue;
                const int T = x2 + l + rho;  // CTA time of the cell
                out[dst] = col[((int64_t)((T + c3::U) * c3::W + w) * 32 + l) * c3::R + r];
            }
        }
    }
    return MSA_OK;
}

int msa_plan_get_info(const msa_plan *plan, msa_plan_info *out) {
    if (!plan || !out) return set_error(MSA_EINVAL, "NULL plan or info");
    memset(out, 0, sizeof *out);
    const HostPlan &hp = plan->hp;
    out->k = hp.k;
    out->alphabet_size = hp.A;
    out->cells = hp.cells;
    for (int i = 0; i < hp.k; ++i) {
        out->tb_strides[i] = hp.tbstride[i];
        out->tile_grid[i] = hp.G[i];
        out->tile_extent[i] = hp.E[i];
    }
    out->tb_bytes = hp.tbbytes;
    out->workspace_bytes = (int64_t)plan->ws_bytes;
    out->tiles = hp.ntiles;
    out->waves = hp.waves;
    out->fill_kernel = hp.kernel;
    out->d_tb = plan->pp.tb;
    return MSA_OK;
}

int msa_plan_destroy(msa_plan *plan) {
    if (!plan) return MSA_OK;
    for (auto &x : plan->ev)
        if (x) cudaEventDestroy(x);
    if (plan->ws) cudaFree(plan->ws);
    delete plan;
    return MSA_OK;
}

// ---------------------------------------------------------------------------
// msa_align: host buffers in, host buffers out, synchronous.

namespace {
std::mutex g_align_mu;
msa_plan *g_cached = nullptr;
char *g_dev_io = nullptr;
size_t g_dev_io_bytes = 0;
char *g_host_io = nullptr;
size_t g_host_io_bytes = 0;

bool same_shape(const msa_plan *p, int k, const int32_t *lens, const char *alphabet, int kernel) {
    if (!p || p->hp.k != k || strcmp(p->alphabet, alphabet) != 0) return false;
    if (p->hp.kernel != choose_kernel(k, lens, p->hp.A, kernel)) return false;
    for (int i = 0; i < k; ++i)
        if (p->hp.lens[i] != lens[i]) return false;
    return true;
}
}  // namespace

int msa_align(int k, const char *const *seqs, const int32_t *lens, const char *alphabet,
              const int32_t *subst, int32_t gap, int32_t *out_score, char *out_alignment) {
    uint8_t amap[256];
    int rc = validate_request(k, seqs, lens, alphabet, subst, amap);
    if (rc) return rc;
    if (!out_score || !out_alignment) return set_error(MSA_EINVAL, "NULL output pointer");
    std::lock_guard<std::mutex> g(g_align_mu);
    int kernel;
    {
        std::lock_guard<std::mutex> g2(settings_mutex());
        kernel = (int)settings().fill_kernel;
    }
    if (!same_shape(g_cached, k, lens, alphabet, kernel)) {
        msa_plan_destroy(g_cached);
        g_cached = nullptr;
        rc = msa_plan_create(k, lens, alphabet, &g_cached);
        if (rc) return rc;
    }
    msa_plan *p = g_cached;
    const int A = p->hp.A;
    const size_t nres = (size_t)p->hp.len_sum;
    const size_t off_sub = (nres + 15) & ~(size_t)15;
    const size_t off_res = (off_sub + (size_t)A * A * 4 + 15) & ~(size_t)15;
    const size_t off_masks = off_res + 16;
    const size_t need = off_masks + nres + 16;
    if (need > g_dev_io_bytes) {
        if (g_dev_io) cudaFree(g_dev_io);
        if (g_host_io) cudaFreeHost(g_host_io);
        g_dev_io = nullptr;
        g_host_io = nullptr;
        g_dev_io_bytes = g_host_io_bytes = 0;
        cudaError_t e = cudaMalloc(&g_dev_io, need * 2);
        if (e == cudaSuccess) e = cudaMallocHost(&g_host_io, need * 2);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(MSA_ENOMEM, "staging allocation: %s", cudaGetErrorString(e));
        }
        g_dev_io_bytes = g_host_io_bytes = need * 2;
    }
    cudaStream_t s = library_stream(&rc);
    if (rc) return rc;
    // gather inputs into pinned staging, one H2D copy
    size_t o = 0;
    for (int i = 0; i < k; ++i) {
        if (lens[i]) memcpy(g_host_io + o, seqs[i], (size_t)lens[i]);
        o += (size_t)lens[i];
    }
    memcpy(g_host_io + off_sub, subst, (size_t)A * A * 4);
    cudaError_t e = cudaMemcpyAsync(g_dev_io, g_host_io, off_res, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_error(e, "H2D copy");
    msa_device_result *d_res = reinterpret_cast<msa_device_result *>(g_dev_io + off_res);
    uint8_t *d_masks = reinterpret_cast<uint8_t *>(g_dev_io + off_masks);
    rc = msa_plan_execute(p, g_dev_io, reinterpret_cast<const int32_t *>(g_dev_io + off_sub), gap, d_res,
                          d_masks, s);
    if (rc) return rc;
    e = cudaMemcpyAsync(g_host_io + off_res, g_dev_io + off_res, 16 + nres, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_error(e, "D2H copy");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
    msa_device_result res;
    memcpy(&res, g_host_io + off_res, sizeof res);
    rc = status_error(res.status);
    if (rc) return rc;
    expand_alignment(k, seqs, lens, reinterpret_cast<const uint8_t *>(g_host_io + off_masks), res.ncols,
                     out_alignment);
    *out_score = res.score;
    return MSA_OK;
}

// ---------------------------------------------------------------------------
// msa_near_optimal: every alignment within delta of the optimum (host buffers).

int msa_near_optimal(int k, const char *const *seqs, const int32_t *lens, const char *alphabet,
                     const int32_t *subst, int32_t gap, int64_t delta, int32_t max_count, uint8_t *out_masks,
                     int32_t *out_ncols, int64_t *out_scores, int32_t *out_count, int32_t *out_more) {
    uint8_t amap[256];
    int rc = validate_request(k, seqs, lens, alphabet, subst, amap);
    if (rc) return rc;
    if (delta < 0 || max_count < 1 || !out_masks || !out_ncols || !out_scores || !out_count || !out_more)
        return set_error(MSA_EINVAL, "delta < 0, max_count < 1 or a NULL output pointer");
    // the generic tile kernel keeps every cell's score, which the walk reads
    msa_plan *plan = nullptr;
    rc = plan_create(k, lens, alphabet, kKernelTiles, -1, &plan);
    if (rc) return rc;
    const int A = plan->hp.A;
    const size_t total = (size_t)plan->hp.len_sum;
    if ((double)max_count * (double)(total + 1) > (double)(1LL << 36)) {
        msa_plan_destroy(plan);
        return set_error(MSA_ETOOBIG, "max_count x (sum of lengths) is beyond the supported output size");
    }
    // one device buffer: inputs, the single-alignment outputs, the enumeration's
    // outputs and its stack
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_res = take(total + 16), o_sub = take((size_t)A * A * 4), o_out = take(sizeof(msa_device_result)),
                 o_mask1 = take(total + 16), o_masks = take((size_t)max_count * total + 16),
                 o_ncols = take((size_t)max_count * 4), o_scores = take((size_t)max_count * 8), o_cm = take(8),
                 o_path = take(total + 16), o_acc = take((total + 1) * 8), o_next = take((total + 1) * 4);
    char *d = nullptr;
    cudaError_t e = cudaMalloc(&d, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        msa_plan_destroy(plan);
        return set_error(MSA_ENOMEM, "near-optimal buffers: %s", cudaGetErrorString(e));
    }
    std::vector<char> res(total + 1);
    size_t o = 0;
    for (int i = 0; i < k; ++i) {
        if (lens[i]) memcpy(res.data() + o, seqs[i], (size_t)lens[i]);
        o += (size_t)lens[i];
    }
    cudaStream_t s = library_stream(&rc);
    if (!rc) {
        e = cudaMemcpy(d + o_res, res.data(), total, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d + o_sub, subst, (size_t)A * A * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = cuda_error(e, "near-optimal inputs");
    }
    if (!rc)
        rc = msa_plan_execute(plan, d + o_res, reinterpret_cast<const int32_t *>(d + o_sub), gap,
                              reinterpret_cast<msa_device_result *>(d + o_out), reinterpret_cast<uint8_t *>(d + o_mask1),
                              s);
    if (!rc) {
        IODesc io{d + o_res, reinterpret_cast<const int32_t *>(d + o_sub),
                  reinterpret_cast<msa_device_result *>(d + o_out), reinterpret_cast<uint8_t *>(d + o_mask1), gap, 0};
        NearOut no{reinterpret_cast<uint8_t *>(d + o_masks), reinterpret_cast<int32_t *>(d + o_ncols),
                   reinterpret_cast<int64_t *>(d + o_scores), reinterpret_cast<int32_t *>(d + o_cm),
                   reinterpret_cast<uint8_t *>(d + o_path), reinterpret_cast<int64_t *>(d + o_acc),
                   reinterpret_cast<int32_t *>(d + o_next)};
        e = launch_near_optimal(plan->pp.prob, io, delta, max_count, no, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_error(e, "near-optimal enumeration");
    }
    msa_device_result r;
    int32_t cm[2] = {0, 0};
    if (!rc) {
        e = cudaMemcpy(&r, d + o_out, sizeof r, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(cm, d + o_cm, 8, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_error(e, "near-optimal results");
    }
    if (!rc) rc = status_error(r.status);
    if (!rc && cm[1] == 2) rc = set_error(MSA_ECUDA, "near-optimal walk found an inconsistent score tensor");
    if (!rc && cm[0] > 0) {
        e = cudaMemcpy(out_masks, d + o_masks, (size_t)cm[0] * total, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(out_ncols, d + o_ncols, (size_t)cm[0] * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(out_scores, d + o_scores, (size_t)cm[0] * 8, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_error(e, "near-optimal results");
    }
    if (!rc) {
        *out_count = cm[0];
        *out_more = cm[1];
    }
    cudaFree(d);
    msa_plan_destroy(plan);
    return rc;
}

// ---------------------------------------------------------------------------
// Exact pruning: msa_align_pruned and msa_tile_bounds (host buffers).

namespace {

// Pruning descriptor for a plan's problem and tile extents E; returns the device
// bytes its tables, rectangle maxima, bounds and flags need (laid out from `base`).
size_t prune_layout(const HostPlan &hp, const int32_t *E, char *base, PruneDesc &D) {
    memset(&D, 0, sizeof D);
    const int k = hp.k;
    D.k = k;
    D.A = hp.A;
    D.len_sum = hp.len_sum;
    int32_t off = 0;
    int64_t nt = 1;
    for (int i = 0; i < k; ++i) {
        D.len[i] = hp.lens[i];
        D.cofs[i] = off;
        off += hp.lens[i];
        D.E[i] = E[i];
        D.G[i] = (hp.rho[i] + E[i] - 1) / E[i];
    }
    for (int i = k - 1; i >= 0; --i) {
        D.gstride[i] = nt;
        nt *= D.G[i];
    }
    D.ntiles = nt;
    int64_t toff = 0, boff = 0;
    for (int i = 0; i < k; ++i)
        for (int j = i + 1; j < k; ++j) {
            D.pi[D.npairs] = i;
            D.pj[D.npairs] = j;
            D.toff[D.npairs] = toff;
            D.boff[D.npairs] = boff;
            toff += 2 * (int64_t)hp.rho[i] * hp.rho[j];
            boff += (int64_t)D.G[i] * D.G[j];
            ++D.npairs;
        }
    D.table_elems = toff;
    D.nblocks = boff;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + o : nullptr;
        o = (o + bytes + 255) & ~(size_t)255;
        return p;
    };
    D.tables = reinterpret_cast<int32_t *>(take((size_t)toff * 4));
    D.blk = reinterpret_cast<int64_t *>(take((size_t)boff * 8));
    D.bound = reinterpret_cast<int64_t *>(take((size_t)nt * 8));
    D.skip = reinterpret_cast<uint8_t *>(take((size_t)nt + 16));
    D.lower = reinterpret_cast<int64_t *>(take(8));
    D.stats = reinterpret_cast<int64_t *>(take(16));
    return o;
}

// Shared set-up: request checks, a generic-tile-kernel plan, the pruning
// descriptor, one device buffer holding inputs, outputs and the pruning arrays.
struct PruneRun {
    msa_plan *plan = nullptr;
    char *d = nullptr;
    PruneDesc D;
    size_t o_res = 0, o_sub = 0, o_out = 0, o_masks = 0, o_prune = 0;
    ~PruneRun() {
        if (d) cudaFree(d);
        if (plan) msa_plan_destroy(plan);
    }
};

int prune_setup(int k, const char *const *seqs, const int32_t *lens, const char *alphabet, const int32_t *subst,
                const int32_t *E, PruneRun &R) {
    uint8_t amap[256];
    int rc = validate_request(k, seqs, lens, alphabet, subst, amap);
    if (rc) return rc;
    for (int i = 0; i < k; ++i)
        if (lens[i] > 16383) return set_error(MSA_ETOOBIG, "pruning takes sequences of at most 16383 residues");
    rc = plan_create(k, lens, alphabet, kKernelTiles, -1, &R.plan);
    if (rc) return rc;
    const HostPlan &hp = R.plan->hp;
    if (E)
        for (int i = 0; i < k; ++i)
            if (E[i] < 1) return set_error(MSA_EINVAL, "tile extent %d of axis %d is below 1", E[i], i);
    const size_t pbytes = prune_layout(hp, E ? E : hp.E, nullptr, R.D);
    const size_t total = (size_t)hp.len_sum, A = (size_t)hp.A;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return o;
    };
    R.o_res = take(total + 16);
    R.o_sub = take(A * A * 4);
    R.o_out = take(sizeof(msa_device_result));
    R.o_masks = take(total + 16);
    R.o_prune = take(pbytes);
    cudaError_t e = cudaMalloc(&R.d, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        R.d = nullptr;
        return set_error(MSA_ENOMEM, "pruning buffers: %s", cudaGetErrorString(e));
    }
    prune_layout(hp, E ? E : hp.E, R.d + R.o_prune, R.D);
    R.D.codes = R.plan->pp.codes;
    R.D.sub = reinterpret_cast<const int32_t *>(R.d + R.o_sub);
    std::vector<char> res(total + 1);
    size_t o = 0;
    for (int i = 0; i < k; ++i) {
        if (lens[i]) memcpy(res.data() + o, seqs[i], (size_t)lens[i]);
        o += (size_t)lens[i];
    }
    e = cudaMemcpy(R.d + R.o_res, res.data(), total, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(R.d + R.o_sub, subst, A * A * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(R.D.stats, 0, 16);
    if (e != cudaSuccess) return cuda_error(e, "pruning inputs");
    return MSA_OK;
}

}  // namespace

int msa_align_pruned(int k, const char *const *seqs, const int32_t *lens, const char *alphabet,
                     const int32_t *subst, int32_t gap, int32_t have_lower_bound, int64_t lower_bound,
                     int32_t *out_score, char *out_alignment, msa_prune_stats *out_stats) {
    if (!out_score || !out_alignment) return set_error(MSA_EINVAL, "NULL output pointer");
    PruneRun R;
    int rc = prune_setup(k, seqs, lens, alphabet, subst, nullptr, R);
    if (rc) return rc;
    const HostPlan &hp = R.plan->hp;
    R.D.gap = gap;
    R.D.greedy = have_lower_bound ? 0 : 1;
    R.D.bound = nullptr;
    cudaError_t e = cudaMemcpy(R.D.lower, &lower_bound, 8, cudaMemcpyHostToDevice);
    // the fill reads the tiles' flags through the plan's problem descriptor
    ProblemDesc pd;
    fill_problem_desc(hp, R.plan->pp, 0, pd);
    pd.skip = R.D.skip;
    if (e == cudaSuccess) e = cudaMemcpy(R.plan->pp.prob, &pd, sizeof pd, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "pruning set-up");
    cudaStream_t s = library_stream(&rc);
    if (rc) return rc;
    msa_device_result *d_res = reinterpret_cast<msa_device_result *>(R.d + R.o_out);
    uint8_t *d_masks = reinterpret_cast<uint8_t *>(R.d + R.o_masks);
    rc = run_plan(R.plan, R.d + R.o_res, R.D.sub, gap, d_res, d_masks, s, &R.D);
    if (rc) return rc;
    e = cudaStreamSynchronize(s);
    msa_device_result res;
    int64_t L = 0, st[2] = {0, 0};
    std::vector<uint8_t> masks((size_t)hp.len_sum + 1);
    if (e == cudaSuccess) e = cudaMemcpy(&res, d_res, sizeof res, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&L, R.D.lower, 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(st, R.D.stats, 16, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(masks.data(), d_masks, (size_t)hp.len_sum, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "pruning results");
    // a bound above the optimum leaves out tiles of every optimal alignment: the
    // corner is then unreachable or its best kept path scores below the bound
    if (have_lower_bound && (res.status != MSA_OK || res.score < lower_bound))
        return set_error(MSA_EINVAL, "lower bound %lld exceeds the optimum", (long long)lower_bound);
    rc = status_error(res.status);
    if (rc) return rc;
    expand_alignment(k, seqs, lens, masks.data(), res.ncols, out_alignment);
    *out_score = res.score;
    if (out_stats) {
        out_stats->lower_bound = L;
        out_stats->tiles = hp.ntiles;
        out_stats->tiles_skipped = st[0];
        out_stats->cells_skipped = st[1];
        out_stats->cells = hp.cells;
    }
    return MSA_OK;
}

int msa_tile_bounds(int k, const char *const *seqs, const int32_t *lens, const char *alphabet,
                    const int32_t *subst, int32_t gap, const int32_t *extents, int64_t *out_bounds) {
    if (!extents || !out_bounds) return set_error(MSA_EINVAL, "NULL extents or output");
    PruneRun R;
    int rc = prune_setup(k, seqs, lens, alphabet, subst, extents, R);
    if (rc) return rc;
    R.D.gap = gap;
    R.D.greedy = 0;
    R.D.skip = nullptr;
    cudaStream_t s = library_stream(&rc);
    if (rc) return rc;
    IODesc io{R.d + R.o_res, R.D.sub, reinterpret_cast<msa_device_result *>(R.d + R.o_out),
              reinterpret_cast<uint8_t *>(R.d + R.o_masks), gap, 0};
    cudaError_t e = cudaMemsetAsync(R.plan->ws, 0, R.plan->reset_bytes, s);
    if (e == cudaSuccess) e = launch_encode(R.plan->pp.prob, 1, R.plan->hp.len_sum, nullptr, io, s);
    if (e == cudaSuccess) e = launch_prune(R.D, false, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    msa_device_result st;
    if (e == cudaSuccess) e = cudaMemcpy(&st, &R.plan->pp.state->istat, sizeof st, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "tile bounds");
    rc = status_error(st.status);
    if (rc) return rc;
    e = cudaMemcpy(out_bounds, R.D.bound, (size_t)R.D.ntiles * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "tile bounds");
    return MSA_OK;
}

// ---------------------------------------------------------------------------
// Host-only planner queries.

int msa_wave_sizes(int k, const int32_t *grid, int64_t *out_sizes, int32_t max_waves, int32_t *out_waves) {
    if (k < 1 || k > MSA_MAX_K || !grid || !out_waves || (max_waves > 0 && !out_sizes))
        return set_error(MSA_EINVAL, "bad arguments");
    for (int i = 0; i < k; ++i)
        if (grid[i] < 1) return set_error(MSA_EINVAL, "grid[%d] < 1", i);
    std::vector<int64_t> w;
    wave_sizes(k, grid, w);
    *out_waves = (int32_t)w.size();
    for (int32_t i = 0; i < max_waves && i < (int32_t)w.size(); ++i) out_sizes[i] = w[i];
    return MSA_OK;
}

int msa_tile_shape(int k, const int32_t *lens, int32_t *out_extent, int32_t *out_grid) {
    if (k < 2 || k > MSA_MAX_K || !lens || !out_extent || !out_grid)
        return set_error(MSA_EINVAL, "bad arguments");
    int kernel;
    {
        std::lock_guard<std::mutex> g(settings_mutex());
        kernel = (int)settings().fill_kernel;
    }
    HostPlan hp;
    std::string err;
    int rc = make_plan(k, lens, 1, kernel, hp, err);
    if (rc) return set_error(rc, "%s", err.c_str());
    for (int i = 0; i < k; ++i) {
        out_extent[i] = hp.E[i];
        out_grid[i] = hp.G[i];
    }
    return MSA_OK;
}

}  // extern "C"

namespace msadp {

void expand_alignment(int k, const char *const *seqs, const int32_t *lens, const uint8_t *masks_rev,
                      int ncols, char *out) {
    int64_t stride = 1;
    for (int i = 0; i < k; ++i) stride += lens[i];
    int32_t pos[MSA_MAX_K] = {};
    for (int c = 0; c < ncols; ++c) {
        const int m = masks_rev[ncols - 1 - c];
        for (int i = 0; i < k; ++i) out[i * stride + c] = ((m >> i) & 1) ? seqs[i][pos[i]++] : '-';
    }
    for (int i = 0; i < k; ++i) out[i * stride + ncols] = '\0';
}

}  // namespace msadp
