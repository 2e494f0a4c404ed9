// Serving: continuous batching of independent alignment requests on one GPU.
//
// msa_submit copies a request, plans it on the host (shape, tile grid, ticket
// order, device footprint) and queues it. One worker thread owns a device arena
// (a single allocation of the configured budget, carved first-fit) and two batch
// slots, each with its own stream. Whenever a slot is free and queued requests
// fit in the arena, the worker admits them in arrival order (up to max_batch per
// batch), packs their descriptors, inputs and merged ticket lists into the slot's
// pinned staging buffer and launches the batch: one copy in, one encode launch
// for all requests, one persistent fill launch per kernel group (k, kernel) whose
// tickets interleave the group's requests wave by wave, one traceback launch, one
// copy out. With use_graphs the sequence is captured into a CUDA graph per slot
// and replayed (updated in place when the sequence of groups repeats). Requests
// that arrive while a batch runs go into the next batch on the other slot, so
// their work overlaps on the device; each request's tensors stay in the arena
// until its batch completes. With batching = 0 every request runs alone, one
// slot, plain launches, in arrival order: the one-at-a-time baseline.
//
// The request tensors are independent problems; a persistent kernel only runs
// tickets that resident CTAs fetched in topological order, so two batches in
// flight never wait on each other.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "api_internal.h"
#include "arena.h"

namespace msadp {
namespace {

constexpr int kSlots = 2;

struct ServeReq {
    uint64_t id = 0;
    int k = 0, A = 0;
    std::vector<std::string> seqs;
    std::vector<int32_t> lens;
    std::string alphabet;
    std::vector<int32_t> subst;
    int32_t gap = 0;
    uint8_t amap[256];
    HostPlan hp;
    int64_t total_len = 0;
    size_t ws_bytes = 0, ws_off = 0;
    bool has_ws = false;
    enum State { kQueued, kRunning, kDone } state = kQueued;
    bool cancelled = false;
    int status = MSA_PENDING;
    int32_t score = 0;
    std::string message;
    std::string alignment;  // k rows at stride total_len + 1
};

struct Group {
    int kernel = 0, k = 0, edge = 0, maxA = 1;
    int first = 0, count = 0;  // slice of the batch's (sorted) requests
    int64_t tickets = 0, tiles = 0;
    size_t order_off = 0, done_off = 0;
    int grid = 1;
};

struct Slot {
    cudaStream_t s = nullptr;
    char *h = nullptr;  // pinned staging, same layout as d
    char *d = nullptr;  // device batch buffer
    size_t cap = 0;
    std::unordered_map<uint64_t, cudaGraphExec_t> execs;  // by sequence of groups
    std::vector<ServeReq *> reqs;
    bool busy = false;
    bool finished = false;  // set by the stream callback
    size_t off_results = 0;
    std::vector<size_t> mask_off;
    int launch_rc = MSA_OK;
};

size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

class Server {
  public:
    int submit(const msa_request *req, uint64_t *out);
    int poll(uint64_t h, int32_t *score, char *alignment);
    int cancel(uint64_t h);
    int drain();
    int wait_any(int64_t timeout_us, uint64_t *out);
    ~Server();

  private:
    void run();
    bool slot_free(int *idx) const;
    int launch(Slot &sl, std::vector<ServeReq *> &batch, const Settings &cfg);
    void complete(Slot &sl);
    void retire(ServeReq *r);  // under mu_
    static void CUDART_CB on_done(void *p);

    std::mutex mu_;
    std::condition_variable cv_, done_cv_;
    std::deque<ServeReq *> queue_;
    std::deque<uint64_t> completed_;  // finished handles, in completion order, not yet reported
    std::unordered_map<uint64_t, ServeReq *> reqs_;
    uint64_t next_id_ = 1;
    std::thread worker_;
    bool started_ = false, stop_ = false;
    bool wake_ = false;  // something changed: a submit, a cancel, a finished batch
    int device_ = 0;
    Arena arena_;
    char *arena_base_ = nullptr;
    size_t arena_bytes_ = 0;
    Slot slots_[kSlots];
    int running_ = 0;
    int32_t epoch_ = 0;
    int init_rc_ = MSA_OK;
    std::string init_msg_;
};

Server &server() {
    static Server s;
    return s;
}

Server::~Server() {
    {
        std::lock_guard<std::mutex> g(mu_);
        stop_ = true;
    }
    cv_.notify_all();
    done_cv_.notify_all();
    if (worker_.joinable()) worker_.join();
    // no stream callback may outlive the server (errors at process teardown are ignored)
    for (auto &sl : slots_)
        if (sl.s) cudaStreamSynchronize(sl.s);
}

void CUDART_CB Server::on_done(void *p) {
    Slot *sl = static_cast<Slot *>(p);
    Server &sv = server();
    {
        std::lock_guard<std::mutex> g(sv.mu_);
        sl->finished = true;
        sv.wake_ = true;
    }
    sv.cv_.notify_all();
}

bool Server::slot_free(int *idx) const {
    for (int i = 0; i < kSlots; ++i)
        if (!slots_[i].busy) {
            *idx = i;
            return true;
        }
    return false;
}

void Server::retire(ServeReq *r) {
    if (r->has_ws) arena_.release(r->ws_off);
    r->has_ws = false;
    r->state = ServeReq::kDone;
    if (r->cancelled) {
        reqs_.erase(r->id);
        delete r;
        return;
    }
    completed_.push_back(r->id);
}

int Server::wait_any(int64_t timeout_us, uint64_t *out) {
    if (!out) return set_error(MSA_EINVAL, "NULL handle pointer");
    std::unique_lock<std::mutex> lk(mu_);
    const auto until = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
    while (true) {
        while (!completed_.empty()) {
            const uint64_t h = completed_.front();
            completed_.pop_front();
            auto it = reqs_.find(h);
            if (it != reqs_.end() && !it->second->cancelled) {  // released handles are skipped
                *out = h;
                return MSA_OK;
            }
        }
        if (stop_ || done_cv_.wait_until(lk, until) == std::cv_status::timeout) {
            if (!completed_.empty()) continue;
            return MSA_PENDING;
        }
    }
}

int Server::submit(const msa_request *req, uint64_t *out) {
    if (!req || !out) return set_error(MSA_EINVAL, "NULL request or handle pointer");
    uint8_t amap[256];
    int rc = validate_request(req->k, req->seqs, req->lens, req->alphabet, req->subst, amap);
    if (rc) return rc;
    Settings cfg;
    {
        std::lock_guard<std::mutex> g(settings_mutex());
        cfg = settings();
    }
    ServeReq *r = new ServeReq();
    r->k = req->k;
    r->A = (int)strlen(req->alphabet);
    r->alphabet = req->alphabet;
    r->gap = req->gap;
    memcpy(r->amap, amap, 256);
    for (int i = 0; i < r->k; ++i) {
        r->lens.push_back(req->lens[i]);
        r->seqs.emplace_back(req->lens[i] ? req->seqs[i] : "", (size_t)req->lens[i]);
        r->total_len += req->lens[i];
    }
    r->subst.assign(req->subst, req->subst + (size_t)r->A * r->A);
    std::string err;
    // the streamed line kernel stays out of serving: its faces would have to be
    // cleared in every reused arena region (8 bytes per cell); the line kernel
    // synchronises by flags instead
    const int choice = cfg.fill_kernel == kKernelStream ? kKernelLines : (int)cfg.fill_kernel;
    rc = make_plan(r->k, r->lens.data(), r->A, choice, r->hp, err, -1, false);
    if (rc) {
        delete r;
        return set_error(rc, "%s", err.c_str());
    }
    r->hp.check_corner = r->hp.kernel != kKernelCol3 || cfg.verify_corner ? 1 : 0;
    size_t rb = 0;
    r->ws_bytes = plan_layout(r->hp, nullptr, nullptr, &rb);
    const size_t budget = (size_t)cfg.budget_mb << 20;
    std::unique_lock<std::mutex> lk(mu_);
    if (started_ && init_rc_ != MSA_OK) {
        delete r;
        return set_error(init_rc_, "serving loop unavailable: %s", init_msg_.c_str());
    }
    const size_t cap = started_ ? arena_bytes_ : budget;  // the arena keeps the budget it started with
    const bool fits = r->ws_bytes + Arena::kAlign <= cap;
    if (!fits) {
        const double mb = r->ws_bytes / 1048576.0;
        delete r;
        return set_error(MSA_ETOOBIG, "request needs %.1f MiB of device memory; the serving budget is %lld MiB",
                         mb, (long long)cfg.budget_mb);
    }
    if (!started_) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) {
            delete r;
            return cuda_error(e, "cudaGetDevice");
        }
        device_ = dev;
        arena_bytes_ = budget;
        started_ = true;
        worker_ = std::thread([this] { run(); });
    }
    r->id = next_id_++;
    reqs_[r->id] = r;
    queue_.push_back(r);
    *out = r->id;
    wake_ = true;
    lk.unlock();
    cv_.notify_all();
    return MSA_OK;
}

int Server::poll(uint64_t h, int32_t *score, char *alignment) {
    std::lock_guard<std::mutex> g(mu_);
    auto it = reqs_.find(h);
    if (it == reqs_.end() || it->second->cancelled) return set_error(MSA_EBADHANDLE, "unknown handle %llu",
                                                                     (unsigned long long)h);
    ServeReq *r = it->second;
    if (r->state != ServeReq::kDone) return MSA_PENDING;
    const int status = r->status;
    if (status == MSA_OK) {
        if (score) *score = r->score;
        if (alignment) memcpy(alignment, r->alignment.data(), r->alignment.size());
    } else {
        set_error(status, "%s", r->message.c_str());
    }
    reqs_.erase(it);
    delete r;
    return status;
}

int Server::cancel(uint64_t h) {
    std::lock_guard<std::mutex> g(mu_);
    auto it = reqs_.find(h);
    if (it == reqs_.end() || it->second->cancelled)
        return set_error(MSA_EBADHANDLE, "unknown handle %llu", (unsigned long long)h);
    ServeReq *r = it->second;
    if (r->state == ServeReq::kQueued) {
        queue_.erase(std::find(queue_.begin(), queue_.end(), r));
        reqs_.erase(it);
        delete r;
    } else if (r->state == ServeReq::kRunning) {
        r->cancelled = true;  // released when its batch completes
    } else {
        reqs_.erase(it);
        delete r;
    }
    wake_ = true;
    cv_.notify_all();
    done_cv_.notify_all();
    return MSA_OK;
}

int Server::drain() {
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] { return stop_ || (queue_.empty() && running_ == 0); });
    return MSA_OK;
}

void Server::run() {
    cudaError_t e = cudaSetDevice(device_);
    if (e == cudaSuccess) e = prepare_kernel_attributes();
    if (e == cudaSuccess) e = cudaMalloc(&arena_base_, arena_bytes_);
    // face entries must start with a tag no launch uses
    if (e == cudaSuccess) e = cudaMemset(arena_base_, 0, arena_bytes_);
    for (int i = 0; i < kSlots && e == cudaSuccess; ++i)
        e = cudaStreamCreateWithFlags(&slots_[i].s, cudaStreamNonBlocking);
    std::unique_lock<std::mutex> lk(mu_);
    if (e != cudaSuccess) {
        cudaGetLastError();
        init_rc_ = e == cudaErrorMemoryAllocation ? MSA_ENOMEM : MSA_ECUDA;
        init_msg_ = std::string("device set-up: ") + cudaGetErrorString(e);
        for (ServeReq *r : queue_) {
            r->status = init_rc_;
            r->message = init_msg_;
            r->state = ServeReq::kDone;
            completed_.push_back(r->id);
        }
        queue_.clear();
        done_cv_.notify_all();
        // keep failing later requests at submit
        cv_.wait(lk, [&] { return stop_; });
        return;
    }
    arena_.reset(arena_bytes_);
    while (true) {
        // sleep until something changed; a queue that cannot advance (no free
        // slot, no room in the arena, or a one-at-a-time run in flight) waits for
        // the next completion instead of spinning
        cv_.wait(lk, [&] { return stop_ || wake_; });
        if (stop_) break;
        wake_ = false;
        int free_idx = -1;
        // completions first: they free memory for admission
        for (auto &sl : slots_) {
            if (!(sl.busy && sl.finished)) continue;
            lk.unlock();
            complete(sl);
            lk.lock();
            for (ServeReq *r : sl.reqs) retire(r);
            sl.reqs.clear();
            sl.busy = false;
            sl.finished = false;
            --running_;
        }
        done_cv_.notify_all();
        Settings cfg;
        {
            std::lock_guard<std::mutex> g(settings_mutex());
            cfg = settings();
        }
        const int max_batch = cfg.batching ? (int)std::max<int64_t>(1, cfg.max_batch) : 1;
        // admission: arrival order, while a slot is free and the arena has room
        while (!queue_.empty() && slot_free(&free_idx) && (cfg.batching || running_ == 0)) {
            std::vector<ServeReq *> batch;
            while (!queue_.empty() && (int)batch.size() < max_batch) {
                ServeReq *r = queue_.front();
                size_t off = 0;
                if (!arena_.alloc(r->ws_bytes, &off)) break;  // wait for memory, keep the order
                r->ws_off = off;
                r->has_ws = true;
                r->state = ServeReq::kRunning;
                queue_.pop_front();
                batch.push_back(r);
            }
            if (batch.empty()) break;
            Slot &sl = slots_[free_idx];
            sl.busy = true;
            sl.finished = false;
            ++running_;
            lk.unlock();
            const int rc = launch(sl, batch, cfg);
            lk.lock();
            if (rc != MSA_OK) {  // nothing was enqueued for this batch
                for (ServeReq *r : sl.reqs) {
                    r->status = rc;
                    r->message = "batch launch failed";
                    retire(r);
                }
                sl.reqs.clear();
                sl.busy = false;
                --running_;
                done_cv_.notify_all();
            }
        }
    }
}

// Pack, enqueue (or capture and replay) one batch on the slot's stream.
int Server::launch(Slot &sl, std::vector<ServeReq *> &batch, const Settings &cfg) {
    // requests grouped by fill kernel and k; each group is one persistent launch
    auto gkey = [](const ServeReq *r) { return (r->hp.kernel * 16 + r->k) * 256 + r->hp.edge; };
    std::stable_sort(batch.begin(), batch.end(),
                     [&](const ServeReq *a, const ServeReq *b) { return gkey(a) < gkey(b); });
    sl.reqs = batch;
    const int n = (int)batch.size();
    std::vector<Group> groups;
    for (int i = 0; i < n; ++i) {
        const HostPlan &hp = batch[i]->hp;
        if (groups.empty() || groups.back().kernel != hp.kernel || groups.back().k != hp.k ||
            groups.back().edge != hp.edge) {
            Group g;
            g.kernel = hp.kernel;
            g.k = hp.k;
            g.edge = hp.edge;
            g.first = i;
            groups.push_back(g);
        }
        Group &g = groups.back();
        g.count++;
        g.tickets += hp.ntiles;
        g.tiles += hp.ntiles;
        g.maxA = std::max(g.maxA, hp.A);
    }
    // batch buffer layout: [in: descs | ios | orders | amaps | residues | tables]
    //                      [zeroed: launch states | istat | done flags] [out: results | masks]
    size_t off = 0;
    const size_t off_desc = off;
    off = a16(off + (size_t)n * sizeof(ProblemDesc));
    const size_t off_io = off;
    off = a16(off + (size_t)n * sizeof(IODesc));
    for (Group &g : groups) {
        g.order_off = off;
        off = a16(off + (size_t)g.tickets * 8);
    }
    const size_t off_amap = off;
    off = a16(off + (size_t)n * 256);
    std::vector<size_t> res_off(n), tab_off(n);
    for (int i = 0; i < n; ++i) {
        res_off[i] = off;
        off = a16(off + (size_t)batch[i]->total_len + 1);
    }
    for (int i = 0; i < n; ++i) {
        tab_off[i] = off;
        off = a16(off + (size_t)batch[i]->A * batch[i]->A * 4);
    }
    const size_t in_bytes = off;
    const size_t off_state = off;
    off = a16(off + groups.size() * sizeof(LaunchState));
    const size_t off_istat = off;
    off = a16(off + (size_t)n * sizeof(msa_device_result));
    for (Group &g : groups) {
        g.done_off = off;
        off = a16(off + (size_t)g.tiles * 4);
    }
    const size_t zero_bytes = off - off_state;
    sl.off_results = off;
    off = a16(off + (size_t)n * sizeof(msa_device_result));
    sl.mask_off.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        sl.mask_off[i] = off;
        off = a16(off + (size_t)batch[i]->total_len + 1);
    }
    const size_t total = off;
    if (total > sl.cap) {
        if (sl.d) cudaFree(sl.d);
        if (sl.h) cudaFreeHost(sl.h);
        sl.d = nullptr;
        sl.h = nullptr;
        sl.cap = 0;
        const size_t cap = total + total / 2 + 4096;
        cudaError_t e = cudaMalloc(&sl.d, cap);
        if (e == cudaSuccess) e = cudaHostAlloc(&sl.h, cap, cudaHostAllocDefault);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(MSA_ENOMEM, "serving batch buffer: %s", cudaGetErrorString(e));
        }
        sl.cap = cap;
        for (auto &x : sl.execs) cudaGraphExecDestroy(x.second);
        sl.execs.clear();
    }
    char *H = sl.h, *D = sl.d;
    ProblemDesc *hdesc = reinterpret_cast<ProblemDesc *>(H + off_desc);
    IODesc *hio = reinterpret_cast<IODesc *>(H + off_io);
    const ProblemDesc *ddesc = reinterpret_cast<const ProblemDesc *>(D + off_desc);
    const IODesc *dio = reinterpret_cast<const IODesc *>(D + off_io);
    LaunchState *dstate = reinterpret_cast<LaunchState *>(D + off_state);
    msa_device_result *distat = reinterpret_cast<msa_device_result *>(D + off_istat);
    msa_device_result *dres = reinterpret_cast<msa_device_result *>(D + sl.off_results);
    int64_t max_ncode = 1;
    bool clear = false;
    for (Group &g : groups) {
        int64_t tile_base = 0;
        for (int j = 0; j < g.count; ++j) {
            const int i = g.first + j;
            ServeReq *r = batch[i];
            PlanPointers pp;
            size_t rb = 0;
            plan_layout(r->hp, arena_base_ + r->ws_off, &pp, &rb);
            fill_problem_desc(r->hp, pp, tile_base, hdesc[i]);
            hdesc[i].clear_faces = tagged_faces(r->hp.kernel) ? 1 : 0;
            clear = clear || tagged_faces(r->hp.kernel);
            tile_base += r->hp.ntiles;
            hdesc[i].amap = reinterpret_cast<uint8_t *>(D + off_amap + (size_t)i * 256);
            hdesc[i].istat = distat + i;
            memcpy(H + off_amap + (size_t)i * 256, r->amap, 256);
            size_t o = res_off[i];
            for (int s = 0; s < r->k; ++s) {
                memcpy(H + o, r->seqs[s].data(), r->seqs[s].size());
                o += r->seqs[s].size();
            }
            memcpy(H + tab_off[i], r->subst.data(), r->subst.size() * 4);
            hio[i] = IODesc{D + res_off[i], reinterpret_cast<const int32_t *>(D + tab_off[i]), dres + i,
                            reinterpret_cast<uint8_t *>(D + sl.mask_off[i]), r->gap, 0};
            max_ncode = std::max<int64_t>(max_ncode, r->hp.len_sum);
        }
        // merged ticket order: every request's own topological order, interleaved
        // wave by wave (tiles: equal tile index sum; columns: equal a + b), each
        // wave taking the requests in batch order -- one pass over the tickets
        uint64_t *ord = reinterpret_cast<uint64_t *>(H + g.order_off);
        size_t nw = 0;
        for (int j = 0; j < g.count; ++j) nw = std::max(nw, batch[g.first + j]->hp.wave_start.size());
        size_t pos = 0;
        for (size_t w = 0; w + 1 < nw; ++w)
            for (int j = 0; j < g.count; ++j) {
                const HostPlan &hp = batch[g.first + j]->hp;
                if (w + 1 >= hp.wave_start.size()) continue;
                for (int64_t t = hp.wave_start[w]; t < hp.wave_start[w + 1]; ++t)
                    ord[pos++] = ((uint64_t)j << 32) | hp.order[(size_t)t];
            }
        if (pos != (size_t)g.tickets) return set_error(MSA_EINVAL, "ticket merge: %zu of %lld tickets", pos,
                                                        (long long)g.tickets);
        g.grid = persistent_grid(g.k, g.kernel, g.tickets, g.maxA, g.edge);  // no occupancy query in a capture
    }
    bool tagged = false;
    for (const Group &g : groups) tagged = tagged || tagged_faces(g.kernel);
    cudaStream_t s = sl.s;
    if (tagged) {
        if (epoch_ >= 32767) {
            // tags (epoch << 16) + T would repeat: clear every face the arena may hold
            for (auto &o : slots_)
                if (&o != &sl && cudaStreamSynchronize(o.s) != cudaSuccess)
                    return cuda_error(cudaGetLastError(), "serving stream");
            cudaError_t e = cudaMemsetAsync(arena_base_, 0, arena_bytes_, s);
            if (e != cudaSuccess) return cuda_error(e, "arena clear");
            epoch_ = 0;
        }
        ++epoch_;
    }
    const bool graphs = cfg.use_graphs && cfg.batching;
    uint64_t sig = 1469598103934665603ull;
    for (const Group &g : groups) sig = (sig ^ (uint64_t)((g.kernel * 16 + g.k) * 256 + g.edge)) * 1099511628211ull;
    cudaError_t e = cudaSuccess;
    if (graphs) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    int rc = MSA_OK;
    if (e == cudaSuccess) e = cudaMemcpyAsync(D, H, in_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(D + off_state, 0, zero_bytes, s);
    if (e == cudaSuccess) e = launch_encode(ddesc, n, max_ncode, dio, IODesc{}, s, clear ? 32 : 1);
    for (size_t gi = 0; gi < groups.size() && e == cudaSuccess; ++gi) {
        const Group &g = groups[gi];
        LaunchDesc L;
        memset(&L, 0, sizeof L);
        L.probs = ddesc + g.first;
        L.order = reinterpret_cast<const uint64_t *>(D + g.order_off);
        L.ntickets = g.tickets;
        L.done = reinterpret_cast<int32_t *>(D + g.done_off);
        L.ticket = &dstate[gi].ticket;
        L.err = &dstate[0].err;
        L.spin_ns = cfg.spin_ms * 1000000LL;
        L.withhold = -1;
        L.nprob = g.count;
        L.tab_ints = g.maxA * (g.maxA + 1) * 32;
        L.epoch = epoch_;
        for (int j = 0; j < g.count; ++j) L.corner |= batch[g.first + j]->hp.check_corner;
        e = g.kernel == kKernelCol3    ? launch_fill_col3(L, g.grid, col3_smem_bytes(g.maxA), s)
          : g.kernel == kKernelBand2 ? launch_fill_band2(L, g.grid, s)
          : g.kernel == kKernelLines ? launch_fill_lines(g.k, g.edge, L, g.grid, s)
                                     : launch_fill_tiles(g.k, g.edge, L, g.grid, s);
    }
    if (e == cudaSuccess) e = launch_traceback(ddesc, n, &dstate[0].err, dio, IODesc{}, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(H + sl.off_results, D + sl.off_results, total - sl.off_results, cudaMemcpyDeviceToHost,
                            s);
    if (graphs) {
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(s, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) {
            cudaGraphExec_t &ex = sl.execs[sig];
            bool ready = false;
            if (ex) {
                cudaGraphExecUpdateResultInfo info;
                ready = cudaGraphExecUpdate(ex, graph, &info) == cudaSuccess;
                if (!ready) {
                    cudaGetLastError();
                    cudaGraphExecDestroy(ex);
                    ex = nullptr;
                }
            }
            if (!ready) e = cudaGraphInstantiate(&ex, graph, 0);
            if (e == cudaSuccess) e = cudaGraphLaunch(ex, s);
        }
        if (graph) cudaGraphDestroy(graph);
    }
    if (e == cudaSuccess) e = cudaLaunchHostFunc(s, on_done, &sl);
    if (e != cudaSuccess) {
        rc = cuda_error(e, "serving batch launch");
        cudaStreamSynchronize(s);
        cudaGetLastError();
    }
    return rc;
}

// Host side of a finished batch: read the copied-out results, expand alignments.
void Server::complete(Slot &sl) {
    const msa_device_result *res = reinterpret_cast<const msa_device_result *>(sl.h + sl.off_results);
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
        ServeReq *r = sl.reqs[i];
        const msa_device_result &x = res[i];
        if (x.status != MSA_OK) {
            r->status = x.status == MSA_EINVAL || x.status == MSA_ETOOBIG || x.status == MSA_ETIMEOUT ? x.status
                                                                                                       : MSA_ECUDA;
            r->message = x.status == MSA_EINVAL    ? "device check: residue outside the alphabet or non-symmetric table"
                         : x.status == MSA_ETOOBIG ? "scores could leave the exact int32 range for this table and gap"
                         : x.status == MSA_ETIMEOUT ? "a device dependency wait exceeded its limit; the fill stopped"
                                                    : "device traceback found an inconsistent traceback tensor";
            continue;
        }
        std::vector<const char *> sp(r->k);
        for (int s = 0; s < r->k; ++s) sp[s] = r->seqs[s].data();
        r->alignment.assign((size_t)r->k * (size_t)(r->total_len + 1), '\0');
        expand_alignment(r->k, sp.data(), r->lens.data(), reinterpret_cast<const uint8_t *>(sl.h + sl.mask_off[i]),
                         x.ncols, &r->alignment[0]);
        r->score = x.score;
        r->status = MSA_OK;
    }
}

}  // namespace
}  // namespace msadp

using namespace msadp;

extern "C" {

int msa_submit(const msa_request *req, uint64_t *out_handle) { return server().submit(req, out_handle); }

int msa_poll(uint64_t handle, int32_t *out_score, char *out_alignment) {
    return server().poll(handle, out_score, out_alignment);
}

int msa_cancel(uint64_t handle) { return server().cancel(handle); }

int msa_drain(void) { return server().drain(); }

int msa_wait_any(int64_t timeout_us, uint64_t *out_handle) { return server().wait_any(timeout_us, out_handle); }

}  // extern "C"
