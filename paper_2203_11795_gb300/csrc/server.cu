// Serving loop over whole transforms (fftu_serve.h): per-key queues, memory-budget admission,
// same-key batching into one persistent launch, CUDA graph replay, completion polling.
//
// Data structures
//   Key       (d, n, dtype, dir): one resident plan (twiddle tables) shared by every batch of the key.
//   Instance  a resident launch of k requests of one key: device slots for k inputs and k outputs,
//             its own fftu_batch (the batch's counters are per launch, so an instance runs one
//             launch at a time) or, for large requests, its own plan (a plan's workspace is per
//             launch too), a stream, a completion event and, once used with page-locked buffers,
//             an instantiated graph whose copy nodes are re-pointed at each replay.
// The server thread alone touches keys and instances; submitters and pollers share two
// mutex-protected queues with it.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "fftu.h"
#include "fftu_serve.h"

namespace fftu {
void record_error(const char *msg);
}

namespace {

using Clock = std::chrono::steady_clock;

struct Key {
    int d = 0;
    int64_t n[FFTU_MAX_DIMS] = {};
    int dtype = 0, dir = 0;
    bool operator<(const Key &o) const {
        if (d != o.d) return d < o.d;
        if (dtype != o.dtype) return dtype < o.dtype;
        if (dir != o.dir) return dir < o.dir;
        for (int l = 0; l < d; ++l)
            if (n[l] != o.n[l]) return n[l] < o.n[l];
        return false;
    }
};

struct WarmJob;

struct Req {
    fftu_request r;
    double t_submit = 0;
    std::shared_ptr<WarmJob> warm;  // set: not a transform but a warm-up of the key (fftu_server_warm)
};

// A warm-up request: create the key's instances for every batch size up to max_k and their graphs,
// then signal the waiting caller.
struct WarmJob {
    int max_k = 1;
    std::mutex mu;
    std::condition_variable cv;
    bool done = false;
    fftu_status status = FFTU_OK;
    int prepared = 0;
};

struct KeyState;
struct GraphBuild;

struct Instance {
    KeyState *ks = nullptr;
    int k = 0;
    bool large = false;
    void *dev = nullptr;  // [k inputs][k outputs]
    size_t slot_bytes = 0;
    size_t bytes = 0;     // device bytes charged to the budget
    fftu_batch batch = nullptr;
    fftu_handle own_plan = nullptr;
    int launches = 0;     // kernels per use
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<cudaGraphNode_t> h2d, d2h;
    bool graph_failed = false;
    bool building = false;             // a graph for it is being built off the server thread
    int piece_mib = 0;
    bool busy = false;
    std::vector<Req> reqs;
    double t_start = 0;
    uint64_t last_used = 0;

    void *in_slot(int i) const { return static_cast<char *>(dev) + (size_t)i * slot_bytes; }
    void *out_slot(int i) const { return static_cast<char *>(dev) + (size_t)(k + i) * slot_bytes; }
};

struct KeyState {
    Key key;
    int64_t N = 0;
    size_t esize = 0;
    fftu_handle plan = nullptr;  // shared by the batched instances
    size_t plan_bytes = 0;
    bool solo = false;           // requests run alone through their own plan (large, or not batchable)
    std::deque<Req> pending;
    std::vector<std::unique_ptr<Instance>> inst;
    uint64_t last_used = 0;
};

}  // namespace

struct fftu_server_st {
    fftu_server_config cfg;
    int device = 0;
    Clock::time_point t0;
    std::vector<cudaStream_t> streams;  // [0, split): batched instances, [split, size): solo ones
    int split = 0;
    int next_small = 0, next_large = 0;

    std::mutex in_mu;              // inbox and counters shared with submitters
    std::condition_variable in_cv;
    std::deque<Req> inbox;
    std::mutex out_mu;             // completions shared with pollers
    std::deque<fftu_completion> outbox;
    std::atomic<int64_t> outstanding{0};
    std::atomic<bool> stop{false};

    std::mutex stats_mu;
    fftu_server_stats stats;

    // graph builder thread: instantiating a graph takes milliseconds, so it runs beside the server
    // thread, which keeps dispatching (plain copies) until the graph arrives
    std::thread builder;
    std::mutex b_mu;
    std::condition_variable b_cv;
    std::deque<GraphBuild *> b_jobs;
    std::vector<GraphBuild *> b_done;
    bool b_stop = false;
    cudaStream_t b_stream = nullptr;
    cudaStream_t w_stream = nullptr;  // graphs built by fftu_server_warm on the server thread

    std::map<Key, std::unique_ptr<KeyState>> keys;  // server thread only
    size_t used = 0;
    uint64_t tick = 0;
    std::thread thread;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

int64_t elems(const Key &k) {
    int64_t N = 1;
    for (int l = 0; l < k.d; ++l) N *= k.n[l];
    return N;
}

void complete(fftu_server_st *S, const Req &q, int status, int batch_size, double t_start) {
    fftu_completion c;
    c.tag = q.r.tag;
    c.status = status;
    c.batch_size = batch_size;
    c.submit_s = q.t_submit;
    c.start_s = t_start;
    c.done_s = S->now();
    {
        std::lock_guard<std::mutex> lk(S->out_mu);
        S->outbox.push_back(c);
    }
    {
        std::lock_guard<std::mutex> lk(S->stats_mu);
        S->stats.completed++;
        if (status != FFTU_OK && batch_size == 0) S->stats.rejected++;
    }
    S->outstanding.fetch_sub(1);
}

void update_bytes(fftu_server_st *S) {
    std::lock_guard<std::mutex> lk(S->stats_mu);
    S->stats.bytes_in_use = (int64_t)S->used;
    S->stats.peak_bytes = std::max(S->stats.peak_bytes, (int64_t)S->used);
    int64_t ni = 0, np = 0;
    for (auto &kv : S->keys) {
        ni += (int64_t)kv.second->inst.size();
        np += kv.second->plan ? 1 : 0;
        for (auto &in : kv.second->inst) np += in->own_plan ? 1 : 0;
    }
    S->stats.instances = ni;
    S->stats.plans = np;
}

size_t plan_device_bytes(fftu_handle h) {
    fftu_info info;
    if (fftu_plan_info(h, &info) != FFTU_OK) return 0;
    return (size_t)(info.table_bytes + info.workspace_bytes) + 256;
}

int plan_launches(fftu_handle h) {
    fftu_info info;
    if (fftu_plan_info(h, &info) != FFTU_OK) return 0;
    return info.launches_phase_a + info.launches_phase_b;
}

void note_cuda_error(fftu_server_st *S, cudaError_t e, int site) {
    std::lock_guard<std::mutex> lk(S->stats_mu);
    S->stats.last_cuda_error = (int)e;
    S->stats.last_error_site = site;
}

void destroy_instance(fftu_server_st *S, Instance *in) {
    if (in->gexec) cudaGraphExecDestroy(in->gexec);
    if (in->graph) cudaGraphDestroy(in->graph);
    if (in->batch) fftu_batch_destroy(in->batch);
    if (in->own_plan) fftu_destroy(in->own_plan);
    if (in->done) cudaEventDestroy(in->done);
    // stream-ordered: freed after the instance's last use on its stream, without a device-wide wait
    if (in->dev) cudaFreeAsync(in->dev, in->stream);
    S->used -= in->bytes;
}

// Free idle instances and unused plans, least recently used first, until `need` more bytes fit.
bool make_room(fftu_server_st *S, size_t need, const KeyState *keep) {
    const size_t budget = (size_t)S->cfg.device_bytes;
    while (S->used + need > budget) {
        Instance *victim = nullptr;
        KeyState *vks = nullptr;
        KeyState *plan_victim = nullptr;
        for (auto &kv : S->keys) {
            KeyState *ks = kv.second.get();
            for (auto &in : ks->inst)
                if (!in->busy && !in->building && (!victim || in->last_used < victim->last_used)) {
                    victim = in.get();
                    vks = ks;
                }
            if (ks != keep && ks->plan && ks->inst.empty() && ks->pending.empty() &&
                (!plan_victim || ks->last_used < plan_victim->last_used))
                plan_victim = ks;
        }
        if (victim) {
            destroy_instance(S, victim);
            auto &v = vks->inst;
            v.erase(std::remove_if(v.begin(), v.end(), [&](const std::unique_ptr<Instance> &p) { return p.get() == victim; }),
                    v.end());
        } else if (plan_victim) {
            fftu_destroy(plan_victim->plan);
            plan_victim->plan = nullptr;
            S->used -= plan_victim->plan_bytes;
            plan_victim->plan_bytes = 0;
        } else {
            return false;
        }
        std::lock_guard<std::mutex> lk(S->stats_mu);
        S->stats.evictions++;
    }
    return true;
}

// The resident plan of a key (batched requests); nullptr if it does not fit now or fails.
fftu_status ensure_plan(fftu_server_st *S, KeyState *ks) {
    if (ks->plan) return FFTU_OK;
    // the batch kernel runs the plan's in-place passes and never its workspace: the plan allocates none
    fftu_options opts;
    std::memset(&opts, 0, sizeof(opts));
    opts.workspace_mode = FFTU_WORKSPACE_CALLER;
    fftu_handle h = nullptr;
    fftu_status st = fftu_plan_ex(ks->key.d, ks->key.n, nullptr, (fftu_dtype)ks->key.dtype, (fftu_dir)ks->key.dir,
                                  &opts, &h);
    if (st != FFTU_OK) return st;
    const size_t b = plan_device_bytes(h);
    if (S->used + b > (size_t)S->cfg.device_bytes && !make_room(S, b, ks)) {
        fftu_destroy(h);
        return FFTU_ERR_NOMEM;
    }
    ks->plan = h;
    ks->plan_bytes = b;
    S->used += b;
    return FFTU_OK;
}

Instance *new_instance_impl(fftu_server_st *S, KeyState *ks, int k, bool large, fftu_status *err);

// A new instance of k requests of ks; nullptr when the budget cannot hold it right now.
Instance *new_instance(fftu_server_st *S, KeyState *ks, int k, bool large, fftu_status *err) {
    const double t0 = S->now();
    Instance *in = new_instance_impl(S, ks, k, large, err);
    const double dt = S->now() - t0;
    std::lock_guard<std::mutex> lk(S->stats_mu);
    S->stats.creation_s += dt;
    if (in) S->stats.instance_creations++;
    return in;
}

Instance *new_instance_impl(fftu_server_st *S, KeyState *ks, int k, bool large, fftu_status *err) {
    *err = FFTU_OK;
    auto in = std::make_unique<Instance>();
    in->ks = ks;
    in->k = k;
    in->large = large;
    in->piece_mib = S->cfg.copy_piece_mib;
    in->slot_bytes = ((size_t)ks->N * ks->esize + 255) / 256 * 256;
    size_t bytes = 2 * (size_t)k * in->slot_bytes;
    if (large) {
        fftu_status st = fftu_plan(ks->key.d, ks->key.n, nullptr, (fftu_dtype)ks->key.dtype, (fftu_dir)ks->key.dir,
                                   &in->own_plan);
        if (st != FFTU_OK) {
            *err = st;
            return nullptr;
        }
        bytes += plan_device_bytes(in->own_plan);
        in->launches = plan_launches(in->own_plan);
    } else {
        fftu_status st = ensure_plan(S, ks);
        if (st != FFTU_OK) {
            *err = st == FFTU_ERR_NOMEM ? FFTU_OK : st;  // no room yet: wait
            return nullptr;
        }
        bytes += 4096 * 4;  // the batch's job table and counters
        in->launches = 1;
    }
    if (S->used + bytes > (size_t)S->cfg.device_bytes && !make_room(S, bytes, ks)) {
        if (in->own_plan) fftu_destroy(in->own_plan);
        return nullptr;
    }
    // solo (large) requests get their own low-priority streams, so that a small batch never waits in a
    // stream behind a large request's copies and its blocks are scheduled first
    const int ns = (int)S->streams.size();
    if (large && S->split < ns) {
        in->stream = S->streams[S->split + S->next_large];
        S->next_large = (S->next_large + 1) % (ns - S->split);
    } else {
        in->stream = S->streams[S->next_small];
        S->next_small = (S->next_small + 1) % (S->split > 0 ? S->split : ns);
    }
    // stream-ordered allocation from the device's memory pool: no device-wide synchronisation when an
    // instance is created or evicted
    if (cudaMallocAsync(&in->dev, 2 * (size_t)k * in->slot_bytes, in->stream) != cudaSuccess) {
        cudaGetLastError();
        in->dev = nullptr;
        if (in->own_plan) fftu_destroy(in->own_plan);
        return nullptr;
    }
    if (!large) {
        std::vector<fftu_handle> hs(k, ks->plan);
        fftu_status st = fftu_batch_create(k, hs.data(), &in->batch);
        if (st != FFTU_OK) {
            cudaFreeAsync(in->dev, in->stream);
            if (st == FFTU_ERR_UNSUPPORTED) {
                ks->solo = true;  // e.g. long lines: phase A alternates with a workspace
                return nullptr;   // the caller retries as a solo request
            }
            *err = st;
            return nullptr;
        }
    }
    cudaEventCreateWithFlags(&in->done, cudaEventDisableTiming);
    in->bytes = bytes;
    S->used += bytes;
    Instance *raw = in.get();
    ks->inst.push_back(std::move(in));
    return raw;
}

fftu_status compute(Instance *in, cudaStream_t st) {
    if (in->large) return fftu_exec(in->own_plan, in->in_slot(0), in->out_slot(0), st);
    std::vector<const void *> ins(in->k);
    std::vector<void *> outs(in->k);
    for (int i = 0; i < in->k; ++i) {
        ins[i] = in->in_slot(i);
        outs[i] = in->out_slot(i);
    }
    return fftu_batch_exec(in->batch, ins.data(), outs.data(), st);
}

// Host copies of one array: one piece, or pieces of copy_piece_mib MiB issued in order.
size_t piece_bytes(const Instance *in, size_t bytes) {
    return in->piece_mib > 0 ? std::min(bytes, (size_t)in->piece_mib << 20) : bytes;
}

int pieces(const Instance *in, size_t bytes) {
    const size_t pb = piece_bytes(in, bytes);
    return (int)((bytes + pb - 1) / pb);
}

// A graph of one instance's launch (copies in, transform, copies out), built off the server thread.
struct GraphBuild {
    Instance *in = nullptr;
    std::vector<const void *> hin;  // host addresses the copy nodes start with (re-pointed at each replay)
    std::vector<void *> hout;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<cudaGraphNode_t> h2d, d2h;
    cudaError_t error = cudaSuccess;
    bool ok = false;
};

// Capture the transform on `cs` (a stream of the builder's own) and instantiate the graph.
void build_graph(GraphBuild &b, cudaStream_t cs) {
    Instance *in = b.in;
    const size_t bytes = (size_t)in->ks->N * in->ks->esize;
    const size_t piece = piece_bytes(in, bytes);
    const int c = pieces(in, bytes);
    cudaGraph_t g = nullptr, child = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) {
        b.error = cudaGetLastError();
        return;
    }
    bool ok = true;
    b.h2d.assign((size_t)in->k * c, nullptr);
    b.d2h.assign((size_t)in->k * c, nullptr);
    for (int i = 0; ok && i < in->k; ++i)
        for (int j = 0; ok && j < c; ++j) {
            const size_t off = (size_t)j * piece, len = std::min(piece, bytes - off);
            cudaGraphNode_t *prev = j > 0 ? &b.h2d[(size_t)i * c + j - 1] : nullptr;
            ok = cudaGraphAddMemcpyNode1D(&b.h2d[(size_t)i * c + j], g, prev, prev ? 1 : 0,
                                          static_cast<char *>(in->in_slot(i)) + off,
                                          static_cast<const char *>(b.hin[i]) + off, len,
                                          cudaMemcpyHostToDevice) == cudaSuccess;
        }
    if (ok) {
        ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            const fftu_status st = compute(in, cs);
            ok = cudaStreamEndCapture(cs, &child) == cudaSuccess && st == FFTU_OK && child;
        }
    }
    cudaGraphNode_t cn = nullptr;
    if (ok) ok = cudaGraphAddChildGraphNode(&cn, g, b.h2d.data(), b.h2d.size(), child) == cudaSuccess;
    for (int i = 0; ok && i < in->k; ++i)
        for (int j = 0; ok && j < c; ++j) {
            const size_t off = (size_t)j * piece, len = std::min(piece, bytes - off);
            cudaGraphNode_t *prev = j > 0 ? &b.d2h[(size_t)i * c + j - 1] : &cn;
            ok = cudaGraphAddMemcpyNode1D(&b.d2h[(size_t)i * c + j], g, prev, 1,
                                          static_cast<char *>(b.hout[i]) + off,
                                          static_cast<const char *>(in->out_slot(i)) + off, len,
                                          cudaMemcpyDeviceToHost) == cudaSuccess;
        }
    if (child) cudaGraphDestroy(child);
    if (ok) ok = cudaGraphInstantiate(&b.gexec, g, 0) == cudaSuccess;
    // upload now, on the builder's stream, so that the first replay does not pay for it
    if (ok) ok = cudaGraphUpload(b.gexec, cs) == cudaSuccess && cudaStreamSynchronize(cs) == cudaSuccess;
    if (!ok) {
        b.error = cudaGetLastError();
        if (b.gexec) cudaGraphExecDestroy(b.gexec);
        b.gexec = nullptr;
        cudaGraphDestroy(g);
        return;
    }
    b.graph = g;
    b.ok = true;
}

bool page_locked(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// Issue one use of an instance for its reqs; on failure every request completes with the error.
void launch(fftu_server_st *S, Instance *in) {
    const size_t bytes = (size_t)in->ks->N * in->ks->esize;
    in->busy = true;
    in->t_start = S->now();
    struct LaunchTimer {  // longest host time of one launch, in the stats
        fftu_server_st *S;
        double t0;
        ~LaunchTimer() {
            const double dt = S->now() - t0;
            std::lock_guard<std::mutex> lk(S->stats_mu);
            if (dt > S->stats.max_launch_s) S->stats.max_launch_s = dt;
        }
    } timer{S, in->t_start};
    in->last_used = ++S->tick;
    in->ks->last_used = S->tick;
    bool locked = S->cfg.use_graphs && !in->graph_failed;
    for (int i = 0; locked && i < in->k; ++i) locked = page_locked(in->reqs[i].r.in) && page_locked(in->reqs[i].r.out);
    fftu_status st = FFTU_OK;
    bool graphed = false;
    if (locked && !in->gexec && !in->building) {  // first use with page-locked buffers: build a graph
        auto *job = new GraphBuild();
        job->in = in;
        for (int i = 0; i < in->k; ++i) {
            job->hin.push_back(in->reqs[i].r.in);
            job->hout.push_back(in->reqs[i].r.out);
        }
        in->building = true;
        {
            std::lock_guard<std::mutex> lk(S->b_mu);
            S->b_jobs.push_back(job);
        }
        S->b_cv.notify_one();
    }
    if (locked) {
        if (in->gexec) {
            bool ok = true;
            const size_t piece = piece_bytes(in, bytes);
            const int c = pieces(in, bytes);
            for (int i = 0; ok && i < in->k; ++i)
                for (int j = 0; ok && j < c; ++j) {
                    const size_t off = (size_t)j * piece, len = std::min(piece, bytes - off);
                    const size_t q = (size_t)i * c + j;
                    ok = cudaGraphExecMemcpyNodeSetParams1D(in->gexec, in->h2d[q],
                                                           static_cast<char *>(in->in_slot(i)) + off,
                                                           static_cast<const char *>(in->reqs[i].r.in) + off, len,
                                                           cudaMemcpyHostToDevice) == cudaSuccess &&
                         cudaGraphExecMemcpyNodeSetParams1D(in->gexec, in->d2h[q],
                                                           static_cast<char *>(in->reqs[i].r.out) + off,
                                                           static_cast<const char *>(in->out_slot(i)) + off, len,
                                                           cudaMemcpyDeviceToHost) == cudaSuccess;
                }
            if (ok) ok = cudaGraphLaunch(in->gexec, in->stream) == cudaSuccess;
            if (ok) {
                graphed = true;
            } else {
                note_cuda_error(S, cudaGetLastError(), 7);
                in->graph_failed = true;
            }
        }
    }
    if (!graphed) {
        for (int i = 0; st == FFTU_OK && i < in->k; ++i) {
            const cudaError_t e = cudaMemcpyAsync(in->in_slot(i), in->reqs[i].r.in, bytes, cudaMemcpyHostToDevice,
                                                  in->stream);
            if (e != cudaSuccess) {
                note_cuda_error(S, e, 1);
                st = FFTU_ERR_CUDA;
            }
        }
        if (st == FFTU_OK) {
            st = compute(in, in->stream);
            if (st != FFTU_OK) note_cuda_error(S, cudaPeekAtLastError(), 2);
        }
        for (int i = 0; st == FFTU_OK && i < in->k; ++i) {
            const cudaError_t e = cudaMemcpyAsync(in->reqs[i].r.out, in->out_slot(i), bytes, cudaMemcpyDeviceToHost,
                                                  in->stream);
            if (e != cudaSuccess) {
                note_cuda_error(S, e, 3);
                st = FFTU_ERR_CUDA;
            }
        }
    }
    if (st == FFTU_OK) {
        const cudaError_t e = cudaEventRecord(in->done, in->stream);
        if (e != cudaSuccess) {
            note_cuda_error(S, e, 4);
            st = FFTU_ERR_CUDA;
        }
    }
    {
        std::lock_guard<std::mutex> lk(S->stats_mu);
        S->stats.batches++;
        S->stats.kernel_launches += in->launches;
        if (graphed) S->stats.graph_replays++;
        else S->stats.direct_launches++;
        S->stats.bytes_h2d += (int64_t)(bytes * in->k);
        S->stats.bytes_d2h += (int64_t)(bytes * in->k);
    }
    if (st != FFTU_OK) {
        cudaGetLastError();
        cudaStreamSynchronize(in->stream);
        for (auto &q : in->reqs) complete(S, q, st, in->k, in->t_start);
        in->reqs.clear();
        in->busy = false;
    }
}

// Completed instances: stamp their requests and free the instance for reuse.
bool reap(fftu_server_st *S) {
    bool any = false;
    for (auto &kv : S->keys)
        for (auto &in : kv.second->inst) {
            if (!in->busy) continue;
            const cudaError_t e = cudaEventQuery(in->done);
            if (e == cudaErrorNotReady) continue;
            int status = e == cudaSuccess ? FFTU_OK : FFTU_ERR_CUDA;
            if (e != cudaSuccess) {
                note_cuda_error(S, e, 5);
                cudaGetLastError();
            }
            for (auto &q : in->reqs) complete(S, q, status, in->k, in->t_start);
            in->reqs.clear();
            in->busy = false;
            any = true;
        }
    return any;
}

bool any_busy(fftu_server_st *S);

int pow2_floor(int v) {
    int k = 1;
    while (2 * k <= v) k *= 2;
    return k;
}

// Start batches for every key with queued requests, oldest head first.
bool dispatch(fftu_server_st *S) {
    std::vector<KeyState *> order;
    for (auto &kv : S->keys)
        if (!kv.second->pending.empty()) order.push_back(kv.second.get());
    std::sort(order.begin(), order.end(),
              [](const KeyState *a, const KeyState *b) { return a->pending.front().t_submit < b->pending.front().t_submit; });
    bool any = false;
    int inflight = 0, inflight_large = 0;
    for (auto &kv : S->keys)
        for (auto &in : kv.second->inst) {
            inflight += in->busy ? 1 : 0;
            inflight_large += in->busy && in->large ? 1 : 0;
        }
    // at most max_inflight_solo solo launches: more would only queue inside the solo streams (holding
    // instances, deepening the device's queue and delaying the small requests' copies); they wait here
    const int large_cap = S->cfg.max_inflight_solo;
    for (KeyState *ks : order) {
        if (ks->N >= S->cfg.large_elems) ks->solo = true;
        while (!ks->pending.empty() && inflight < S->cfg.max_inflight) {
            const bool large = ks->solo;
            if (large && inflight_large >= large_cap) break;
            const int k = large ? 1 : pow2_floor(std::min<int>((int)ks->pending.size(), S->cfg.max_batch));
            Instance *in = nullptr;
            for (auto &c : ks->inst)
                if (!c->busy && c->k == k && c->large == large) {
                    in = c.get();
                    break;
                }
            fftu_status err = FFTU_OK;
            if (!in) in = new_instance(S, ks, k, large, &err);
            if (!in && !large && ks->solo) continue;  // not batchable: go again as solo requests
            if (!in && err == FFTU_ERR_NOMEM && any_busy(S)) err = FFTU_OK;  // wait for memory
            if (!in) {
                if (err != FFTU_OK) {  // the key cannot run at all
                    while (!ks->pending.empty()) {
                        complete(S, ks->pending.front(), err, 0, 0);
                        ks->pending.pop_front();
                    }
                }
                break;  // wait for memory
            }
            in->reqs.assign(ks->pending.begin(), ks->pending.begin() + k);
            ks->pending.erase(ks->pending.begin(), ks->pending.begin() + k);
            launch(S, in);
            inflight += in->busy ? 1 : 0;
            inflight_large += in->busy && large ? 1 : 0;
            any = true;
        }
    }
    update_bytes(S);
    return any;
}

// Warm-up of one key on the server thread: an idle instance for every power-of-two batch size up to
// the job's max_k (one solo instance for large keys) and its graph, built here on the server's warm
// stream with the request's host buffers as placeholders (every replay re-points the copies).
void warm_key(fftu_server_st *S, KeyState *ks, const Req &q) {
    WarmJob &job = *q.warm;
    fftu_status status = FFTU_OK;
    int prepared = 0;
    if (ks->N >= S->cfg.large_elems) ks->solo = true;
    const int kmax = ks->solo ? 1 : std::max(1, std::min(job.max_k, S->cfg.max_batch));
    for (int k = 1, copy = 0; k <= kmax && status == FFTU_OK;) {
        const bool large = ks->solo;
        // an instance runs one launch at a time, so launches of one key that overlap each take their own:
        // one batch instance of each size per batched stream, max_inflight_solo solo instances
        const int copies = large ? S->cfg.max_inflight_solo : std::max(1, S->split);
        Instance *in = nullptr;
        int have = 0;
        for (auto &c : ks->inst)
            if (c->k == k && c->large == large && have++ == copy) in = c.get();
        fftu_status err = FFTU_OK;
        if (!in) in = new_instance(S, ks, k, large, &err);
        if (!in) {
            if (!large && ks->solo) {  // not batchable: warm the solo path instead
                k = 1;
                copy = 0;
                continue;
            }
            status = err != FFTU_OK ? err : FFTU_ERR_NOMEM;
            break;
        }
        if (S->cfg.use_graphs && !in->gexec && !in->graph_failed && !in->building && page_locked(q.r.in) &&
            page_locked(q.r.out)) {
            GraphBuild b;
            b.in = in;
            b.hin.assign(in->k, q.r.in);
            b.hout.assign(in->k, q.r.out);
            build_graph(b, S->w_stream);
            if (b.ok) {
                in->graph = b.graph;
                in->gexec = b.gexec;
                in->h2d = std::move(b.h2d);
                in->d2h = std::move(b.d2h);
                std::lock_guard<std::mutex> lk(S->stats_mu);
                S->stats.graph_builds++;
            } else {
                in->graph_failed = true;
                note_cuda_error(S, b.error, 6);
            }
        }
        ++prepared;
        if (++copy == copies) {
            copy = 0;
            if (large) break;
            k *= 2;
        }
    }
    update_bytes(S);
    {
        std::lock_guard<std::mutex> lk(job.mu);
        job.status = status;
        job.prepared = prepared;
        job.done = true;
    }
    job.cv.notify_all();
    S->outstanding.fetch_sub(1);
}

void intake(fftu_server_st *S, std::deque<Req> &batch) {
    for (auto &q : batch) {
        Key k;
        k.d = q.r.d;
        for (int l = 0; l < k.d; ++l) k.n[l] = q.r.n[l];
        k.dtype = q.r.dtype;
        k.dir = q.r.dir;
        auto it = S->keys.find(k);
        if (it == S->keys.end()) {
            auto ks = std::make_unique<KeyState>();
            ks->key = k;
            ks->N = elems(k);
            ks->esize = k.dtype == FFTU_C128 ? 16 : 8;
            it = S->keys.emplace(k, std::move(ks)).first;
        }
        KeyState *ks = it->second.get();
        if (q.warm) {
            warm_key(S, ks, q);
            continue;
        }
        // a request that cannot fit even alone is refused at once (a plan's workspace is at most
        // N elements, its twiddle tables sum_l n_l elements)
        const size_t slot = ((size_t)ks->N * ks->esize + 255) / 256 * 256;
        const size_t alone = 2 * slot + (ks->plan ? 0 : (size_t)ks->N * ks->esize + (64u << 10));
        if (alone > (size_t)S->cfg.device_bytes) {
            complete(S, q, FFTU_ERR_NOMEM, 0, 0);
            continue;
        }
        ks->pending.push_back(q);
    }
    batch.clear();
}

bool any_busy(fftu_server_st *S) {
    for (auto &kv : S->keys)
        for (auto &in : kv.second->inst)
            if (in->busy) return true;
    return false;
}

bool any_pending(fftu_server_st *S) {
    for (auto &kv : S->keys)
        if (!kv.second->pending.empty()) return true;
    return false;
}

void builder_main(fftu_server_st *S) {
    cudaSetDevice(S->device);
    for (;;) {
        GraphBuild *job = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->b_mu);
            S->b_cv.wait(lk, [&] { return S->b_stop || !S->b_jobs.empty(); });
            if (S->b_jobs.empty()) return;  // stopping
            job = S->b_jobs.front();
            S->b_jobs.pop_front();
        }
        build_graph(*job, S->b_stream);
        std::lock_guard<std::mutex> lk(S->b_mu);
        S->b_done.push_back(job);
    }
}

// Attach graphs the builder has finished to their (idle or busy) instances.
void collect_graphs(fftu_server_st *S) {
    std::vector<GraphBuild *> done;
    {
        std::lock_guard<std::mutex> lk(S->b_mu);
        done.swap(S->b_done);
    }
    for (GraphBuild *b : done) {
        Instance *in = b->in;
        in->building = false;
        if (b->ok) {
            in->graph = b->graph;
            in->gexec = b->gexec;
            in->h2d = std::move(b->h2d);
            in->d2h = std::move(b->d2h);
            std::lock_guard<std::mutex> lk(S->stats_mu);
            S->stats.graph_builds++;
        } else {
            in->graph_failed = true;
            note_cuda_error(S, b->error, 6);
        }
        delete b;
    }
}

void server_main(fftu_server_st *S) {
    cudaSetDevice(S->device);
    std::deque<Req> local;
    double last = S->now();
    for (;;) {
        {
            const double now = S->now();
            if (now - last > S->stats.max_loop_gap_s) {
                std::lock_guard<std::mutex> lk(S->stats_mu);
                S->stats.max_loop_gap_s = now - last;
            }
            last = now;
        }
        {
            std::unique_lock<std::mutex> lk(S->in_mu);
            if (S->inbox.empty() && !S->stop.load() && !any_busy(S) && !any_pending(S))
                S->in_cv.wait_for(lk, std::chrono::milliseconds(5));
            local.swap(S->inbox);
        }
        intake(S, local);
        collect_graphs(S);
        const bool reaped = reap(S);
        const bool started = dispatch(S);
        if (S->stop.load() && !any_busy(S)) break;
        if (!reaped && !started && (any_busy(S) || any_pending(S)))
            std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
    for (auto &kv : S->keys)
        for (auto &q : kv.second->pending) complete(S, q, FFTU_ERR_ARG, 0, 0);
    {
        std::lock_guard<std::mutex> lk(S->in_mu);
        for (auto &q : S->inbox) complete(S, q, FFTU_ERR_ARG, 0, 0);
        S->inbox.clear();
    }
    {
        std::lock_guard<std::mutex> lk(S->b_mu);
        S->b_stop = true;
    }
    S->b_cv.notify_all();
    if (S->builder.joinable()) S->builder.join();
    {  // graphs that finished after the last collection, and jobs never started
        std::lock_guard<std::mutex> lk(S->b_mu);
        for (GraphBuild *b : S->b_done) {
            if (b->gexec) cudaGraphExecDestroy(b->gexec);
            if (b->graph) cudaGraphDestroy(b->graph);
            delete b;
        }
        for (GraphBuild *b : S->b_jobs) delete b;
        S->b_done.clear();
        S->b_jobs.clear();
    }
    for (auto &kv : S->keys) {
        for (auto &in : kv.second->inst) destroy_instance(S, in.get());
        kv.second->inst.clear();
        if (kv.second->plan) fftu_destroy(kv.second->plan);
        kv.second->plan = nullptr;
    }
    S->keys.clear();
}

// Shape, type and direction checks shared by fftu_server_submit and fftu_server_warm.
fftu_status check_request(const fftu_request *req) {
    if (req->d < 1 || req->d > FFTU_MAX_DIMS || (req->dtype != FFTU_C64 && req->dtype != FFTU_C128) ||
        (req->dir != FFTU_FORWARD && req->dir != FFTU_INVERSE)) {
        fftu::record_error("server: bad d, dtype or direction");
        return FFTU_ERR_ARG;
    }
    int64_t N = 1;
    for (int l = 0; l < req->d; ++l) {
        if (req->n[l] < 1 || (req->n[l] & (req->n[l] - 1))) {
            fftu::record_error("server: every n_l must be a power of two");
            return req->n[l] < 1 ? FFTU_ERR_ARG : FFTU_ERR_UNSUPPORTED;
        }
        if (req->n[l] > ((int64_t)1 << 40) || N > ((int64_t)1 << 40) / req->n[l]) {  // the plans' limit
            fftu::record_error("server: N exceeds 2^40 elements");
            return FFTU_ERR_ARG;
        }
        N *= req->n[l];
    }
    return FFTU_OK;
}

}  // namespace

extern "C" {

fftu_status fftu_server_create(const fftu_server_config *cfg, fftu_server *out) {
    if (!out) return FFTU_ERR_ARG;
    *out = nullptr;
    fftu_server_config c;
    std::memset(&c, 0, sizeof(c));
    if (cfg) c = *cfg;
    for (int i = 0; i < 4; ++i)
        if (c.reserved[i]) {
            fftu::record_error("server: reserved config fields must be zero");
            return FFTU_ERR_ARG;
        }
    if (c.max_batch == 0) c.max_batch = 64;
    if (c.streams == 0) c.streams = 8;
    if (c.large_elems == 0) c.large_elems = 1ll << 22;
    if (c.max_inflight == 0) c.max_inflight = 2 * c.streams;
    if (c.max_inflight_solo == 0) c.max_inflight_solo = c.streams >= 2 ? c.streams - c.streams / 2 : c.streams;
    if (c.max_batch < 1 || c.max_batch > 128 || c.streams < 1 || c.streams > 16 || c.large_elems < 1 ||
        c.device_bytes < 0 || c.max_inflight < 1 || c.max_inflight > 256 || c.copy_piece_mib < 0 ||
        c.max_inflight_solo < 1 || c.max_inflight_solo > 256) {
        fftu::record_error("server: max_batch must be in [1, 128], streams in [1, 16], max_inflight and "
                           "max_inflight_solo in [1, 256], large_elems >= 1");
        return FFTU_ERR_ARG;
    }
    auto S = new (std::nothrow) fftu_server_st();
    if (!S) return FFTU_ERR_NOMEM;
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        fftu::record_error("server: no CUDA device");
        return FFTU_ERR_CUDA;
    }
    if (c.device_bytes == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            delete S;
            return FFTU_ERR_CUDA;
        }
        c.device_bytes = (int64_t)(fr / 2);
    }
    S->cfg = c;
    std::memset(&S->stats, 0, sizeof(S->stats));
    S->stats.budget_bytes = c.device_bytes;
    S->t0 = Clock::now();
    // batched (small) requests on the highest stream priority, solo (large) ones on the lowest: when
    // both have work pending, the small requests' blocks are scheduled first
    int prio_low = 0, prio_high = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) {
        cudaGetLastError();
        prio_low = prio_high = 0;
    }
    const int split = c.streams >= 2 ? c.streams / 2 : c.streams;
    for (int i = 0; i < c.streams; ++i) {
        cudaStream_t s;
        if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, i < split ? prio_high : prio_low) !=
            cudaSuccess) {
            cudaGetLastError();
            for (auto x : S->streams) cudaStreamDestroy(x);
            delete S;
            return FFTU_ERR_CUDA;
        }
        S->streams.push_back(s);
    }
    S->split = split;
    if (cudaStreamCreateWithFlags(&S->b_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->w_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        for (auto x : S->streams) cudaStreamDestroy(x);
        if (S->b_stream) cudaStreamDestroy(S->b_stream);
        delete S;
        return FFTU_ERR_CUDA;
    }
    S->builder = std::thread(builder_main, S);
    S->thread = std::thread(server_main, S);
    *out = S;
    return FFTU_OK;
}

fftu_status fftu_server_warm(fftu_server S, const fftu_request *like, int max_k, double timeout_s) {
    if (!S || !like || !like->in || !like->out || max_k < 1) return FFTU_ERR_ARG;
    fftu_status st = check_request(like);
    if (st != FFTU_OK) return st;
    Req q;
    q.r = *like;
    q.t_submit = S->now();
    q.warm = std::make_shared<WarmJob>();
    q.warm->max_k = max_k;
    auto job = q.warm;
    S->outstanding.fetch_add(1);
    {
        std::lock_guard<std::mutex> lk(S->in_mu);
        S->inbox.push_back(q);
    }
    S->in_cv.notify_one();
    std::unique_lock<std::mutex> lk(job->mu);
    if (!job->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return job->done; }))
        return FFTU_ERR_TIMEOUT;
    return job->status;
}

fftu_status fftu_server_submit(fftu_server S, const fftu_request *req) {
    if (!S || !req || !req->in || !req->out) return FFTU_ERR_ARG;
    const fftu_status cst = check_request(req);
    if (cst != FFTU_OK) return cst;
    Req q;
    q.r = *req;
    q.t_submit = S->now();
    S->outstanding.fetch_add(1);
    {
        std::lock_guard<std::mutex> lk(S->stats_mu);
        S->stats.submitted++;
    }
    {
        std::lock_guard<std::mutex> lk(S->in_mu);
        S->inbox.push_back(q);
    }
    S->in_cv.notify_one();
    return FFTU_OK;
}

int fftu_server_poll(fftu_server S, fftu_completion *out, int max) {
    if (!S || (!out && max > 0) || max < 0) return -1;
    std::lock_guard<std::mutex> lk(S->out_mu);
    int n = 0;
    while (n < max && !S->outbox.empty()) {
        out[n++] = S->outbox.front();
        S->outbox.pop_front();
    }
    return n;
}

fftu_status fftu_server_drain(fftu_server S, double timeout_s) {
    if (!S) return FFTU_ERR_ARG;
    const auto end = Clock::now() + std::chrono::duration<double>(timeout_s);
    while (S->outstanding.load() > 0) {
        if (Clock::now() > end) return FFTU_ERR_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    return FFTU_OK;
}

fftu_status fftu_server_stats_get(fftu_server S, fftu_server_stats *st) {
    if (!S || !st) return FFTU_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->stats_mu);
    *st = S->stats;
    return FFTU_OK;
}

fftu_status fftu_server_destroy(fftu_server S) {
    if (!S) return FFTU_OK;
    S->stop.store(true);
    S->in_cv.notify_one();
    if (S->thread.joinable()) S->thread.join();
    for (auto s : S->streams) cudaStreamDestroy(s);
    if (S->b_stream) cudaStreamDestroy(S->b_stream);
    if (S->w_stream) cudaStreamDestroy(S->w_stream);
    delete S;
    return FFTU_OK;
}

}  // extern "C"
