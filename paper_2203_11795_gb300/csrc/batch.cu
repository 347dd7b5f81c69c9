// Many transforms of different shapes in one persistent launch.
//
// A batch is built from existing plans (same element type and direction).  Every
// pass of every transform becomes a job: phase A's strided sub-FFT passes (one per
// axis, Superstep 0 + the Superstep 1 store, Algorithm 2.3), then phase B
// (Superstep 2), either fused or one pass per axis.  Jobs are ordered pass-major
// (all transforms' first pass, then all second passes, ...); their tiles form one
// task list that persistent CTAs take in order with an atomic counter.  A tile of
// pass k of transform i first waits (bounded) until every tile of pass k - 1 of
// transform i is done; that pass is earlier in the order, so the earliest
// unfinished task can always run.  Exec makes no host synchronisation: the counters
// are cleared with a memset on the stream, so a batch exec can be captured into a
// CUDA graph (the in/out pointers travel as kernel parameters).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "bounded_wait.cuh"
#include "fft_device.cuh"
#include "fftu_internal.h"
#include "generic_tiles.cuh"

namespace fftu {

namespace {

constexpr int kBatchThreads = 512;
constexpr int kMaxBatchJobs = 4 * kMaxBatch;

struct BatchJob {
    int kind;         // 1 = axis pass, 2 = fused phase B
    int r0;           // first-stage radix of an axis pass (1 = none)
    int transform;    // index into the in/out pointer arrays
    int reads_input;  // 1: the first pass of phase A (reads in[], writes out[]); else in place on out[]
    int dep;          // job this one waits for (-1: none)
    int pad;
    int64_t tiles;
    int64_t first;    // first global task index
    int64_t dep_tiles;
    AxisPass a;
    PhaseBFused b;
};

struct BatchParams {
    const BatchJob *jobs;
    const int64_t *firsts;   // jobs[j].first, for the binary search
    int njobs;
    int64_t total;
    unsigned long long *task_ctr;
    unsigned *done;          // per job
    int *status;
    long long spin_limit_ns;
    const void *in[kMaxBatch];
    void *out[kMaxBatch];
};

// Each radix variant of the axis tile is its own function so that one kernel can hold
// all of them without the register allocation of the largest applying to the rest.
template <typename C, int DIR, int R0>
__device__ __noinline__ void axis_tile_call(const AxisPass &a, int64_t t, C *sm, const C *src, C *dst) {
    axis_tile<C, DIR, R0>(a, t, sm, src, dst, static_cast<const C *>(a.tw));
}
template <typename C, int DIR>
__device__ __noinline__ void phaseb_tile_call(const PhaseBFused &b, int64_t t, C *sm, C *data) {
    phaseb_tile<C, DIR>(b, t, sm, data);
}

template <typename C, int DIR>
__global__ void __launch_bounds__(kBatchThreads) batch_kernel(const __grid_constant__ BatchParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw);
    __shared__ __align__(16) BatchJob s_job;
    __shared__ int64_t s_firsts[kMaxBatchJobs];
    __shared__ long long s_task;
    __shared__ int s_jobi, s_ok, s_loaded;
    const int tid = threadIdx.x;
    for (int j = tid; j < P.njobs; j += blockDim.x) s_firsts[j] = P.firsts[j];
    if (tid == 0) s_loaded = -1;
    __syncthreads();
    for (;;) {
        if (tid == 0) {
            const long long t = (long long)atomicAdd(P.task_ctr, 1ull);
            s_task = t;
            if (t < P.total) {
                int lo = 0, hi = P.njobs - 1;  // last job with first <= t
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_firsts[mid] <= t) lo = mid;
                    else hi = mid - 1;
                }
                s_jobi = lo;
                int ok = 1;
                const int dep = P.jobs[lo].dep;
                if (dep >= 0 &&
                    !wait_counter_geq(P.done + dep, (unsigned)P.jobs[lo].dep_tiles, P.spin_limit_ns, P.status))
                    ok = 0;
                s_ok = ok;
            }
        }
        __syncthreads();
        const long long t = s_task;
        if (t >= P.total) break;
        const int j = s_jobi;
        if (j != s_loaded) {  // bring the job descriptor into shared memory
            const int *srcw = reinterpret_cast<const int *>(P.jobs + j);
            int *dstw = reinterpret_cast<int *>(&s_job);
            for (int w = tid; w < (int)(sizeof(BatchJob) / sizeof(int)); w += blockDim.x) dstw[w] = srcw[w];
            __syncthreads();
            if (tid == 0) s_loaded = j;
        }
        __syncthreads();
        if (s_ok) {
            const BatchJob &J = s_job;
            const int64_t lt = t - J.first;
            C *out = static_cast<C *>(P.out[J.transform]);
            if (J.kind == 1) {
                const C *src = J.reads_input ? static_cast<const C *>(P.in[J.transform]) : out;
                switch (J.r0) {
                    case 2: axis_tile_call<C, DIR, 2>(J.a, lt, sm, src, out); break;
                    case 4: axis_tile_call<C, DIR, 4>(J.a, lt, sm, src, out); break;
                    case 16: axis_tile_call<C, DIR, 16>(J.a, lt, sm, src, out); break;
                    default: axis_tile_call<C, DIR, 1>(J.a, lt, sm, src, out); break;
                }
            } else {
                phaseb_tile_call<C, DIR>(J.b, lt, sm, out);
            }
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(P.done + j, 1u);
        }
    }
}

// Diagnostic for fftu_selftest_bounded_wait: one thread waits, with the batch kernel's bounded
// wait, on words[0], which nothing advances; the expired wait leaves FFTU_ERR_TIMEOUT in words[1]
// and the time it waited in words[2..3].
__global__ void wait_probe_kernel(unsigned *words, long long limit_ns) {
    if (threadIdx.x != 0) return;
    const unsigned long long t0 = globaltimer_ns();
    wait_counter_geq(words, 1u, limit_ns, reinterpret_cast<int *>(words + 1));
    const unsigned long long dt = globaltimer_ns() - t0;
    words[2] = (unsigned)dt;
    words[3] = (unsigned)(dt >> 32);
}

template <typename C, int DIR>
cudaError_t batch_setup(size_t smem, int threads, int *grid) {
    // The limit is a property of the kernel, shared by every batch: set it to the largest tile any
    // batch can use, never to this batch's (a later, smaller batch would make this one's launches fail).
    if (smem > (size_t)kMaxDynSmem) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<C, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<C, DIR>, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *grid = sms * per_sm;
    return cudaSuccess;
}

}  // namespace

struct Batch {
    int count = 0, is_double = 0, dir = 0, device = 0, grid = 0;
    int threads = kBatchThreads;  // the largest block any job's tile needs (a multiple of 32, <= 512)
    size_t smem = 0;
    int njobs = 0;
    int64_t total = 0;
    void *dev_mem = nullptr;  // jobs | firsts | task counter | done counters
    BatchJob *jobs = nullptr;
    int64_t *firsts = nullptr;
    unsigned long long *task_ctr = nullptr;
    unsigned *done = nullptr;
    int *status = nullptr;
    size_t counter_bytes = 0;
};

fftu_status batch_create(int count, const fftu_handle *plans, Batch **out_batch) {
    *out_batch = nullptr;
    if (count < 1 || count > kMaxBatch || !plans) {
        record_error("batch: count must be in [1, 128] and plans non-NULL");
        return FFTU_ERR_ARG;
    }
    std::vector<PlanView> views(count);
    for (int i = 0; i < count; ++i) {
        fftu_status s = plan_view(plans[i], &views[i]);
        if (s != FFTU_OK) return s;
        if (views[i].dtype != views[0].dtype || views[i].dir != views[0].dir || views[i].device != views[0].device) {
            record_error("batch: every plan needs the same dtype, direction and device");
            return FFTU_ERR_ARG;
        }
        if (views[i].layout != 0) {
            record_error("batch: CYCLIC-layout plans are not batched");
            return FFTU_ERR_UNSUPPORTED;
        }
        if (views[i].precision != 0 || views[i].radix != 8) {
            record_error("batch: split-precision and radix-16 plans are not batched");
            return FFTU_ERR_UNSUPPORTED;
        }
        if (views[i].pingpong) {
            record_error("batch: plans whose phase A alternates with a workspace (long lines) are not batched");
            return FFTU_ERR_UNSUPPORTED;
        }
    }
    // jobs, pass-major
    std::vector<BatchJob> jobs;
    std::vector<std::vector<int>> job_of(count);
    size_t max_tile_bytes = 0;
    const size_t esize = views[0].dtype == FFTU_C128 ? 16 : 8;
    int max_passes = 0;
    int max_threads = 128;  // phase-B tiles loop over any block size
    for (auto &v : views) max_passes = std::max(max_passes, (int)(v.a_passes.size() + v.b_steps.size()));
    for (int k = 0; k < max_passes; ++k) {
        for (int i = 0; i < count; ++i) {
            const PlanView &v = views[i];
            const int na = (int)v.a_passes.size();
            if (k >= na + (int)v.b_steps.size()) continue;
            BatchJob J;
            std::memset(&J, 0, sizeof(J));
            J.transform = i;
            J.dep = job_of[i].empty() ? -1 : job_of[i].back();
            J.dep_tiles = J.dep >= 0 ? jobs[J.dep].tiles : 0;
            const StepView &sv = k < na ? v.a_passes[k] : v.b_steps[k - na];
            if (sv.is_axis) {
                J.kind = 1;
                J.a = sv.axis;
                J.r0 = sv.axis.nstages > 0 && sv.axis.radix[0] != 8 ? sv.axis.radix[0] : 1;
                J.tiles = sv.axis.tiles;
                J.reads_input = k == 0;
                max_tile_bytes = std::max(max_tile_bytes, (size_t)sv.axis.tile * esize);
                max_threads = std::max(max_threads, sv.axis.threads);
            } else {
                J.kind = 2;
                J.b = sv.pb;
                J.tiles = sv.pb.tiles;
                J.reads_input = 0;
                max_tile_bytes = std::max(max_tile_bytes, (size_t)sv.pb.P * sv.pb.Mt * esize);
            }
            job_of[i].push_back((int)jobs.size());
            jobs.push_back(J);
        }
    }
    if ((int)jobs.size() > kMaxBatchJobs) {
        record_error("batch: too many passes in total");
        return FFTU_ERR_UNSUPPORTED;
    }
    // every transform must read its input: a transform without phase-A passes is a copy
    for (int i = 0; i < count; ++i)
        if (views[i].a_passes.empty()) {
            record_error("batch: a transform with no phase-A pass (all n_l = 1) is not batched");
            return FFTU_ERR_UNSUPPORTED;
        }
    int64_t first = 0;
    std::vector<int64_t> firsts(jobs.size());
    for (size_t j = 0; j < jobs.size(); ++j) {
        jobs[j].first = first;
        firsts[j] = first;
        first += jobs[j].tiles;
    }
    Batch *b = new (std::nothrow) Batch();
    if (!b) {
        record_error("batch: host allocation failed");
        return FFTU_ERR_NOMEM;
    }
    b->count = count;
    b->is_double = views[0].dtype == FFTU_C128;
    b->dir = views[0].dir;
    b->device = views[0].device;
    b->njobs = (int)jobs.size();
    b->total = first;
    b->smem = max_tile_bytes;
    b->threads = std::min(kBatchThreads, (max_threads + 31) / 32 * 32);
    const size_t jb = sizeof(BatchJob) * jobs.size(), fb = sizeof(int64_t) * jobs.size();
    b->counter_bytes = 16 + sizeof(unsigned) * jobs.size();
    const size_t bytes = jb + fb + b->counter_bytes + 16;
    cudaError_t e = cudaMalloc(&b->dev_mem, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete b;
        record_error("batch: device allocation failed");
        return FFTU_ERR_NOMEM;
    }
    char *base = static_cast<char *>(b->dev_mem);
    b->jobs = reinterpret_cast<BatchJob *>(base);
    b->firsts = reinterpret_cast<int64_t *>(base + jb);
    b->task_ctr = reinterpret_cast<unsigned long long *>(base + jb + fb);
    b->status = reinterpret_cast<int *>(base + jb + fb + 8);
    b->done = reinterpret_cast<unsigned *>(base + jb + fb + 16);
    // uploads on a private stream: creating a batch does not wait for transforms in flight
    cudaStream_t ps = nullptr;
    e = cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->jobs, jobs.data(), jb, cudaMemcpyHostToDevice, ps);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->firsts, firsts.data(), fb, cudaMemcpyHostToDevice, ps);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->status, 0, sizeof(int), ps);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ps);
    if (ps) cudaStreamDestroy(ps);
    if (e == cudaSuccess) {
        if (b->is_double)
            e = b->dir < 0 ? batch_setup<double2, -1>(b->smem, b->threads, &b->grid)
                           : batch_setup<double2, 1>(b->smem, b->threads, &b->grid);
        else
            e = b->dir < 0 ? batch_setup<float2, -1>(b->smem, b->threads, &b->grid)
                           : batch_setup<float2, 1>(b->smem, b->threads, &b->grid);
    }
    if (e != cudaSuccess) {
        cudaFree(b->dev_mem);
        delete b;
        record_error("batch: set-up failed");
        return FFTU_ERR_CUDA;
    }
    *out_batch = b;
    return FFTU_OK;
}

fftu_status batch_exec(Batch *b, const void *const *ins, void *const *outs, cudaStream_t st) {
    BatchParams P;
    std::memset(&P, 0, sizeof(P));
    P.jobs = b->jobs;
    P.firsts = b->firsts;
    P.njobs = b->njobs;
    P.total = b->total;
    P.task_ctr = b->task_ctr;
    P.done = b->done;
    P.status = b->status;
    P.spin_limit_ns = 2000000000ll;
    for (int i = 0; i < b->count; ++i) {
        if (!ins[i] || !outs[i] || ((reinterpret_cast<uintptr_t>(ins[i]) | reinterpret_cast<uintptr_t>(outs[i])) & 15)) {
            record_error("batch: in/out pointers must be non-NULL and 16-byte aligned");
            return FFTU_ERR_ARG;
        }
        P.in[i] = ins[i];
        P.out[i] = outs[i];
    }
    // the task counter and the per-job counters start at zero on every exec
    cudaError_t e = cudaMemsetAsync(b->task_ctr, 0, 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->done, 0, sizeof(unsigned) * b->njobs, st);
    if (e != cudaSuccess) {
        record_error("batch: counter reset failed");
        return FFTU_ERR_CUDA;
    }
    int64_t grid = b->grid;
    if (grid > b->total) grid = b->total;
    if (b->is_double) {
        if (b->dir < 0)
            batch_kernel<double2, -1><<<(unsigned)grid, b->threads, b->smem, st>>>(P);
        else
            batch_kernel<double2, 1><<<(unsigned)grid, b->threads, b->smem, st>>>(P);
    } else {
        if (b->dir < 0)
            batch_kernel<float2, -1><<<(unsigned)grid, b->threads, b->smem, st>>>(P);
        else
            batch_kernel<float2, 1><<<(unsigned)grid, b->threads, b->smem, st>>>(P);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        record_error("batch: kernel launch failed");
        return FFTU_ERR_CUDA;
    }
    return FFTU_OK;
}

fftu_status batch_status(Batch *b) {
    int v = 0;
    cudaError_t e = cudaMemcpy(&v, b->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(b->status, 0, sizeof(int));
    if (e != cudaSuccess) return FFTU_ERR_CUDA;
    return v == 0 ? FFTU_OK : v == FFTU_ERR_TIMEOUT ? FFTU_ERR_TIMEOUT : FFTU_ERR_INTERNAL;
}

void batch_destroy(Batch *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->dev_mem) cudaFree(b->dev_mem);
    delete b;
}

}  // namespace fftu

struct fftu_batch_st {
    fftu::Batch *impl;
};

extern "C" {

fftu_status fftu_batch_create(int count, const fftu_handle *plans, fftu_batch *out) {
    if (!out) return FFTU_ERR_ARG;
    *out = nullptr;
    fftu::Batch *b = nullptr;
    fftu_status s = fftu::batch_create(count, plans, &b);
    if (s != FFTU_OK) return s;
    fftu_batch_st *h = new (std::nothrow) fftu_batch_st;
    if (!h) {
        fftu::batch_destroy(b);
        return FFTU_ERR_NOMEM;
    }
    h->impl = b;
    *out = h;
    return FFTU_OK;
}

fftu_status fftu_batch_exec(fftu_batch batch, const void *const *ins, void *const *outs, void *stream) {
    if (!batch || !batch->impl || !ins || !outs) {
        fftu::record_error("batch: NULL argument");
        return FFTU_ERR_ARG;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != batch->impl->device) {
        fftu::record_error("batch: wrong current device");
        return FFTU_ERR_ARG;
    }
    return fftu::batch_exec(batch->impl, ins, outs, static_cast<cudaStream_t>(stream));
}

fftu_status fftu_batch_check_status(fftu_batch batch) {
    if (!batch || !batch->impl) return FFTU_ERR_ARG;
    return fftu::batch_status(batch->impl);
}

fftu_status fftu_batch_destroy(fftu_batch batch) {
    if (!batch) return FFTU_OK;
    fftu::batch_destroy(batch->impl);
    delete batch;
    return FFTU_OK;
}

fftu_status fftu_selftest_bounded_wait(double limit_s, double *waited_s) {
    using namespace fftu;
    if (!(limit_s >= 1e-3 && limit_s <= 2.0)) {
        record_error("selftest: limit_s must be in [0.001, 2]");
        return FFTU_ERR_ARG;
    }
    // words: [0] the counter nothing advances, [1] status, [2..3] waited nanoseconds
    unsigned *words = nullptr;
    cudaError_t e = cudaMalloc(&words, 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FFTU_ERR_NOMEM;
    }
    cudaStream_t ps = nullptr;
    e = cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemsetAsync(words, 0, 16, ps);
    if (e == cudaSuccess) {
        wait_probe_kernel<<<1, 32, 0, ps>>>(words, (long long)(limit_s * 1e9));
        e = cudaGetLastError();
    }
    unsigned host[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, words, 16, cudaMemcpyDeviceToHost, ps);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ps);
    if (ps) cudaStreamDestroy(ps);
    cudaFree(words);
    if (e != cudaSuccess) {
        record_error("selftest: CUDA call failed");
        return FFTU_ERR_CUDA;
    }
    unsigned long long ns = (unsigned long long)host[2] | ((unsigned long long)host[3] << 32);
    if (waited_s) *waited_s = (double)ns * 1e-9;
    if ((int)host[1] != (int)FFTU_ERR_TIMEOUT) {
        record_error("selftest: the wait did not report FFTU_ERR_TIMEOUT");
        return FFTU_ERR_INTERNAL;
    }
    return FFTU_OK;
}

}  // extern "C"
