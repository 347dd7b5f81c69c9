// fftu_exec_noalloc: the whole 3D transform without any device allocation.
//
// Who needs this: callers that cannot call cudaMalloc on the path where they
// run the FFT -- for example code that is being captured into a CUDA graph
// (an allocation would break or be left out of the capture), plugins living
// inside a host application that owns every device allocation and forbids
// others, and real-time or embedded loops that must not block in the driver's
// allocator or risk an out-of-memory failure after start-up.  fftu_plan
// allocates the plan's twiddle tables and its workspace, so those callers
// cannot use fftu_plan / fftu_exec at that point.
//
// What it runs: the persistent two-stage phase-A kernel (phase_a3.cu, ring
// mode) followed by the in-place 3D phase-B kernel (phase_b3.cu), i.e. the same
// kernels fftu_exec uses for these shapes.  The kernel's scratch ring, its
// completion counters, the twiddle tables and the status word live in
// file-scope static __device__ arrays below instead of plan-owned memory.  The
// scratch holds kStaticRing residue units of at most kStaticUnitBytes each;
// shapes whose residue unit (all elements sharing s_0 and s_1) is larger are
// rejected with FFTU_ERR_UNSUPPORTED.  With the fused kernels that exist, that
// leaves 512^3 complex64 with p = 8^3 as the one accepted problem.
//
// Memory: every GPU that loads this part of the library holds the static
// arrays (about 32 MiB) until the process exits.
//
// Set-up: the first call on each device (with that device current) looks up
// the arrays' device addresses with cudaGetSymbolAddress and sets the kernels'
// attributes, and the first call with a given axis length n_l writes that
// length's twiddle table into its own fixed slot (one slot per power of two, so
// a table is written once per device and never overwritten).  Make those first
// calls before any stream capture: a call that would need this set-up while
// its stream is capturing returns FFTU_ERR_ARG instead.
//
// Sharing: all calls on a device share the same arrays, which keep the last
// call's contents.  The completion counters are cleared on the stream at the
// start of every call.  Calls whose execution overlaps on the GPU (on
// different streams, or from different threads without ordering) race on
// these arrays and give wrong results: order them.
//
// Errors found on the GPU: every device wait of the ring kernel is bounded; one
// that expires records FFTU_ERR_TIMEOUT in the shared status word and leaves
// that call's output invalid.  The word is sticky: fftu_noalloc_check_status
// reads and clears it.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "bounded_wait.cuh"
#include "fftu_internal.h"

namespace fftu {

namespace {

constexpr int kStaticRing = 2;                         // ring slots (>= 2 for the persistent kernel)
constexpr size_t kStaticUnitBytes = (size_t)16 << 20;  // largest residue unit accepted
constexpr size_t kStaticScratchBytes = kStaticRing * kStaticUnitBytes;
constexpr int kStaticMaxLogN = 12;                     // largest n_l = 2^12 = 4096
constexpr int kStaticMaxN = 1 << kStaticMaxLogN;
// Twiddle tables: one slot per power of two n = 2^k (k = 1 .. 12) at offset n - 2, 8190 entries in all.
constexpr int kStaticTableElems = 2 * kStaticMaxN;
constexpr int kStaticMaxUnits = 4096;                  // largest p_0 * p_1
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kStaticScratchBytes];
static __device__ __align__(256) float2 g_noalloc_tables[kStaticTableElems];
static __device__ __align__(256) unsigned g_noalloc_counters[1 + 2 * kStaticMaxUnits];
static __device__ __align__(256) int g_noalloc_status;
static __device__ __align__(256) unsigned g_noalloc_probe_word;  // never advanced (status self-test)

struct DeviceState {
    bool ready = false;
    void *scratch = nullptr;
    float2 *tables = nullptr;
    unsigned *counters = nullptr;
    int *status = nullptr;
    unsigned *probe = nullptr;
    bool table_ready[kStaticMaxLogN + 1] = {};          // [log2 n]: slot written
    int grids[kPhaseA3Configs][3] = {};                 // [which][stage1, stage2, ring]
    bool prepared[kPhaseA3Configs][2] = {};             // [which][dir < 0]
};

int log2_exact(int64_t n) {  // log2 of a power of two, else -1
    if (n < 1 || (n & (n - 1))) return -1;
    int k = 0;
    while ((int64_t(1) << k) < n) ++k;
    return k;
}

// Once per device, with that device current: the device addresses of the static arrays.
// Caller holds g_mutex.
cudaError_t ensure_ready(DeviceState &ds) {
    if (ds.ready) return cudaSuccess;
    cudaError_t e = cudaGetSymbolAddress(&ds.scratch, g_noalloc_scratch);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void **)&ds.tables, g_noalloc_tables);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void **)&ds.counters, g_noalloc_counters);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void **)&ds.status, g_noalloc_status);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void **)&ds.probe, g_noalloc_probe_word);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;
    }
    ds.ready = true;
    return cudaSuccess;
}

bool stream_capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// Status self-test: one thread waits, with the library's bounded wait, on a word nothing advances;
// the expired wait records FFTU_ERR_TIMEOUT in the status word fftu_exec_noalloc's kernels use.
__global__ void noalloc_probe_kernel(const unsigned *word, int *status, long long limit_ns) {
    if (threadIdx.x == 0) wait_counter_geq(word, 1u, limit_ns, status);
}

DeviceState g_state[kMaxDevices];
std::mutex g_mutex;

fftu_status fail(fftu_status s, const char *msg) {
    record_error(msg);
    return s;
}

}  // namespace

}  // namespace fftu

extern "C" fftu_status fftu_exec_noalloc(int d, const int64_t *n, const int64_t *p, fftu_dtype dtype,
                                         fftu_dir dir, const void *in, void *out, void *stream) {
    using namespace fftu;
    record_error("");
    if (d != 3 || !n || !p) return fail(FFTU_ERR_ARG, "fftu_exec_noalloc: d must be 3 and n, p non-NULL");
    if (dtype != FFTU_C64) return fail(FFTU_ERR_UNSUPPORTED, "fftu_exec_noalloc: complex64 only");
    if (dir != FFTU_FORWARD && dir != FFTU_INVERSE) return fail(FFTU_ERR_ARG, "fftu_exec_noalloc: bad dir");
    if (!in || !out || in == out)
        return fail(FFTU_ERR_ARG, "fftu_exec_noalloc: in and out must be distinct non-NULL device pointers");
    if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15)
        return fail(FFTU_ERR_ARG, "fftu_exec_noalloc: in/out must be 16-byte aligned");
    for (int l = 0; l < 3; ++l) {
        if (n[l] < 1 || p[l] < 1) return fail(FFTU_ERR_ARG, "fftu_exec_noalloc: n_l and p_l must be >= 1");
        if (p[l] > n[l] / p[l] || n[l] % (p[l] * p[l]) != 0)
            return fail(FFTU_ERR_DIVISIBILITY, "fftu_exec_noalloc: p_l^2 must divide n_l");
        if (n[l] > kStaticMaxN)
            return fail(FFTU_ERR_UNSUPPORTED, "fftu_exec_noalloc: n_l above 4096 (static twiddle table size)");
    }
    if (!(p[0] == p[1] && p[1] == p[2]))
        return fail(FFTU_ERR_UNSUPPORTED, "fftu_exec_noalloc: needs p_0 = p_1 = p_2");
    Phase3Info info;
    const int which = phase_a3_select(3, n, p, 0, &info);
    if (which < 0)
        return fail(FFTU_ERR_UNSUPPORTED, "fftu_exec_noalloc: no fused phase-A kernel for this shape and p");
    if ((size_t)info.unit_elems * sizeof(float2) > kStaticUnitBytes)
        return fail(FFTU_ERR_UNSUPPORTED,
                    "fftu_exec_noalloc: residue unit exceeds the 16 MiB static scratch slot (use fftu_exec)");
    const int units = (int)(p[0] * p[1]);
    if (units > kStaticMaxUnits || units <= kStaticRing)
        return fail(FFTU_ERR_UNSUPPORTED, "fftu_exec_noalloc: p_0 p_1 must be in (2, 4096]");
    const int mt3 = phase_b3_tile_mt((int)p[0], (int)p[1], (int)p[2], 0);
    if (mt3 == 0 || (n[2] / p[2]) % mt3 != 0)
        return fail(FFTU_ERR_UNSUPPORTED, "fftu_exec_noalloc: no fused phase-B kernel for this p");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(FFTU_ERR_CUDA, "fftu_exec_noalloc: cudaGetDevice failed");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int dslot = dir < 0 ? 1 : 0;
    Phase3Launch l;
    PhaseBFused b;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        DeviceState &ds = g_state[dev];
        if (which >= kPhaseA3Configs)
            return fail(FFTU_ERR_INTERNAL, "fftu_exec_noalloc: unknown phase-A configuration");
        int lg[3];
        for (int ax = 0; ax < 3; ++ax) {
            lg[ax] = log2_exact(n[ax]);
            if (lg[ax] < 1 || lg[ax] > kStaticMaxLogN)
                return fail(FFTU_ERR_UNSUPPORTED, "fftu_exec_noalloc: n_l must be a power of two in [2, 4096]");
        }
        const bool capturing = stream_capturing(st);
        const bool setup_needed = !ds.ready || !ds.prepared[which][dslot] || !ds.table_ready[lg[0]] ||
                                  !ds.table_ready[lg[1]] || !ds.table_ready[lg[2]];
        if (capturing && setup_needed)
            return fail(FFTU_ERR_ARG,
                        "fftu_exec_noalloc: first call for this device, shape or direction made under stream "
                        "capture; make one call before capturing");
        if (ensure_ready(ds) != cudaSuccess)
            return fail(FFTU_ERR_CUDA, "fftu_exec_noalloc: cudaGetSymbolAddress failed");
        if (!ds.prepared[which][dslot]) {
            size_t smem = 0;
            e = prepare_phase_a3(which, dir, (int)n[0], (int)n[1], ds.grids[which], &smem);
            if (e == cudaSuccess) e = prepare_phase_b3(0, dir);
            if (e != cudaSuccess) return fail(FFTU_ERR_CUDA, "fftu_exec_noalloc: kernel attributes");
            ds.prepared[which][dslot] = true;
        }
        for (int ax = 0; ax < 3; ++ax) {
            if (!ds.table_ready[lg[ax]]) {
                // written once per device into the slot of this length; stream-ordered before this call's
                // kernels, and every later call on any stream comes after it on the host
                e = launch_twiddle_table(ds.tables + (n[ax] - 2), n[ax], 0, st);
                if (e != cudaSuccess) return fail(FFTU_ERR_CUDA, "fftu_exec_noalloc: twiddle generation launch");
                e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) return fail(FFTU_ERR_CUDA, "fftu_exec_noalloc: twiddle generation");
                ds.table_ready[lg[ax]] = true;
            }
        }
        std::memset(&l, 0, sizeof(l));
        l.which = which;
        l.dir = dir;
        l.mode = 1;
        l.in = in;
        l.out = out;
        l.scratch = ds.scratch;
        l.tw[0] = ds.tables + (n[0] - 2);
        l.tw[1] = ds.tables + (n[1] - 2);
        l.tw[2] = ds.tables + (n[2] - 2);
        l.status = ds.status;
        l.counters = ds.counters;
        l.p0 = (int)p[0];
        l.p1 = (int)p[1];
        l.n0 = (int)n[0];
        l.n1 = (int)n[1];
        l.ring = kStaticRing;
        l.lag = 1;
        l.grid1 = ds.grids[which][0];
        l.grid2 = ds.grids[which][1];
        l.grid = ds.grids[which][2];
        l.spin_limit_ns = 2000000000ll;
    }
    std::memset(&b, 0, sizeof(b));
    b.data = out;
    b.d = 3;
    int64_t stride = 1;
    for (int ax = 2; ax >= 0; --ax) {
        b.n[ax] = n[ax];
        b.p[ax] = (int)p[ax];
        b.L[ax] = n[ax] / p[ax];
        b.stride[ax] = stride;
        stride *= n[ax];
    }
    b.P = (int)(p[0] * p[1] * p[2]);
    b.Mt = mt3;
    b.tiles = b.L[0] * b.L[1] * (b.L[2] / mt3);
    b.threads = 256;
    b.scale = dir == FFTU_INVERSE ? 1.0 / (double)(n[0] * n[1] * n[2]) : 1.0;

    e = launch_phase_a3(l, st);  // clears the counters on the stream, then the persistent kernel
    if (e == cudaSuccess) e = launch_phase_b3(b, 0, dir, st);
    if (e != cudaSuccess) return fail(FFTU_ERR_CUDA, "fftu_exec_noalloc: kernel launch failed");
    return FFTU_OK;
}

// Read and clear the status word shared by fftu_exec_noalloc's kernels on the current device.  The
// copy and the clear are ordered after the work already queued on `stream`, and the call waits for
// them; no allocation.
extern "C" fftu_status fftu_noalloc_check_status(void *stream) {
    using namespace fftu;
    record_error("");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(FFTU_ERR_CUDA, "fftu_noalloc_check_status: cudaGetDevice failed");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (stream_capturing(st)) return fail(FFTU_ERR_ARG, "fftu_noalloc_check_status: stream is capturing");
    int *status = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        DeviceState &ds = g_state[dev];
        if (!ds.ready) return FFTU_OK;  // no call has run on this device: nothing can have been recorded
        status = ds.status;
    }
    int v = 0;
    e = cudaMemcpyAsync(&v, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(FFTU_ERR_CUDA, "fftu_noalloc_check_status: status word read");
    }
    if (v == 0) return FFTU_OK;
    record_error(v == FFTU_ERR_TIMEOUT ? "fftu_exec_noalloc: a bounded device wait expired (output invalid)"
                                       : "fftu_exec_noalloc: device status word set");
    return v == FFTU_ERR_TIMEOUT ? FFTU_ERR_TIMEOUT : FFTU_ERR_INTERNAL;
}

// Failure-detection self-test of the path above: a one-thread kernel runs the library's bounded wait
// on a static word that nothing advances, with a budget of limit_s seconds, and records the expiry in
// the status word fftu_exec_noalloc's kernels share.  The next fftu_noalloc_check_status on this
// stream then reports FFTU_ERR_TIMEOUT.  Nothing traps; the context stays usable.
extern "C" fftu_status fftu_noalloc_selftest_timeout(double limit_s, void *stream) {
    using namespace fftu;
    record_error("");
    if (!(limit_s >= 1e-3 && limit_s <= 2.0))
        return fail(FFTU_ERR_ARG, "fftu_noalloc_selftest_timeout: limit_s must be in [0.001, 2]");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(FFTU_ERR_CUDA, "fftu_noalloc_selftest_timeout: cudaGetDevice failed");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (stream_capturing(st)) return fail(FFTU_ERR_ARG, "fftu_noalloc_selftest_timeout: stream is capturing");
    DeviceState *ds = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        ds = &g_state[dev];
        if (ensure_ready(*ds) != cudaSuccess)
            return fail(FFTU_ERR_CUDA, "fftu_noalloc_selftest_timeout: cudaGetSymbolAddress failed");
    }
    e = cudaMemsetAsync(ds->probe, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) {
        noalloc_probe_kernel<<<1, 32, 0, st>>>(ds->probe, ds->status, (long long)(limit_s * 1e9));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(FFTU_ERR_CUDA, "fftu_noalloc_selftest_timeout: launch failed");
    }
    return FFTU_OK;
}
