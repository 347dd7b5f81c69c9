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
// rejected with FFTU_ERR_UNSUPPORTED.
//
// Memory: every GPU that loads this part of the library holds the static
// arrays (about 32 MiB) until the process exits.
//
// Set-up: the first call on each device (with that device current) looks up
// the arrays' device addresses with cudaGetSymbolAddress and sets the kernels'
// attributes; make that first call before any stream capture begins.
//
// Sharing: all calls on a device share the same arrays, which keep the last
// call's contents.  The completion counters are cleared on the stream at the
// start of every call, and the twiddle tables are regenerated on the stream
// whenever the shape differs from the previous call's.  Calls whose execution
// overlaps on the GPU (on different streams, or from different threads
// without ordering) race on these arrays and give wrong results: order them.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "fftu_internal.h"

namespace fftu {

namespace {

constexpr int kStaticRing = 2;                         // ring slots (>= 2 for the persistent kernel)
constexpr size_t kStaticUnitBytes = (size_t)16 << 20;  // largest residue unit accepted
constexpr size_t kStaticScratchBytes = kStaticRing * kStaticUnitBytes;
constexpr int kStaticMaxN = 4096;                      // largest n_l (table entries per axis)
constexpr int kStaticMaxUnits = 4096;                  // largest p_0 * p_1
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kStaticScratchBytes];
static __device__ __align__(256) float2 g_noalloc_tables[3 * kStaticMaxN];
static __device__ __align__(256) unsigned g_noalloc_counters[1 + 2 * kStaticMaxUnits];
static __device__ __align__(256) int g_noalloc_status;

struct DeviceState {
    bool ready = false;
    void *scratch = nullptr;
    float2 *tables = nullptr;
    unsigned *counters = nullptr;
    int *status = nullptr;
    int64_t table_n[3] = {0, 0, 0};
    int grids[2][3] = {};   // [which][stage1, stage2, ring]
    bool prepared[2][2] = {};  // [which][dir < 0]
};

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
        if (!ds.ready) {
            // once per device, with the device current: device addresses of the static arrays
            e = cudaGetSymbolAddress(&ds.scratch, g_noalloc_scratch);
            if (e == cudaSuccess) e = cudaGetSymbolAddress((void **)&ds.tables, g_noalloc_tables);
            if (e == cudaSuccess) e = cudaGetSymbolAddress((void **)&ds.counters, g_noalloc_counters);
            if (e == cudaSuccess) e = cudaGetSymbolAddress((void **)&ds.status, g_noalloc_status);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(FFTU_ERR_CUDA, "fftu_exec_noalloc: cudaGetSymbolAddress failed");
            }
            ds.ready = true;
        }
        if (!ds.prepared[which][dslot]) {
            size_t smem = 0;
            e = prepare_phase_a3(which, dir, (int)n[0], (int)n[1], ds.grids[which], &smem);
            if (e == cudaSuccess) e = prepare_phase_b3(0, dir);
            if (e != cudaSuccess) return fail(FFTU_ERR_CUDA, "fftu_exec_noalloc: kernel attributes");
            ds.prepared[which][dslot] = true;
        }
        for (int ax = 0; ax < 3; ++ax) {
            if (ds.table_n[ax] != n[ax]) {
                e = launch_twiddle_table(ds.tables + ax * kStaticMaxN, n[ax], 0, st);
                if (e != cudaSuccess) return fail(FFTU_ERR_CUDA, "fftu_exec_noalloc: twiddle generation launch");
                ds.table_n[ax] = n[ax];
            }
        }
        std::memset(&l, 0, sizeof(l));
        l.which = which;
        l.dir = dir;
        l.mode = 1;
        l.in = in;
        l.out = out;
        l.scratch = ds.scratch;
        l.tw[0] = ds.tables;
        l.tw[1] = ds.tables + kStaticMaxN;
        l.tw[2] = ds.tables + 2 * kStaticMaxN;
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
