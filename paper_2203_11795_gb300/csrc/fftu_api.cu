// C ABI of libfftu: validation, planning, and stream-ordered execution of
// Algorithm 2.3 (Sec. 2.2) on one GPU.
//
// A plan is a list of kernel launches for phase A (Superstep 0 + the
// Superstep 1 redistribution, realised by the store positions) and for phase B
// (Superstep 2, in place).  The plan owns the FP64-generated twiddle tables
// (one table of w_{n_l}^e, e in [n_l], per axis: sum_l n_l entries; the
// paper's per-processor table of eq. weights holds the n_l/p_l entries one
// processor needs, here every virtual processor reads the shared table) and a
// device status word.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "fftu_internal.h"

namespace fftu {

namespace {

thread_local char g_err[320] = "";

void set_err(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

}  // namespace

void record_error(const char *msg) { set_err("%s", msg); }

namespace {

fftu_status cuda_fail(cudaError_t e, const char *what) {
    set_err("%s: %s", what, cudaGetErrorString(e));
    return FFTU_ERR_CUDA;
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

int ilog2(int64_t v) {
    int r = 0;
    while ((int64_t(1) << r) < v) ++r;
    return r;
}

// Radix sequence for a power-of-two length: radix 8 where possible, a single
// 16 or 4 to absorb the remainder, radix 2 only for length 2.
int radix_plan(int len, int *radix) {
    int k = ilog2(len), n = 0;
    if (k == 0) return 0;
    int eights = k / 3, rem = k % 3;
    if (rem == 1) {
        if (eights >= 1) {
            radix[n++] = 16;
            --eights;
        } else {
            radix[n++] = 2;
        }
    } else if (rem == 2) {
        radix[n++] = 4;
    }
    for (int i = 0; i < eights; ++i) radix[n++] = 8;
    return n;
}

// Radix sequence of the split-precision passes: radix-16 stages (tensor cores), then one stage of
// the remaining factor 2, 4 or 8 (CUDA cores).
int radix_plan_tc(int len, int *radix) {
    int k = ilog2(len), n = 0;
    for (; k >= 4; k -= 4) radix[n++] = 16;
    if (k > 0) radix[n++] = 1 << k;
    return n;
}

enum StepKind {
    STEP_AXIS = 1, STEP_PHASE_B_FUSED = 2, STEP_PHASE_B3 = 3, STEP_PHASE_A3 = 4, STEP_LINE = 5, STEP_PAIR = 6,
    STEP_TRIPLE = 7
};

struct Step {
    int kind;
    AxisPass axis;   // STEP_LINE and STEP_PAIR keep the strided-pass form of the same axis (in place; batching)
    AxisPass axis2;  // STEP_PAIR / STEP_TRIPLE: the strided-pass form of the next axis down (run after `axis`)
    AxisPass axis3;  // STEP_TRIPLE: the strided-pass form of the third axis (run after `axis2`)
    PhaseBFused pb;
    Phase3Launch a3;
    LinePass line;
    PairPass pair;
    TriplePass triple;

    int passes() const { return kind == STEP_TRIPLE ? 3 : kind == STEP_PAIR ? 2 : 1; }
    const AxisPass &strided(int i) const { return i == 0 ? axis : i == 1 ? axis2 : axis3; }
    bool whole_lines() const {
        for (int i = 0; i < passes(); ++i)
            if (strided(i).Gt < strided(i).G) return false;
        return true;
    }
};

// Residue units up to this size run phase A as one persistent kernel through a
// scratch ring of kRingSlots units.  Rings up to 48 MiB (16 MiB units, e.g. 512^3 at
// p = 8^3) stay in L2; a 96 MiB ring (1024^3 at p = 16^3) partly spills to HBM and
// is still faster than the two-kernel schedule.
constexpr int64_t kRingUnitMaxBytes = 32ll << 20;
constexpr int kRingSlots = 3;
constexpr int kRingLag = 1;  // stage 2 of unit u follows stage 1 of unit u + kRingLag (needs kRingLag < kRingSlots)
constexpr long long kSpinLimitNs = 2000000000ll;

}  // namespace

struct Plan {
    int d = 0;
    int64_t n[FFTU_MAX_DIMS] = {};
    int64_t p[FFTU_MAX_DIMS] = {};
    int dtype = 0, dir = 0, device = 0, schedule = 0, precision = 0;
    int64_t N = 0;
    size_t esize = 0;
    void *tables = nullptr;
    size_t table_bytes = 0;
    int64_t table_off[FFTU_MAX_DIMS] = {};
    int64_t line_table_off[FFTU_MAX_DIMS] = {};  // line-pass tables (complex64, len in [256, 2048]), else -1
    void *workspace = nullptr;   // [natural schedule's part | CYCLIC layout temp], plan-owned or caller's
    size_t workspace_bytes = 0;  // bytes the plan allocated itself (0 when the caller supplies it)
    bool ws_owned = false;
    size_t ws_natural = 0;       // bytes the natural schedule needs (ring or two-kernel scratch, ping-pong)
    size_t ws_need = 0;          // total: natural part rounded to 256 B, plus N elements for CYCLIC
    size_t ring_counter_off = 0; // ring schedule: offset of its counters in the workspace
    int layout = 0;              // fftu_layout
    int workspace_mode = 0;      // fftu_workspace_mode
    int tile = 0;                // whole-line tile target of the strided passes (0 = default)
    int radix = 8;               // 8 or 16: stage radix of the strided passes
    int *dstatus = nullptr;
    int tuned = 0;
    std::vector<Step> phase_a, phase_b;
    std::vector<Step> phase_a_inplace;  // used when in == out and phase_a cannot run in place
    bool generic_pingpong = false;      // generic phase A alternates between out and the workspace
    bool axis_pingpong = false;         // ... even in its strided-pass form (a line longer than the tile)

    const void *table(int l) const { return static_cast<const char *>(tables) + table_off[l] * esize; }
    const void *line_table(int l) const {
        return line_table_off[l] < 0 ? nullptr : static_cast<const char *>(tables) + line_table_off[l] * esize;
    }
};

// Sub-FFT length of axis l's phase-A pass when the register-resident line pass serves it, else 0.
inline int64_t line_len(const int64_t *n, const int64_t *p, int l, int dtype, int precision) {
    if (dtype != FFTU_C64 || precision != FFTU_PREC_NATIVE) return 0;
    const int64_t len = n[l] / p[l];
    return (p[l] > 1 && len >= 256 && len <= 2048) ? len : 0;
}

namespace {

// Whole-line tiles aim at this many elements: 256 threads of 16 (complex64) or 8 (complex128)
// values, so that two CTAs share an SM at the kernels' register count.
constexpr int64_t kTileTargetC64 = 4096, kTileTargetC128 = 2048;
// Threads per CTA of a line pass: T threads per line, min(16, max(8, kLineThreads / T)) lines (16 lines of
// 256 points take 256 threads, 8 lines of 2048 points 1024; the 16 / W pad between the lines' shared regions
// needs W <= 16).
constexpr int kLineThreads = 512;

// Generic schedule: one strided pass per axis.  mode 0 = phase A, mode 1 = phase B.
fftu_status make_axis_pass(const Plan &pl, int l, int mode, double scale, AxisPass &a) {
    std::memset(&a, 0, sizeof(a));
    const int is_double = pl.dtype == FFTU_C128;
    int64_t outer = 1, inner = 1;
    for (int k = 0; k < l; ++k) outer *= pl.n[k];
    for (int k = l + 1; k < pl.d; ++k) inner *= pl.n[k];
    const int64_t nl = pl.n[l], Ll = pl.n[l] / pl.p[l];
    const int64_t target = pl.tile > 0 ? pl.tile : (is_double ? kTileTargetC128 : kTileTargetC64);
    const int64_t maxtile = is_double ? kMaxGenericTile / 4 : kMaxGenericTile / 2;
    a.outer = outer;
    a.inner = inner;
    a.nl = (int)nl;
    if (mode == 0) {
        a.len = (int)Ll;
        a.G = (int)pl.p[l];
    } else {
        a.len = (int)pl.p[l];
        a.G = (int)Ll;
    }
    if (a.len > maxtile) {
        set_err("axis %d: sub-FFT length %d exceeds the generic pass tile limit %lld", l, a.len, (long long)maxtile);
        return FFTU_ERR_UNSUPPORTED;
    }
    a.mode = mode;
    a.contiguous = inner == 1;
    a.swz = a.contiguous ? 14 : 0;  // class-strided accesses along contiguous lines: spread the banks
    int64_t V, Gt;
    if (nl <= maxtile) {  // whole lines: the pass can run in place
        V = target / nl;
        if (V < 1) V = 1;
        const int64_t cap = a.contiguous ? outer : inner;
        if (V > cap) V = cap;
        Gt = a.G;
    } else {  // long line: a tile takes Gt of the G classes (runs of Gt along the line, or V across it)
        V = a.contiguous ? 1 : (inner < (is_double ? 4 : 8) ? inner : (is_double ? 4 : 8));
        while (V > 1 && a.len * V > maxtile) V /= 2;  // one sub-FFT of every vector must fit the tile
        Gt = (target < maxtile ? target : maxtile) / (a.len * V);  // classes per tile, up to the tile target
        if (Gt < 1) Gt = 1;
        if (Gt > a.G) Gt = a.G;
    }
    a.V = (int)V;
    a.Gt = (int)Gt;
    a.nlt = (int)(Gt * a.len);
    a.tile = (int)(a.nlt * V);
    const int64_t chunks = a.G / a.Gt;
    a.tiles = (a.contiguous ? outer / V : outer * (inner / V)) * chunks;
    a.lg_V = ilog2(a.V);
    a.lg_Gt = ilog2(a.Gt);
    a.lg_nlt = ilog2(a.nlt);
    a.lg_len = ilog2(a.len);
    a.lg_G = ilog2(a.G);
    a.lg_chunks = ilog2(chunks);
    a.lg_tpo = a.contiguous ? 0 : ilog2(inner / V);
    const int ept = is_double ? kEptMax / 2 : kEptMax;
    if (a.tile > 512 * ept) {  // a block of at most 512 threads holds ept values per thread and stage
        set_err("axis %d: tile of %d elements exceeds 512 threads x %d", l, a.tile, ept);
        return FFTU_ERR_UNSUPPORTED;
    }
    int th = (a.tile + ept - 1) / ept;
    th = ((th + 31) / 32) * 32;
    if (th < 32) th = 32;
    if (th > 512) th = 512;
    a.threads = th;
    a.tw = pl.table(l);
    a.status = pl.dstatus;
    a.scale = scale;
    // tc: 1 / 2 split-precision tensor-core radix-16 stages, 3 CUDA-core radix-16 stages, 0 radix 8
    a.tc = pl.precision ? pl.precision : (pl.radix == 16 ? 3 : 0);
    a.nstages = a.tc ? radix_plan_tc(a.len, a.radix) : radix_plan(a.len, a.radix);
    return FFTU_OK;
}

bool make_phase_b_fused(const Plan &pl, double scale, PhaseBFused &b) {
    std::memset(&b, 0, sizeof(b));
    const size_t es = pl.esize;
    int P = 1;
    for (int l = 0; l < pl.d; ++l) {
        if (pl.p[l] > 16) return false;
        P *= (int)pl.p[l];
    }
    b.data = nullptr;
    b.d = pl.d;
    int64_t stride = 1;
    for (int l = pl.d - 1; l >= 0; --l) {
        b.n[l] = pl.n[l];
        b.p[l] = (int)pl.p[l];
        b.L[l] = pl.n[l] / pl.p[l];
        b.stride[l] = stride;
        stride *= pl.n[l];
    }
    b.P = P;
    for (int l = 0; l < pl.d; ++l) {
        b.lg_p[l] = ilog2(b.p[l]);
        b.lg_L[l] = ilog2(b.L[l]);
    }
    const size_t budget = 64 * 1024;
    int64_t Mt = b.L[pl.d - 1];
    while (Mt > 1 && (size_t)P * Mt * es > budget) Mt /= 2;
    if ((size_t)P * Mt * es > (size_t)kMaxDynSmem) return false;
    b.Mt = (int)Mt;
    b.lg_Mt = ilog2(Mt);
    // complex64: the first DFT pass (the same grouping as the device's phaseb_dfts) reads runs of S = Mt
    // elements, groups S R apart; for S < 16 a warp's runs would share 8-byte slots, so bits
    // [log2 S R, + log2 16/S) of the tile index are XORed into bits [log2 S, 4).  Only where that first
    // pass is a single axis: with a two-axis first pass (e.g. 32^5 at p = 4^5) the index arithmetic on
    // every shared access measured slower than the conflicts it removes (phase B 0.152 -> 0.173 ms), with
    // a single axis faster (64^4 at p = 8^4: 0.147 -> 0.111 ms).
    b.swz_src = b.swz_mask = b.swz_dst = 0;
    if (es == 8) {
        int S = (int)Mt, R = 0;
        bool paired = false;
        for (int l = pl.d - 1; l >= 0 && R == 0; --l) {
            const int pp = (l > 0 && b.p[l] > 1 && b.p[l - 1] > 1) ? b.p[l] * b.p[l - 1] : 0;
            if (pp > 0 && pp <= 16) {
                R = pp;
                paired = true;
            } else if (b.p[l] > 1) {
                R = b.p[l];
            } else {
                S *= b.p[l];
            }
        }
        if (R > 0 && !paired && S < 16 && S * R >= 16) {
            b.swz_src = ilog2(S * R);
            b.swz_mask = 16 / S - 1;
            b.swz_dst = ilog2(S);
        }
    }
    int64_t groups = 1;
    for (int l = 0; l < pl.d - 1; ++l) groups *= b.L[l];
    b.tiles = groups * (b.L[pl.d - 1] / Mt);
    b.threads = 256;
    b.scale = scale;
    return true;
}

// The register-resident form of axis l's phase-A pass (line_pass.cu), when it serves the axis.
bool make_line_pass(const Plan &pl, int l, LinePass &a) {
    std::memset(&a, 0, sizeof(a));
    const int64_t len = line_len(pl.n, pl.p, l, pl.dtype, pl.precision);
    if (len == 0 || !pl.line_table(l)) return false;
    int64_t outer = 1, inner = 1;
    for (int k = 0; k < l; ++k) outer *= pl.n[k];
    for (int k = l + 1; k < pl.d; ++k) inner *= pl.n[k];
    a.outer = outer;
    a.inner = inner;
    a.nl = (int)pl.n[l];
    a.len = (int)len;
    a.G = (int)pl.p[l];
    a.T = (int)(len / 16);
    a.contiguous = inner == 1;
    int W = std::min(16, std::max(8, kLineThreads / a.T));  // lines per CTA
    if (a.contiguous) {
        a.Wc = (int)std::min<int64_t>(W, a.G);
        a.Wo = (int)std::min<int64_t>(W / a.Wc, outer);
        W = a.Wc * a.Wo;
        a.ctas = (outer / a.Wo) * (a.G / a.Wc);
    } else {
        W = (int)std::min<int64_t>(W, inner);
        a.Wc = 1;
        a.Wo = 1;
        a.ctas = outer * a.G * (inner / W);
    }
    a.W = W;
    a.lg_W = ilog2(W);
    a.lg_Wc = ilog2(a.Wc);
    a.pad = W >= 2 ? 16 / W : 0;
    a.threads = a.T * W;
    a.smem = (size_t)W * (size_t)(len + a.pad) * pl.esize;
    if (a.threads < 32 || a.threads > (a.T == 128 ? 1024 : 512) || a.smem > (size_t)kMaxDynSmem ||
        a.ctas > 0x7fffffffll)
        return false;
    a.tw = pl.table(l);
    a.tw1 = pl.line_table(l);
    a.tw2 = static_cast<const char *>(pl.line_table(l)) + len * pl.esize;
    a.twp = static_cast<const char *>(pl.line_table(l)) + (len + len / 16) * pl.esize;
    return true;
}

// Axes a = b - 1 and b in one register-resident pass (pair_pass.cu), when it serves them.
bool make_pair_pass(const Plan &pl, int b, PairPass &a) {
    std::memset(&a, 0, sizeof(a));
    if (b < 1 || pl.dtype != FFTU_C64 || pl.precision != FFTU_PREC_NATIVE) return false;
    const int ax = b - 1;
    if (pl.p[ax] < 2 || pl.p[b] < 2) return false;
    const int64_t L = pl.n[b] / pl.p[b];
    if (pl.n[ax] / pl.p[ax] != L || (L != 8 && L != 16) || pl.p[ax] * pl.p[b] < 16) return false;
    int64_t outer = 1, inner = 1;
    for (int k = 0; k < ax; ++k) outer *= pl.n[k];
    for (int k = b + 1; k < pl.d; ++k) inner *= pl.n[k];
    const int64_t per_item = pl.p[ax] * pl.p[b] * L;  // threads per item
    if (per_item > 1024) return false;
    a.outer = outer;
    a.inner = inner;
    a.na = (int)pl.n[ax];
    a.nb = (int)pl.n[b];
    a.pa = (int)pl.p[ax];
    a.pb = (int)pl.p[b];
    a.L = (int)L;
    a.lg_pa = ilog2(a.pa);
    a.lg_pb = ilog2(a.pb);
    a.contiguous = inner == 1;
    int64_t W;
    if (a.contiguous) {  // adjacent planes: up to 512 threads
        W = std::max<int64_t>(1, 512 / per_item);
        W = std::min(W, outer);
        a.ctas = outer / W;
        a.pad = 0;
    } else {  // adjacent inner positions: runs of W elements, at least 4
        W = std::min<int64_t>(std::min<int64_t>(16, 1024 / per_item), inner);
        if (W < 4) return false;
        a.ctas = outer * (inner / W);
        a.pad = (int)(16 / W);
    }
    a.W = (int)W;
    a.lg_W = ilog2(a.W);
    a.threads = (int)(W * per_item);
    a.smem = (size_t)W * (size_t)(per_item * L + a.pad) * pl.esize;
    if (a.smem > (size_t)kMaxDynSmem || a.ctas > 0x7fffffffll) return false;
    a.twa = pl.table(ax);
    a.twb = pl.table(b);
    return true;
}

// The last three axes in one register-resident pass (triple_pass.cu), when it serves them.
bool make_triple_pass(const Plan &pl, TriplePass &a) {
    std::memset(&a, 0, sizeof(a));
    const int c = pl.d - 1, b = c - 1, ax = c - 2;
    if (pl.d < 3 || pl.dtype != FFTU_C64 || pl.precision != FFTU_PREC_NATIVE) return false;
    for (int l = ax; l <= c; ++l)
        if (pl.p[l] < 2 || pl.n[l] != 8 * pl.p[l]) return false;
    if (pl.p[b] * pl.p[c] != 16) return false;
    int64_t outer = 1;
    for (int k = 0; k < ax; ++k) outer *= pl.n[k];
    a.outer = outer;
    a.na = (int)pl.n[ax];
    a.nb = (int)pl.n[b];
    a.nc = (int)pl.n[c];
    a.pa = (int)pl.p[ax];
    a.pb = (int)pl.p[b];
    a.pc = (int)pl.p[c];
    a.lg_pa = ilog2(a.pa);
    a.lg_pc = ilog2(a.pc);
    a.ctas = outer * a.pa;
    a.smem = (size_t)8192 * pl.esize;
    if (a.ctas > 0x7fffffffll) return false;
    a.twa = pl.table(ax);
    a.twb = pl.table(b);
    a.twc = pl.table(c);
    return true;
}

fftu_status build_generic_phase_a(Plan &pl, std::vector<Step> &out, bool allow_line) {
    // Contiguous axis first (reads the caller's array in long runs).  Out of place, two adjacent axes
    // with short sub-FFTs go through HBM once (pair pass); long sub-FFTs take the line pass.
    for (int l = pl.d - 1; l >= 0; --l) {
        if (pl.n[l] == 1) continue;
        Step s;
        std::memset(&s.line, 0, sizeof(s.line));
        std::memset(&s.pair, 0, sizeof(s.pair));
        std::memset(&s.triple, 0, sizeof(s.triple));
        std::memset(&s.axis2, 0, sizeof(s.axis2));
        std::memset(&s.axis3, 0, sizeof(s.axis3));
        s.kind = STEP_AXIS;
        fftu_status st = make_axis_pass(pl, l, 0, 1.0, s.axis);
        if (st != FFTU_OK) return st;
        if (allow_line && l == pl.d - 1 && make_triple_pass(pl, s.triple)) {
            st = make_axis_pass(pl, l - 1, 0, 1.0, s.axis2);
            if (st == FFTU_OK) st = make_axis_pass(pl, l - 2, 0, 1.0, s.axis3);
            if (st != FFTU_OK) return st;
            s.kind = STEP_TRIPLE;
            out.push_back(s);
            l -= 2;
            continue;
        }
        if (allow_line && l >= 1 && pl.n[l - 1] > 1 && make_pair_pass(pl, l, s.pair)) {
            st = make_axis_pass(pl, l - 1, 0, 1.0, s.axis2);
            if (st != FFTU_OK) return st;
            s.kind = STEP_PAIR;
            out.push_back(s);
            --l;
            continue;
        }
        if (allow_line && make_line_pass(pl, l, s.line)) s.kind = STEP_LINE;
        out.push_back(s);
    }
    return FFTU_OK;
}

// Fused 3D phase A when an instantiation matches; allocates the workspace.
fftu_status build_fused_phase_a(Plan &pl, bool *used) {
    *used = false;
    Phase3Info info;
    const int which = phase_a3_select(pl.d, pl.n, pl.p, pl.dtype == FFTU_C128, &info);
    if (which < 0) return FFTU_OK;
    Step s;
    std::memset(&s.a3, 0, sizeof(s.a3));
    s.kind = STEP_PHASE_A3;
    Phase3Launch &l = s.a3;
    l.which = which;
    l.dir = pl.dir;
    l.p0 = (int)pl.p[0];
    l.p1 = (int)pl.p[1];
    l.n0 = (int)pl.n[0];
    l.n1 = (int)pl.n[1];
    l.tw[0] = pl.table(0);
    l.tw[1] = pl.table(1);
    l.tw[2] = pl.table(2);
    l.status = pl.dstatus;
    l.spin_limit_ns = kSpinLimitNs;
    size_t smem = 0;
    int grids[3] = {0, 0, 0};
    cudaError_t e = prepare_phase_a3(which, pl.dir, l.n0, l.n1, grids, &smem);
    l.grid1 = grids[0];
    l.grid2 = grids[1];
    l.grid = grids[2];
    if (e != cudaSuccess) return cuda_fail(e, "fused phase A attributes");
    const int64_t unit_bytes = info.unit_elems * (int64_t)pl.esize;
    const int64_t units = pl.p[0] * pl.p[1];
    size_t ws;
    if (unit_bytes <= kRingUnitMaxBytes && units > kRingSlots && units > kRingLag) {
        l.mode = 1;
        l.ring = kRingSlots;
        l.lag = kRingLag;
        ws = (size_t)kRingSlots * unit_bytes + 256 + sizeof(unsigned) * (size_t)(1 + 2 * units);
    } else {
        l.mode = 0;
        l.ring = 0;
        ws = (size_t)pl.N * pl.esize;
    }
    pl.ws_natural = ws;  // scratch and counters are bound to the workspace once it exists
    if (l.mode == 1) pl.ring_counter_off = ((size_t)kRingSlots * unit_bytes + 255) / 256 * 256;
    pl.phase_a.push_back(s);
    *used = true;
    return FFTU_OK;
}

fftu_status build_schedule(Plan &pl, int sched) {
    const double scale = pl.dir == FFTU_INVERSE ? 1.0 / (double)pl.N : 1.0;
    bool fused_a = false;
    if (sched != FFTU_SCHED_GENERIC && sched != FFTU_SCHED_GENERIC_A) {
        fftu_status st = build_fused_phase_a(pl, &fused_a);
        if (st != FFTU_OK) return st;
    }
    {
        // line passes are never in place: only the plain phase-A list takes them
        fftu_status st = build_generic_phase_a(pl, fused_a ? pl.phase_a_inplace : pl.phase_a, !fused_a);
        if (st != FFTU_OK) return st;
    }
    if (!fused_a) {
        // a pass over part of the classes of a line, or a line pass, is not in place: alternate with a
        // workspace
        for (const Step &s : pl.phase_a) {
            const bool long_line = !s.whole_lines();
            if (long_line) pl.axis_pingpong = true;
            if (s.kind != STEP_AXIS || long_line) pl.generic_pingpong = true;
        }
        if (pl.generic_pingpong) pl.ws_natural = (size_t)pl.N * pl.esize;
    }
    // Phase B: one fused pass when every p_l <= 16, else one pass per axis.
    Step s;
    const int is_double = pl.dtype == FFTU_C128;
    const int mt3 = pl.d == 3 && pl.p[0] > 1 ? phase_b3_tile_mt((int)pl.p[0], (int)pl.p[1], (int)pl.p[2], is_double)
                                             : 0;
    if (sched != FFTU_SCHED_GENERIC && mt3 > 0 && (pl.n[2] / pl.p[2]) % mt3 == 0 &&
        make_phase_b_fused(pl, scale, s.pb)) {
        s.kind = STEP_PHASE_B3;
        s.pb.Mt = mt3;
        s.pb.tiles = (pl.n[0] / pl.p[0]) * (pl.n[1] / pl.p[1]) * ((pl.n[2] / pl.p[2]) / mt3);
        pl.phase_b.push_back(s);
    } else if (sched != FFTU_SCHED_GENERIC && make_phase_b_fused(pl, scale, s.pb)) {
        s.kind = STEP_PHASE_B_FUSED;
        pl.phase_b.push_back(s);
    } else {
        int last = -1;
        for (int l = 0; l < pl.d; ++l)
            if (pl.p[l] > 1) last = l;
        if (last < 0) last = pl.d - 1;  // every p_l = 1: a single pass applies the scale
        for (int l = pl.d - 1; l >= 0; --l) {
            if (pl.p[l] == 1 && l != last) continue;
            Step t;
            t.kind = STEP_AXIS;
            fftu_status st = make_axis_pass(pl, l, 1, l == last ? scale : 1.0, t.axis);
            if (st != FFTU_OK) return st;
            pl.phase_b.push_back(t);
        }
    }
    pl.schedule = sched == FFTU_SCHED_GENERIC ? FFTU_SCHED_GENERIC
                  : sched == FFTU_SCHED_GENERIC_A ? FFTU_SCHED_GENERIC_A : FFTU_SCHED_FUSED;
    return FFTU_OK;
}

// Kernel launches one list of steps makes (the two-kernel fused phase A counts 2).
int kernel_count(const std::vector<Step> &steps) {
    int k = 0;
    for (const Step &s : steps) k += (s.kind == STEP_PHASE_A3 && s.a3.mode == 0) ? 2 : 1;
    return k;
}

// Point the steps that use the workspace at pl->workspace (NULL when the caller has not supplied one).
void bind_workspace(Plan *pl) {
    for (Step &s : pl->phase_a)
        if (s.kind == STEP_PHASE_A3) {
            s.a3.scratch = pl->workspace;
            s.a3.counters = pl->workspace && s.a3.mode == 1
                                ? reinterpret_cast<unsigned *>(static_cast<char *>(pl->workspace) + pl->ring_counter_off)
                                : nullptr;
        }
}

void *layout_temp(const Plan *pl) {
    return static_cast<char *>(pl->workspace) + (pl->ws_natural + 255) / 256 * 256;
}

void free_plan(Plan *pl) {
    if (!pl) return;
    if (pl->tables) cudaFree(pl->tables);
    if (pl->workspace && pl->ws_owned) cudaFree(pl->workspace);
    if (pl->dstatus) cudaFree(pl->dstatus);
    delete pl;
}

fftu_status run_steps(Plan *pl, const std::vector<Step> &steps, const void *first_src, void *dst,
                      cudaStream_t st, const void *mul = nullptr) {
    const int is_double = pl->dtype == FFTU_C128;
    const void *src = first_src;
    if (steps.empty() && src != dst) {  // N = 1 or all n_l = 1: the transform is the identity
        cudaError_t e = cudaMemcpyAsync(dst, src, (size_t)pl->N * pl->esize, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "copy");
    }
    for (const Step &s : steps) {
        cudaError_t e;
        if (s.kind == STEP_AXIS) {
            AxisPass a = s.axis;
            a.src = src;
            a.dst = dst;
            e = launch_axis_pass(a, is_double, pl->dir, st);
        } else if (s.kind == STEP_LINE || s.kind == STEP_PAIR || s.kind == STEP_TRIPLE) {
            record_error("internal: a register-resident pass outside the alternating phase-A schedule");
            return FFTU_ERR_INTERNAL;
        } else if (s.kind == STEP_PHASE_A3) {
            Phase3Launch l = s.a3;
            l.in = src;
            l.out = dst;
            e = launch_phase_a3(l, st);
        } else if (s.kind == STEP_PHASE_B3) {
            PhaseBFused b = s.pb;
            b.data = dst;
            b.mul = mul;
            mul = nullptr;  // consumed by the fused store
            e = launch_phase_b3(b, is_double, pl->dir, st);
        } else {
            PhaseBFused b = s.pb;
            b.data = dst;
            e = launch_phase_b_fused(b, is_double, pl->dir, st);
        }
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
        src = dst;
    }
    if (mul) {  // phase B could not fuse the multiply: one extra elementwise pass
        cudaError_t e = launch_pointwise(dst, mul, pl->N, is_double, st);
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    }
    return FFTU_OK;
}

}  // namespace

}  // namespace fftu

using fftu::Plan;

struct fftu_plan_st {
    Plan *impl;
};

namespace fftu {

fftu_status plan_view(fftu_handle h, PlanView *v) {
    if (!h || !h->impl) {
        record_error("batch: NULL plan");
        return FFTU_ERR_ARG;
    }
    const Plan &pl = *h->impl;
    v->dtype = pl.dtype;
    v->dir = pl.dir;
    v->device = pl.device;
    v->pingpong = pl.axis_pingpong;  // the batch runs the strided-pass form of every step
    v->precision = pl.precision;
    v->layout = pl.layout;
    v->radix = pl.radix;
    v->a_passes.clear();
    v->b_steps.clear();
    const bool fused_a = !pl.phase_a.empty() && pl.phase_a[0].kind == STEP_PHASE_A3;
    for (const Step &s : fused_a ? pl.phase_a_inplace : pl.phase_a) {
        StepView sv;
        std::memset(&sv, 0, sizeof(sv));
        sv.is_axis = true;
        sv.axis = s.axis;
        v->a_passes.push_back(sv);
        for (int i = 1; i < s.passes(); ++i) {  // the step's other axes, in their strided-pass form
            sv.axis = s.strided(i);
            v->a_passes.push_back(sv);
        }
    }
    const double scale = pl.dir == FFTU_INVERSE ? 1.0 / (double)pl.N : 1.0;
    for (const Step &s : pl.phase_b) {
        StepView sv;
        std::memset(&sv, 0, sizeof(sv));
        if (s.kind == STEP_AXIS) {
            sv.is_axis = true;
            sv.axis = s.axis;
        } else {
            sv.is_axis = false;
            if (!make_phase_b_fused(pl, scale, sv.pb)) {  // the generic form of the fused phase B
                record_error("batch: phase B has no generic fused form");
                return FFTU_ERR_UNSUPPORTED;
            }
        }
        v->b_steps.push_back(sv);
    }
    return FFTU_OK;
}

}  // namespace fftu

extern "C" {

fftu_status fftu_plan_ex(int d, const int64_t *n, const int64_t *p, fftu_dtype dtype, fftu_dir dir,
                         const fftu_options *opts, fftu_handle *out) {
    using namespace fftu;
    g_err[0] = '\0';
    if (!out) {
        set_err("out is NULL");
        return FFTU_ERR_ARG;
    }
    *out = nullptr;
    if (d < 1 || d > FFTU_MAX_DIMS || !n) {
        set_err("d must be in [1, %d] and n non-NULL", FFTU_MAX_DIMS);
        return FFTU_ERR_ARG;
    }
    if (dtype != FFTU_C64 && dtype != FFTU_C128) {
        set_err("dtype must be FFTU_C64 or FFTU_C128");
        return FFTU_ERR_ARG;
    }
    if (dir != FFTU_FORWARD && dir != FFTU_INVERSE) {
        set_err("dir must be FFTU_FORWARD or FFTU_INVERSE");
        return FFTU_ERR_ARG;
    }
    int sched = opts ? opts->schedule : FFTU_SCHED_AUTO;
    if (sched < FFTU_SCHED_AUTO || sched > FFTU_SCHED_GENERIC_A) {
        set_err("unknown schedule %d", sched);
        return FFTU_ERR_ARG;
    }
    const int precision = opts ? opts->precision : FFTU_PREC_NATIVE;
    if (precision < FFTU_PREC_NATIVE || precision > FFTU_PREC_SPLIT_FP16) {
        set_err("unknown precision %d", precision);
        return FFTU_ERR_ARG;
    }
    const int layout = opts ? opts->layout : FFTU_LAYOUT_NATURAL;
    const int ws_mode = opts ? opts->workspace_mode : FFTU_WORKSPACE_PLAN;
    if (layout != FFTU_LAYOUT_NATURAL && layout != FFTU_LAYOUT_CYCLIC) {
        set_err("unknown layout %d", layout);
        return FFTU_ERR_ARG;
    }
    if (ws_mode != FFTU_WORKSPACE_PLAN && ws_mode != FFTU_WORKSPACE_CALLER) {
        set_err("unknown workspace mode %d", ws_mode);
        return FFTU_ERR_ARG;
    }
    int tile = opts ? opts->tile : 0;
    int radix = opts && opts->radix ? opts->radix : 8;
    if (tile != 0 && (tile < 1024 || tile > (dtype == FFTU_C128 ? 4096 : 8192) || (tile & (tile - 1)))) {
        set_err("tile must be 0 or a power of two in [1024, %d]", dtype == FFTU_C128 ? 4096 : 8192);
        return FFTU_ERR_ARG;
    }
    if (radix != 8 && radix != 16) {
        set_err("radix must be 0, 8 or 16");
        return FFTU_ERR_ARG;
    }
    if (precision != FFTU_PREC_NATIVE) {
        if (dtype != FFTU_C64) {
            set_err("split-precision tensor-core stages are for complex64 plans");
            return FFTU_ERR_UNSUPPORTED;
        }
        if (sched == FFTU_SCHED_FUSED) {
            set_err("split-precision stages run in the strided passes: use AUTO, GENERIC or GENERIC_A");
            return FFTU_ERR_ARG;
        }
        if (sched == FFTU_SCHED_AUTO) sched = FFTU_SCHED_GENERIC_A;
    }
    if (opts)
        for (int r : opts->reserved)
            if (r != 0) {
                set_err("fftu_options.reserved must be zero");
                return FFTU_ERR_ARG;
            }
    int64_t N = 1;
    int64_t pp[FFTU_MAX_DIMS];
    for (int l = 0; l < d; ++l) {
        if (n[l] < 1) {
            set_err("n[%d] = %lld < 1", l, (long long)n[l]);
            return FFTU_ERR_ARG;
        }
        if (n[l] > (int64_t(1) << 40) || N > (int64_t(1) << 40) / n[l]) {
            set_err("N exceeds 2^40 elements");
            return FFTU_ERR_ARG;
        }
        N *= n[l];
        if (p) {
            if (p[l] < 1) {
                set_err("p[%d] = %lld < 1", l, (long long)p[l]);
                return FFTU_ERR_ARG;
            }
            if (p[l] > n[l] / p[l]) {  // p_l^2 > n_l: it cannot divide (and squaring p_l could overflow)
                set_err("p[%d]^2 exceeds n[%d] = %lld (p[%d] = %lld)", l, l, (long long)n[l], l, (long long)p[l]);
                return FFTU_ERR_DIVISIBILITY;
            }
            if (n[l] % (p[l] * p[l]) != 0) {
                set_err("p[%d]^2 = %lld does not divide n[%d] = %lld", l, (long long)(p[l] * p[l]), l,
                        (long long)n[l]);
                return FFTU_ERR_DIVISIBILITY;
            }
            pp[l] = p[l];
        } else {
            // default grid: the largest power of two with p_l^2 | n_l, at most 8
            int64_t q = 1;
            while (q < 8 && n[l] % ((2 * q) * (2 * q)) == 0) q *= 2;
            pp[l] = q;
        }
    }
    for (int l = 0; l < d; ++l)
        if (!is_pow2(n[l])) {
            set_err("n[%d] = %lld is not a power of two (GPU build supports powers of two)", l, (long long)n[l]);
            return FFTU_ERR_UNSUPPORTED;
        }
    int tuned = 0;
    if (!p) {  // measured tuning on request; otherwise wisdom for this problem, if the process has any
        fftu_options base;
        std::memset(&base, 0, sizeof(base));
        if (opts) base = *opts;
        base.schedule = sched;
        TuneChoice tc;
        if (opts && opts->tune ? autotune(d, n, dtype, dir, base, &tc) : wisdom_lookup(d, n, dtype, dir, base, &tc)) {
            for (int l = 0; l < d; ++l) pp[l] = tc.p[l];
            sched = tc.schedule;
            if (tc.tile) tile = tc.tile;
            if (tc.radix) radix = tc.radix;
            tuned = 1;
        }
        g_err[0] = '\0';
    }

    Plan *pl = new (std::nothrow) Plan();
    if (!pl) {
        set_err("host allocation failed");
        return FFTU_ERR_NOMEM;
    }
    pl->d = d;
    for (int l = 0; l < d; ++l) {
        pl->n[l] = n[l];
        pl->p[l] = pp[l];
    }
    pl->dtype = dtype;
    pl->dir = dir;
    pl->tuned = tuned;
    pl->precision = precision;
    pl->layout = layout;
    pl->workspace_mode = ws_mode;
    pl->tile = tile;
    pl->radix = radix;
    pl->N = N;
    pl->esize = dtype == FFTU_C128 ? 16 : 8;
    cudaError_t e = cudaGetDevice(&pl->device);
    if (e != cudaSuccess) {
        free_plan(pl);
        return cuda_fail(e, "cudaGetDevice");
    }
    // twiddle tables: w_{n_l}^e per axis, then the line-pass tables of the axes a line pass can serve
    int64_t off = 0;
    for (int l = 0; l < d; ++l) {
        pl->table_off[l] = off;
        off += n[l];
    }
    for (int l = 0; l < d; ++l) {
        const int64_t len = line_len(n, pp, l, dtype, precision);
        pl->line_table_off[l] = len ? off : -1;
        off += len ? len + len / 16 + n[l] : 0;
    }
    pl->table_bytes = (size_t)off * pl->esize;
    e = cudaMalloc(&pl->tables, pl->table_bytes);
    if (e != cudaSuccess) {
        free_plan(pl);
        set_err("cudaMalloc of %zu table bytes: %s", pl->table_bytes, cudaGetErrorString(e));
        cudaGetLastError();
        return FFTU_ERR_NOMEM;
    }
    // tables and status word on a private stream: planning waits for its own work only, not for
    // transforms in flight on other streams
    cudaStream_t ps = nullptr;
    e = cudaMalloc(&pl->dstatus, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->dstatus, 0, sizeof(int), ps);
    if (e != cudaSuccess) {
        if (ps) cudaStreamDestroy(ps);
        free_plan(pl);
        cudaGetLastError();
        set_err("status word allocation: %s", cudaGetErrorString(e));
        return FFTU_ERR_NOMEM;
    }
    for (int l = 0; l < d && e == cudaSuccess; ++l) {
        e = launch_twiddle_table(static_cast<char *>(pl->tables) + pl->table_off[l] * pl->esize, n[l],
                                 dtype == FFTU_C128, ps);
        if (e == cudaSuccess && pl->line_table_off[l] >= 0)
            e = launch_line_tables(static_cast<char *>(pl->tables) + pl->line_table_off[l] * pl->esize,
                                   (int)(n[l] / pp[l]), (int)n[l], ps);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ps);
    cudaStreamDestroy(ps);
    if (e != cudaSuccess) {
        free_plan(pl);
        return cuda_fail(e, "twiddle table generation");
    }
    e = prepare_axis_pass(dtype == FFTU_C128, dir);
    if (e == cudaSuccess) e = prepare_phase_b_fused(dtype == FFTU_C128, dir);
    if (e == cudaSuccess) e = prepare_phase_b3(dtype == FFTU_C128, dir);
    if (e == cudaSuccess && dtype == FFTU_C64) e = prepare_line_pass(dir);
    if (e == cudaSuccess && dtype == FFTU_C64) e = prepare_pair_pass(dir);
    if (e == cudaSuccess && dtype == FFTU_C64) e = prepare_triple_pass(dir);
    if (e != cudaSuccess) {
        free_plan(pl);
        return cuda_fail(e, "kernel attributes");
    }
    fftu_status st = build_schedule(*pl, sched);
    if (st != FFTU_OK) {
        free_plan(pl);
        return st;
    }
    // one workspace: the natural schedule's part, then N elements for the CYCLIC permutations
    pl->ws_need = pl->ws_natural == 0 && layout == FFTU_LAYOUT_NATURAL
                      ? 0
                      : (pl->ws_natural + 255) / 256 * 256 +
                            (layout == FFTU_LAYOUT_CYCLIC ? (size_t)pl->N * pl->esize : 0);
    if (pl->ws_need > 0 && ws_mode == FFTU_WORKSPACE_PLAN) {
        e = cudaMalloc(&pl->workspace, pl->ws_need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_err("cudaMalloc of %zu workspace bytes: %s", pl->ws_need, cudaGetErrorString(e));
            free_plan(pl);
            return FFTU_ERR_NOMEM;
        }
        pl->ws_owned = true;
        pl->workspace_bytes = pl->ws_need;
    }
    bind_workspace(pl);
    fftu_plan_st *h = new (std::nothrow) fftu_plan_st;
    if (!h) {
        free_plan(pl);
        set_err("host allocation failed");
        return FFTU_ERR_NOMEM;
    }
    h->impl = pl;
    *out = h;
    return FFTU_OK;
}

fftu_status fftu_plan(int d, const int64_t *n, const int64_t *p, fftu_dtype dtype, fftu_dir dir,
                      fftu_handle *out) {
    return fftu_plan_ex(d, n, p, dtype, dir, nullptr, out);
}

}  // extern "C"

namespace fftu {
namespace {

// The transform on the natural view (every layout ends up here).
fftu_status exec_natural(Plan *pl, fftu_phase phase, const void *in, void *out, cudaStream_t st) {
    if ((phase & FFTU_PHASE_A) && pl->generic_pingpong) {
        // buffers: pass k (of np) writes out when np - k is even, the workspace otherwise.  In place with
        // np odd, the first pass runs in place on out in its strided-pass form (whole lines only).
        const int np = (int)pl->phase_a.size();
        const void *src = in;
        for (int k = 1; k <= np; ++k) {
            const Step &s = pl->phase_a[k - 1];
            void *dst = ((np - k) % 2 == 0) ? out : pl->workspace;
            const bool whole_lines = s.whole_lines();
            if (dst == src && !(k == 1 && whole_lines && src == out)) {
                set_err("in-place transform with a long-line axis needs in != out");
                return FFTU_ERR_UNSUPPORTED;
            }
            cudaError_t e;
            if (dst == src) {  // the in-place first step: its strided passes, then the alternation continues
                e = cudaSuccess;
                for (int i = 0; i < s.passes() && e == cudaSuccess; ++i) {
                    AxisPass a = s.strided(i);
                    a.src = out;
                    a.dst = out;
                    e = launch_axis_pass(a, pl->dtype == FFTU_C128, pl->dir, st);
                }
            } else if (s.kind == STEP_TRIPLE) {
                TriplePass a = s.triple;
                a.src = src;
                a.dst = dst;
                e = launch_triple_pass(a, pl->dir, st);
            } else if (s.kind == STEP_PAIR) {
                PairPass a = s.pair;
                a.src = src;
                a.dst = dst;
                e = launch_pair_pass(a, pl->dir, st);
            } else if (s.kind == STEP_LINE) {
                LinePass a = s.line;
                a.src = src;
                a.dst = dst;
                e = launch_line_pass(a, pl->dir, st);
            } else {
                AxisPass a = s.axis;
                a.src = src;
                a.dst = dst;
                e = launch_axis_pass(a, pl->dtype == FFTU_C128, pl->dir, st);
            }
            if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
            src = dst;
        }
        phase = (fftu_phase)(phase & ~FFTU_PHASE_A);
    }
    if (phase & FFTU_PHASE_A) {
        // the persistent phase-A kernel reads `in` while writing `out`; in place it
        // would overwrite inputs other units have not read yet
        const bool ring_inplace = in == out && !pl->phase_a_inplace.empty() && pl->phase_a.size() == 1 &&
                                  pl->phase_a[0].kind == STEP_PHASE_A3 && pl->phase_a[0].a3.mode == 1;
        fftu_status s = run_steps(pl, ring_inplace ? pl->phase_a_inplace : pl->phase_a, in, out, st);
        if (s != FFTU_OK) return s;
    }
    if (phase & FFTU_PHASE_B) {
        fftu_status s = run_steps(pl, pl->phase_b, out, out, st);
        if (s != FFTU_OK) return s;
    }
    return FFTU_OK;
}

// CYCLIC layout: permute to the natural view, run it, permute back (see fftu_layout).
fftu_status exec_cyclic(Plan *pl, fftu_phase phase, const void *in, void *out, cudaStream_t st) {
    const int dbl = pl->dtype == FFTU_C128;
    const size_t bytes = (size_t)pl->N * pl->esize;
    void *tmp = layout_temp(pl);
    cudaError_t e;
    if (!(phase & FFTU_PHASE_A)) {  // phase B alone, in place on out
        e = launch_cyclic_permute(out, tmp, pl->d, pl->n, pl->p, dbl, 0, st);
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
        fftu_status s = exec_natural(pl, phase, tmp, tmp, st);
        if (s != FFTU_OK) return s;
        e = launch_cyclic_permute(tmp, out, pl->d, pl->n, pl->p, dbl, 1, st);
        return e == cudaSuccess ? FFTU_OK : cuda_fail(e, "kernel launch");
    }
    if (in != out) {  // natural input in out, natural result in tmp, back to CYCLIC in out
        e = launch_cyclic_permute(in, out, pl->d, pl->n, pl->p, dbl, 0, st);
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
        fftu_status s = exec_natural(pl, phase, out, tmp, st);
        if (s != FFTU_OK) return s;
        e = launch_cyclic_permute(tmp, out, pl->d, pl->n, pl->p, dbl, 1, st);
        return e == cudaSuccess ? FFTU_OK : cuda_fail(e, "kernel launch");
    }
    // in place: natural input in tmp, natural result in out, CYCLIC result in tmp, copied to out
    e = launch_cyclic_permute(in, tmp, pl->d, pl->n, pl->p, dbl, 0, st);
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    fftu_status s = exec_natural(pl, phase, tmp, out, st);
    if (s != FFTU_OK) return s;
    e = launch_cyclic_permute(out, tmp, pl->d, pl->n, pl->p, dbl, 1, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? FFTU_OK : cuda_fail(e, "kernel launch");
}

}  // namespace
}  // namespace fftu

extern "C" {

fftu_status fftu_exec_phase(fftu_handle h, fftu_phase phase, const void *in, void *out, void *stream) {
    using namespace fftu;
    g_err[0] = '\0';
    if (!h || !h->impl) {
        set_err("plan is NULL");
        return FFTU_ERR_ARG;
    }
    Plan *pl = h->impl;
    if (phase != FFTU_PHASE_A && phase != FFTU_PHASE_B && phase != FFTU_PHASE_ALL) {
        set_err("unknown phase %d", (int)phase);
        return FFTU_ERR_ARG;
    }
    if (!out || ((phase & FFTU_PHASE_A) && !in)) {
        set_err("in/out must be non-NULL device pointers");
        return FFTU_ERR_ARG;
    }
    if (phase == FFTU_PHASE_B && in && in != out) {
        set_err("phase B runs in place: in must be NULL or equal to out");
        return FFTU_ERR_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) {
        set_err("in/out must be 16-byte aligned");
        return FFTU_ERR_ARG;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != pl->device) {
        set_err("plan was made on device %d, current device is %d", pl->device, dev);
        return FFTU_ERR_ARG;
    }
    if (pl->ws_need > 0 && !pl->workspace) {
        set_err("the plan has no workspace: supply one with fftu_set_workspace");
        return FFTU_ERR_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return pl->layout == FFTU_LAYOUT_CYCLIC ? exec_cyclic(pl, phase, in, out, st) : exec_natural(pl, phase, in, out, st);
}

fftu_status fftu_exec(fftu_handle h, const void *in, void *out, void *stream) {
    return fftu_exec_phase(h, FFTU_PHASE_ALL, in, out, stream);
}

fftu_status fftu_exec_pointwise(fftu_handle fwd, fftu_handle inv, const void *in, const void *mul, void *tmp,
                                void *out, void *stream) {
    using namespace fftu;
    g_err[0] = '\0';
    if (!fwd || !inv || !fwd->impl || !inv->impl) {
        set_err("plans must be non-NULL");
        return FFTU_ERR_ARG;
    }
    Plan *pf = fwd->impl, *pi = inv->impl;
    if (pf->dir != FFTU_FORWARD || pi->dir != FFTU_INVERSE) {
        set_err("fwd must be a forward plan and inv an inverse plan");
        return FFTU_ERR_ARG;
    }
    bool same = pf->d == pi->d && pf->dtype == pi->dtype && pf->device == pi->device;
    for (int l = 0; same && l < pf->d; ++l) same = pf->n[l] == pi->n[l] && pf->p[l] == pi->p[l];
    if (!same) {
        set_err("fwd and inv must have the same shape, cyclic grid, dtype and device");
        return FFTU_ERR_ARG;
    }
    if (pf->layout != FFTU_LAYOUT_NATURAL || pi->layout != FFTU_LAYOUT_NATURAL) {
        set_err("fftu_exec_pointwise takes NATURAL-layout plans");
        return FFTU_ERR_UNSUPPORTED;
    }
    if ((pf->ws_need > 0 && !pf->workspace) || (pi->ws_need > 0 && !pi->workspace)) {
        set_err("a plan has no workspace: supply one with fftu_set_workspace");
        return FFTU_ERR_ARG;
    }
    if (!in || !mul || !tmp || !out || tmp == out || mul == tmp) {
        set_err("in, mul, tmp, out must be non-NULL; tmp must differ from out and mul");
        return FFTU_ERR_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(mul) | reinterpret_cast<uintptr_t>(tmp) |
         reinterpret_cast<uintptr_t>(out)) & 15) {
        set_err("in/mul/tmp/out must be 16-byte aligned");
        return FFTU_ERR_ARG;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != pf->device) {
        set_err("plan was made on device %d, current device is %d", pf->device, dev);
        return FFTU_ERR_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // forward into tmp, the product fused into the forward phase B store
    const bool ring_inplace = in == tmp && pf->phase_a.size() == 1 && pf->phase_a[0].kind == STEP_PHASE_A3 &&
                              pf->phase_a[0].a3.mode == 1 && !pf->phase_a_inplace.empty();
    fftu_status s = FFTU_OK;
    if (pf->generic_pingpong) {
        s = fftu_exec_phase(fwd, FFTU_PHASE_A, in, tmp, stream);
    } else {
        s = run_steps(pf, ring_inplace ? pf->phase_a_inplace : pf->phase_a, in, tmp, st);
    }
    if (s != FFTU_OK) return s;
    s = run_steps(pf, pf->phase_b, tmp, tmp, st, mul);
    if (s != FFTU_OK) return s;
    // inverse from tmp into out (same distribution: no reordering in between)
    return fftu_exec_phase(inv, FFTU_PHASE_ALL, tmp, out, stream);
}

fftu_status fftu_destroy(fftu_handle h) {
    using namespace fftu;
    g_err[0] = '\0';
    if (!h) return FFTU_OK;
    Plan *pl = h->impl;
    fftu_status rc = FFTU_OK;
    if (pl) {
        int prev = -1;
        const int dev = pl->device;
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = cuda_fail(e, "synchronize before destroy");
        free_plan(pl);
        if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    }
    delete h;
    return rc;
}

fftu_status fftu_plan_info(fftu_handle h, fftu_info *info) {
    using namespace fftu;
    if (!h || !h->impl || !info) {
        set_err("plan and info must be non-NULL");
        return FFTU_ERR_ARG;
    }
    const Plan *pl = h->impl;
    std::memset(info, 0, sizeof(*info));
    info->d = pl->d;
    for (int l = 0; l < pl->d; ++l) {
        info->n[l] = pl->n[l];
        info->p[l] = pl->p[l];
    }
    info->dtype = pl->dtype;
    info->dir = pl->dir;
    info->schedule = pl->schedule;
    info->launches_phase_a = kernel_count(pl->phase_a);
    info->launches_phase_b = kernel_count(pl->phase_b);
    info->N = pl->N;
    info->alg_bytes = 4 * pl->N * (int64_t)pl->esize;
    info->table_bytes = (int64_t)pl->table_bytes;
    info->workspace_bytes = (int64_t)pl->workspace_bytes;
    info->tuned = pl->tuned;
    info->precision = pl->precision;
    info->workspace_need = (int64_t)pl->ws_need;
    info->layout = pl->layout;
    info->workspace_mode = pl->workspace_mode;
    info->tile = pl->tile > 0 ? pl->tile : (pl->dtype == FFTU_C128 ? (int)kTileTargetC128 : (int)kTileTargetC64);
    info->radix = pl->radix;
    return FFTU_OK;
}

fftu_status fftu_workspace_size(fftu_handle h, size_t *bytes) {
    using namespace fftu;
    if (!h || !h->impl || !bytes) {
        set_err("plan and bytes must be non-NULL");
        return FFTU_ERR_ARG;
    }
    *bytes = h->impl->ws_need;
    return FFTU_OK;
}

fftu_status fftu_set_workspace(fftu_handle h, void *workspace, size_t bytes) {
    using namespace fftu;
    g_err[0] = '\0';
    if (!h || !h->impl) {
        set_err("plan is NULL");
        return FFTU_ERR_ARG;
    }
    Plan *pl = h->impl;
    if (workspace && (bytes < pl->ws_need || (reinterpret_cast<uintptr_t>(workspace) & 255))) {
        set_err("workspace must hold %zu bytes and be 256-byte aligned", pl->ws_need);
        return FFTU_ERR_ARG;
    }
    if (pl->ws_owned && pl->workspace) {
        cudaError_t e = cudaDeviceSynchronize();  // execs in flight may still use it
        if (e != cudaSuccess) return cuda_fail(e, "synchronize before freeing the workspace");
        cudaFree(pl->workspace);
    }
    pl->workspace = workspace;
    pl->ws_owned = false;
    pl->workspace_bytes = 0;
    bind_workspace(pl);
    return FFTU_OK;
}

fftu_status fftu_check_device_status(fftu_handle h) {
    using namespace fftu;
    if (!h || !h->impl) {
        set_err("plan is NULL");
        return FFTU_ERR_ARG;
    }
    Plan *pl = h->impl;
    int v = 0;
    cudaError_t e = cudaMemcpy(&v, pl->dstatus, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(pl->dstatus, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "status word read");
    if (v == 0) return FFTU_OK;
    set_err("device status word = %d", v);
    return v == FFTU_ERR_TIMEOUT ? FFTU_ERR_TIMEOUT : FFTU_ERR_INTERNAL;
}

const char *fftu_status_string(fftu_status s) {
    switch (s) {
        case FFTU_OK: return "FFTU_OK";
        case FFTU_ERR_ARG: return "FFTU_ERR_ARG: invalid argument";
        case FFTU_ERR_DIVISIBILITY: return "FFTU_ERR_DIVISIBILITY: p_l^2 must divide n_l";
        case FFTU_ERR_UNSUPPORTED: return "FFTU_ERR_UNSUPPORTED: not supported by this GPU build";
        case FFTU_ERR_NOMEM: return "FFTU_ERR_NOMEM: device allocation failed";
        case FFTU_ERR_CUDA: return "FFTU_ERR_CUDA: CUDA runtime error";
        case FFTU_ERR_TIMEOUT: return "FFTU_ERR_TIMEOUT: bounded device wait expired";
        case FFTU_ERR_INTERNAL: return "FFTU_ERR_INTERNAL: device consistency check failed";
    }
    return "FFTU status: unknown code";
}

const char *fftu_last_error(void) { return fftu::g_err; }

const char *fftu_version(void) { return "fftu 0.1.0 sm_103a"; }

}  // extern "C"
