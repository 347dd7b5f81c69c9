// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/fftu.h"

namespace fftu {

constexpr int kMaxStages = 24;
constexpr int kEptMax = 16;            // complex values a thread holds per stage of the generic pass
constexpr int kMaxGenericTile = 16384; // elements per tile of the generic pass (kEptMax * 1024 threads)
constexpr int kMaxDynSmem = 200 * 1024; // dynamic shared memory ceiling requested for any kernel

// One strided sub-FFT pass along one axis (generic schedule).
//
// The array is viewed as [outer][nl][inner].  A line (fixed outer, inner) of
// nl = len * G elements splits into G classes; class c holds the elements at
// line positions c + j G, j in [len].  Each class gets a length-len DFT.
//   mode 0 (phase A, Superstep 0 + Put): class c = residue s of the cyclic
//     distribution (G = p_l, len = n_l/p_l); output m is multiplied by the
//     twiddle w_{n_l}^{m s} and stored at line position s len + m.
//   mode 1 (phase B, Superstep 2): class c = local index m (G = n_l/p_l,
//     len = p_l); output k is stored in place at c + k G, times `scale`.
struct AxisPass {
    const void *src;
    void *dst;
    int64_t outer, inner;
    int nl, len, G;
    int mode;
    int V;            // vectors per tile: inner indices (strided axis) or lines (contiguous axis)
    int contiguous;   // inner == 1
    int Gt;           // classes per tile (G for whole lines; fewer for long lines)
    int nlt;          // Gt * len: tile line length
    // log2 of the power-of-two sizes above (index arithmetic uses shifts and masks)
    int lg_V, lg_Gt, lg_nlt, lg_len, lg_G, lg_chunks, lg_tpo;
    int tile;         // nlt * V
    int threads;
    const void *tw;   // w_{nl}^e, e in [nl] (forward roots)
    double scale;
    int nstages;
    int radix[kMaxStages];
    int64_t tiles;
    int tc;           // 0: radix 8 after a smaller first stage; 1 / 2: radix-16 stages as split bfloat16 /
                      // float16 tcgen05 MMAs; 3: radix-16 CUDA-core stages; (1-3: the remaining factor last)
    int *status;      // plan status word (bounded waits of the tensor-core stages), may be NULL
    int swz;          // shared-memory swizzle mask of the tile (14: bits 1-3 ^= bits 4-6, contiguous passes; 0: none)
};

// Phase-A pass along one axis with each sub-FFT held in registers (complex64; see line_pass.cu).  Same
// operation as an AxisPass of mode 0 for sub-FFT lengths len = 16 T, T in {16, 32, 64, 128}, but never in
// place: it reads src and writes dst.  A CTA runs W = Wc x Wo lines (contiguous axis: Wc adjacent classes
// of Wo adjacent lines) or W adjacent inner positions (strided axis), T threads per line.
struct LinePass {
    const void *src;
    void *dst;
    const void *tw;    // w_{nl}^e, e in [nl] (forward roots)
    const void *tw1;   // w_len^{(j k1) mod len} at k1 T + j, k1 in [16], j in [T]
    const void *tw2;   // w_T^{(j1 k2) mod T} at j1 16 + k2, j1 in [T / 16], k2 in [16]
    const void *twp;   // w_{nl}^{(c k) mod nl} at c len + k (the axis twiddle in Put order)
    int64_t outer, inner;
    int nl, len, G, T;
    int contiguous;
    int W, lg_W, Wc, lg_Wc, Wo;
    int pad;           // shared-memory elements between the lines' regions (bank spread)
    int threads;       // T W
    int64_t ctas;
    size_t smem;       // W (len + pad) elements
};

// Phase A of two adjacent axes a, b = a + 1 in one pass (complex64; see pair_pass.cu), for equal sub-FFT
// lengths L = n_a / p_a = n_b / p_b in {8, 16} and p_a p_b >= 16.  Same result as two AxisPass of mode 0
// (axis b, then axis a), never in place.  The array is viewed as [outer][n_a][n_b][inner]; a CTA runs W
// planes (inner == 1) or W adjacent inner positions, p_a p_b L threads per item.
struct PairPass {
    const void *src;
    void *dst;
    const void *twa, *twb;  // w_{n_a}^e and w_{n_b}^e (forward roots)
    int64_t outer, inner;
    int na, nb, pa, pb, L;
    int lg_pa, lg_pb;
    int contiguous;         // inner == 1
    int W, lg_W;
    int pad;                // shared-memory elements between the items' regions (bank spread)
    int threads;            // W p_a p_b L
    int64_t ctas;
    size_t smem;            // W (p_a p_b L^2 + pad) elements
};

// Phase A of the last three axes a, b, c in one pass (complex64; see triple_pass.cu), for sub-FFT length 8 on
// each and p_b p_c = 16.  Same result as three AxisPass of mode 0 (axes c, b, a), never in place.  The array
// is viewed as [outer][n_a][n_b][n_c]; a CTA of 512 threads takes one outer position and one s_a.
struct TriplePass {
    const void *src;
    void *dst;
    const void *twa, *twb, *twc;  // w_{n_a}^e, w_{n_b}^e, w_{n_c}^e (forward roots)
    int64_t outer;
    int na, nb, nc, pa, pb, pc;
    int lg_pa, lg_pc;
    int64_t ctas;                 // outer p_a
    size_t smem;                  // 8192 elements
};

// Phase B on the d-dim groups {m + s' (n/p)} with every p_l <= 16, in one pass.
// Tile = all p values for Mt consecutive m along the last axis.
struct PhaseBFused {
    void *data;
    const void *mul;               // optional: output k is multiplied by mul[k] (natural index), else NULL
    int d;
    int64_t n[FFTU_MAX_DIMS];
    int64_t L[FFTU_MAX_DIMS];      // n_l / p_l
    int p[FFTU_MAX_DIMS];
    int64_t stride[FFTU_MAX_DIMS]; // element stride of axis l in the global array
    int P;                         // prod p_l
    int Mt;                        // consecutive m_d per tile
    int lg_p[FFTU_MAX_DIMS], lg_L[FFTU_MAX_DIMS], lg_Mt;  // log2 of the power-of-two sizes
    int64_t tiles;
    int threads;
    double scale;
    // shared slot of tile element e: e ^ (((e >> swz_src) & swz_mask) << swz_dst) (swz_mask = 0: e itself);
    // spreads the first DFT pass's runs of Mt < 16 elements over all banks
    int swz_src, swz_mask, swz_dst;
};

// Fused 3D phase A (complex64): see phase_a3.cu.
struct Phase3Info {
    int64_t unit_elems;  // elements of one residue unit (s0, s1)
    int s1_tasks, s2_tasks;
};
struct Phase3Launch {
    int which, dir, mode;  // mode 0: two kernels through a full workspace; 1: persistent L2 ring
    const void *in;
    void *out;
    void *scratch;
    const void *tw[3];
    int *status;
    unsigned *counters;
    int p0, p1, n0, n1, ring, lag;
    int grid, grid1, grid2;  // persistent ring kernel; stage-1 and stage-2 kernels
    long long spin_limit_ns;
};
// Number of compile-time phase-A configurations; phase_a3_select returns an index below it, or -1.
constexpr int kPhaseA3Configs = 5;
int phase_a3_select(int d, const int64_t *n, const int64_t *p, int is_double, Phase3Info *info);
// grids[0..2]: stage-1, stage-2 and ring kernel grid sizes (SMs x resident CTAs).
cudaError_t prepare_phase_a3(int which, int dir, int n0, int n1, int *grids, size_t *smem);
cudaError_t launch_phase_a3(const Phase3Launch &l, cudaStream_t st);

struct Plan;

// A plan seen as a list of generic passes (for batching many plans in one launch).
constexpr int kMaxBatch = 128;
struct StepView {
    bool is_axis;
    AxisPass axis;   // is_axis: a strided sub-FFT pass (mode 0 or 1)
    PhaseBFused pb;  // otherwise: the generic fused phase B
};
struct PlanView {
    int dtype, dir, device;
    bool pingpong;                  // phase A alternates with a workspace (long lines)
    int precision;                  // fftu_precision of the plan's radix-16 stages
    int layout;                     // fftu_layout
    int radix;                      // stage radix of the strided passes (8 or 16)
    std::vector<StepView> a_passes;  // phase A, generic passes (first reads in, then in place on out)
    std::vector<StepView> b_steps;   // phase B, in place on out
};
fftu_status plan_view(fftu_handle h, PlanView *v);

// Move an array between the natural row-major layout and the CYCLIC processor-major layout
// (layout.cu); to_cyclic = 1: natural -> CYCLIC, 0: CYCLIC -> natural.  src != dst.
cudaError_t launch_cyclic_permute(const void *src, void *dst, int d, const int64_t *n, const int64_t *p,
                                  int is_double, int to_cyclic, cudaStream_t st);

// Plan-time tuning (tuner.cu): fills the grid and the choices `base` leaves open (schedule AUTO,
// tile 0, radix 0); false: use the defaults.
struct TuneChoice {
    int64_t p[FFTU_MAX_DIMS];
    int schedule, tile, radix;
};
bool autotune(int d, const int64_t *n, fftu_dtype dtype, fftu_dir dir, const fftu_options &base, TuneChoice *t);
bool wisdom_lookup(int d, const int64_t *n, fftu_dtype dtype, fftu_dir dir, const fftu_options &base, TuneChoice *t);

// Set the calling thread's detail string returned by fftu_last_error().
void record_error(const char *msg);

// Kernel launchers (return cudaGetLastError() of the launch).
// Set per-device kernel attributes (dynamic shared memory); called at plan time.
cudaError_t prepare_axis_pass(int is_double, int dir);
cudaError_t prepare_phase_b_fused(int is_double, int dir);
cudaError_t prepare_phase_b3(int is_double, int dir);
// Phase B for d = 3 with p_0 = p_1 = p_2 = P in {2, 4, 8, 16}: tile length MT
// along the last axis (0 = not instantiated for this P and type).
int phase_b3_tile_mt(int p0, int p1, int p2, int is_double);  // 0: no 3D phase-B kernel for this grid
cudaError_t launch_phase_b3(const PhaseBFused &b, int is_double, int dir, cudaStream_t st);
cudaError_t launch_twiddle_table(void *dst, int64_t n, int is_double, cudaStream_t st);
// out[i] *= mul[i] for i in [n] (used when phase B cannot fuse the multiply).
cudaError_t launch_pointwise(void *out, const void *mul, int64_t n, int is_double, cudaStream_t st);
cudaError_t launch_axis_pass(const AxisPass &a, int is_double, int dir, cudaStream_t st);
cudaError_t prepare_line_pass(int dir);
cudaError_t prepare_pair_pass(int dir);
cudaError_t prepare_triple_pass(int dir);
cudaError_t launch_triple_pass(const TriplePass &a, int dir, cudaStream_t st);
cudaError_t launch_pair_pass(const PairPass &a, int dir, cudaStream_t st);
cudaError_t launch_line_pass(const LinePass &a, int dir, cudaStream_t st);
// tw1 (len entries), tw2 (len / 16 entries) and twp (nl entries) of a line pass, generated in FP64 and
// rounded.
cudaError_t launch_line_tables(void *dst, int len, int nl, cudaStream_t st);
cudaError_t launch_phase_b_fused(const PhaseBFused &b, int is_double, int dir, cudaStream_t st);
size_t axis_pass_smem_bytes(const AxisPass &a, int is_double);
size_t phase_b_fused_smem_bytes(const PhaseBFused &b, int is_double);

}  // namespace fftu
