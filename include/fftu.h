/*
 * fftu.h -- C ABI of the GB300 cyclic multidimensional FFT library (libfftu).
 *
 * The library computes the d-dimensional complex DFT
 *     Y[k] = sum_j X[j] prod_l w_{n_l}^{j_l k_l},   w_n = exp(-2 pi i / n)
 * (Koopman & Bisseling, "Minimizing communication in the multidimensional
 * FFT", Sec. 1, eq. dftd) by the parallel four-step method of Algorithm 2.3
 * (Sec. 2.2): the array is viewed as cyclically distributed over a virtual
 * processor grid p_1 x ... x p_d (Sec. 1.1, phi(s, k) = s + k p); every
 * virtual processor runs local strided sub-FFTs of shape n/p and a twiddle
 * multiply (Superstep 0), the data are redistributed once (Superstep 1, the
 * single all-to-all, realised on one GPU as the store pattern of the first
 * phase), and the remaining length-p DFTs run in place (Superstep 2).  Input
 * and output are in the same distribution, so on one GPU both are the plain
 * row-major global array (Sec. 2.2, Algorithm 2.3 input/output).
 *
 * Everything in this header is plain C: no CUDA or C++ types cross it.
 *
 * Conventions for every entry point
 *   - Arrays are row-major with the last axis contiguous (Sec. 3), n[0] is
 *     the slowest axis.  Elements are interleaved (re, im) pairs: float for
 *     FFTU_C64, double for FFTU_C128 (torch.complex64 / torch.complex128).
 *   - Device pointers are CUDA device addresses on the device that was
 *     current when the plan was made; they must be 16-byte aligned (float2 /
 *     double2 access).  The caller owns them.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Execution is stream-ordered and never synchronises the host.
 *   - Errors are returned as fftu_status; no call aborts, traps or throws.
 *     fftu_last_error() gives a one-line detail for the calling thread.
 */
#ifndef FFTU_H
#define FFTU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FFTU_MAX_DIMS 8

/* Opaque plan handle, owned by the library (fftu_destroy frees it). */
typedef struct fftu_plan_st *fftu_handle;

/* Element type: interleaved complex float (c64) or complex double (c128). */
typedef enum { FFTU_C64 = 1, FFTU_C128 = 2 } fftu_dtype;

/* Sign of the exponent.  FFTU_INVERSE runs the forward computation with every
 * root of unity replaced by its complex conjugate and divides the result by N
 * (the inverse DFT as Sec. 1.3 obtains it). */
typedef enum { FFTU_FORWARD = -1, FFTU_INVERSE = 1 } fftu_dir;

typedef enum {
    FFTU_OK = 0,
    FFTU_ERR_ARG = 1,          /* null pointer, bad d, n_l < 1, p_l < 1, misalignment, wrong device */
    FFTU_ERR_DIVISIBILITY = 2, /* p_l^2 does not divide n_l (Algorithm 2.3 input condition) */
    FFTU_ERR_UNSUPPORTED = 3,  /* valid for the method but not for this GPU build (e.g. non power of two) */
    FFTU_ERR_NOMEM = 4,        /* device allocation for tables or workspace failed */
    FFTU_ERR_CUDA = 5,         /* a CUDA runtime call or kernel launch failed */
    FFTU_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up (status word set by a kernel) */
    FFTU_ERR_INTERNAL = 7      /* a device-side consistency check failed */
} fftu_status;

/* Which part of Algorithm 2.3 fftu_exec_phase runs. */
typedef enum {
    FFTU_PHASE_A = 1,  /* Superstep 0 + Superstep 1: local sub-FFTs, twiddle, redistribution */
    FFTU_PHASE_B = 2,  /* Superstep 2: the length-p DFTs (and 1/N for the inverse), in place */
    FFTU_PHASE_ALL = 3 /* both, i.e. the whole transform */
} fftu_phase;

/* Kernel schedule.  AUTO picks the fastest schedule the plan supports;
 * GENERIC forces one strided pass per axis for each phase (any d, any
 * power-of-two shape) and is kept as a cross-check of the fused kernels;
 * GENERIC_A uses the strided passes for phase A only (phase B as AUTO). */
typedef enum {
    FFTU_SCHED_AUTO = 0,
    FFTU_SCHED_GENERIC = 1,
    FFTU_SCHED_FUSED = 2,
    FFTU_SCHED_GENERIC_A = 3
} fftu_schedule;

/* Arithmetic of the radix-16 DFT stages of the strided passes (complex64 plans only).
 * NATIVE: FP32 (complex64) or FP64 (complex128) on the CUDA cores.
 * SPLIT_BF16 / SPLIT_FP16: each radix-16 stage of 8 butterflies is a real 32 x 32 contraction on
 * the tensor cores (mma.sync m16n8k16, FP32 accumulation) with both operands split into a 16-bit
 * high and low part (three products; the low x low term is dropped); FP16 operands are scaled per
 * group of 8 butterflies by a power of two.  Twiddles, the remaining radix-2/4/8 stage and phase B
 * stay FP32.  Implies the GENERIC_A schedule.  Relative error per stage about 3 u^2 (u = 2^-8 for
 * bfloat16, 2^-11 for float16), against about 2^-24 for FP32. */
typedef enum { FFTU_PREC_NATIVE = 0, FFTU_PREC_SPLIT_BF16 = 1, FFTU_PREC_SPLIT_FP16 = 2 } fftu_precision;

/* Storage of `in` and `out`.  NATURAL: the global row-major array; the cyclic distribution of Sec. 1.1
 * is a view of it (element j belongs to processor s = j mod p at local index j div p, per axis).
 * CYCLIC: the processors' local arrays X^{(s)} (each row-major over n/p) concatenated in row-major
 * order of s, i.e. what each of the paper's processors holds.  Input and output use the same layout
 * (Algorithm 2.3 keeps the distribution).  CYCLIC costs two extra HBM round trips (three in place):
 * the transform runs on the natural view between two permutation passes.  Phase A alone then
 * writes W in CYCLIC layout (W^{(k)} concatenated) and phase B alone reads and writes it. */
typedef enum { FFTU_LAYOUT_NATURAL = 0, FFTU_LAYOUT_CYCLIC = 1 } fftu_layout;

/* Who provides the plan's device workspace (fftu_workspace_size bytes; may be 0).
 * PLAN: the plan allocates it at plan time and frees it in fftu_destroy.
 * CALLER: the plan allocates none; fftu_exec* returns FFTU_ERR_ARG until fftu_set_workspace
 * supplies one (e.g. from the caller's own allocator). */
typedef enum { FFTU_WORKSPACE_PLAN = 0, FFTU_WORKSPACE_CALLER = 1 } fftu_workspace_mode;

typedef struct {
    int schedule;        /* fftu_schedule */
    int tune;            /* with p == NULL: time candidate grids at plan time and keep the fastest */
    int precision;       /* fftu_precision */
    int layout;          /* fftu_layout */
    int workspace_mode;  /* fftu_workspace_mode */
    int tile;            /* strided passes: target elements per tile (whole lines, or the classes of a
                            long line that fit), a power of two in [1024, 8192] (complex128: [1024, 4096]);
                            0 = default (4096 / 2048) */
    int radix;           /* strided passes' stages: 8 = radix 8 after one smaller first stage (default,
                            also 0); 16 = radix-16 stages then one stage of the remaining factor */
    int reserved[1];     /* must be zero */
} fftu_options;

typedef struct {
    int d;
    int64_t n[FFTU_MAX_DIMS];
    int64_t p[FFTU_MAX_DIMS];
    int dtype;                 /* fftu_dtype */
    int dir;                   /* fftu_dir */
    int schedule;              /* schedule in use (fftu_schedule, never AUTO) */
    int launches_phase_a;      /* kernel launches one phase A takes */
    int launches_phase_b;      /* kernel launches one phase B takes */
    int64_t N;                 /* number of elements */
    int64_t alg_bytes;         /* algorithmic HBM bytes per transform: 4 * N * sizeof(element) */
    int64_t table_bytes;       /* device bytes of twiddle tables owned by the plan */
    int64_t workspace_bytes;   /* device bytes of workspace owned by the plan */
    int tuned;                 /* 1 when p (and the options left open) came from tuning or wisdom */
    int precision;             /* fftu_precision of the radix-16 stages */
    int64_t workspace_need;    /* device bytes of workspace the plan uses (owned or supplied) */
    int layout;                /* fftu_layout */
    int workspace_mode;        /* fftu_workspace_mode */
    int tile;                  /* whole-line tile target of the strided passes (elements) */
    int radix;                 /* 8 or 16: the strided passes' stage radix */
} fftu_info;

/*
 * fftu_plan -- validate the problem and build a plan.
 *   d        number of dimensions, 1 <= d <= FFTU_MAX_DIMS.
 *   n[d]     array sizes, n[0] slowest; each n_l >= 1.  This GPU build
 *            accepts powers of two only (else FFTU_ERR_UNSUPPORTED); the
 *            method itself only asks N to have many small factors (Abstract).
 *   p[d]     cyclic factors (virtual processor grid) with p_l^2 | n_l
 *            (Algorithm 2.3 input; Sec. 2.3 gives the limit p_l <= sqrt(n_l)).
 *            NULL lets the planner choose (see fftu_plan_ex).
 *   dtype    FFTU_C64 or FFTU_C128.
 *   dir      FFTU_FORWARD or FFTU_INVERSE.
 *   out      receives the handle; set to NULL on error.
 * Allocates the plan's device tables (sum_l n_l entries of w_{n_l}^e,
 * generated in FP64 on the device; cf. eq. weights) and any workspace, on the
 * current device; the tables are generated on a private stream that the call
 * waits for (work in flight on other streams is not waited for).  Not
 * stream-ordered.
 */
fftu_status fftu_plan(int d, const int64_t *n, const int64_t *p, fftu_dtype dtype, fftu_dir dir,
                      fftu_handle *out);

/* fftu_plan with options (opts may be NULL = defaults).
 * With p == NULL the plan takes the process's wisdom for the problem when there is some (from an
 * earlier tuned plan or fftu_wisdom_import), else the default grid (per axis, the largest power of two
 * up to 8 with p_l^2 | n_l).
 * With p == NULL and opts->tune != 0 the planner measures, on scratch buffers it allocates for the
 * duration (2 N elements), one coordinate at a time: every candidate grid p_l = min(q, pmax_l),
 * q = 1, 2, 4, ... (pmax_l: the largest power of two with p_l^2 | n_l), each also with the last axis at
 * q / 2; then, for the fastest grid, the schedules (AUTO, GENERIC_A, GENERIC) unless opts->schedule
 * fixes one; then the strided passes' tile target (2048, 4096, 8192 for complex64; 1024, 2048, 4096 for
 * complex128) and radix (8, 16), unless fixed.  The choice is remembered per (shape, dtype, direction,
 * requested schedule, precision, GPU) in the process's wisdom table (fftu_wisdom_*).  If the scratch
 * cannot be allocated, the defaults are used. */
fftu_status fftu_plan_ex(int d, const int64_t *n, const int64_t *p, fftu_dtype dtype, fftu_dir dir,
                         const fftu_options *opts, fftu_handle *out);

/*
 * fftu_exec -- run the whole transform (Algorithm 2.3) on `stream`.
 *   in   device array of N elements (read only when in != out).
 *   out  device array of N elements, receives V = DFT(X) in the plan's layout (NATURAL: row-major).
 *   in == out is allowed (in-place transform).  Other partial overlaps are
 *   not allowed.  A plan may run on one stream at a time.
 */
fftu_status fftu_exec(fftu_handle plan, const void *in, void *out, void *stream);

/*
 * fftu_exec_phase -- run one part of Algorithm 2.3 (for staged checks).
 *   FFTU_PHASE_A: in -> out.  out receives the redistributed data W in the
 *                 global view: Z^{(s)}[m] (Superstep 0 output of virtual
 *                 processor s at local index m) is stored at global index
 *                 m + s (n/p), elementwise per axis (Superstep 1 Put).
 *   FFTU_PHASE_B: in place on out (in must be NULL or equal to out): for every
 *                 m in [n/p], the p values at m + s'(n/p) are replaced by
 *                 their p_1 x ... x p_d DFT (Superstep 2), scaled by 1/N for
 *                 the inverse.
 *   FFTU_PHASE_ALL: same as fftu_exec.
 */
fftu_status fftu_exec_phase(fftu_handle plan, fftu_phase phase, const void *in, void *out,
                            void *stream);

/*
 * fftu_exec_pointwise -- out = inverse( forward(in) .* mul ), the transform pair with an elementwise
 * product in between and no data reordering (Sec. 1.3: input and output share the distribution, so the
 * inverse can follow the forward transform directly, with a local elementwise operation interspersed;
 * Sec. 6: the split-step propagation of the time-dependent Schroedinger equation).
 *   fwd, inv  plans of the same shape, cyclic grid, dtype and device; FFTU_FORWARD and FFTU_INVERSE.
 *   in        device array of N elements (not modified unless it equals tmp).
 *   mul       device array of N elements, the multiplier in the frequency domain, natural order.
 *   tmp       device array of N elements for the spectrum; may equal in; must differ from out and mul.
 *   out       device array of N elements; may equal in.
 * When the forward plan's phase B is the fused 3D kernel, the product happens in its store (one extra
 * read of mul, no extra pass); otherwise one elementwise pass follows phase B.  Stream-ordered.
 */
fftu_status fftu_exec_pointwise(fftu_handle fwd, fftu_handle inv, const void *in, const void *mul, void *tmp,
                                void *out, void *stream);

/* Free the plan's device memory and the handle.  Synchronises the device
 * with the plan's last use.  NULL is accepted. */
fftu_status fftu_destroy(fftu_handle plan);

/* Describe a plan (sizes, schedule, launches, byte counts). */
fftu_status fftu_plan_info(fftu_handle plan, fftu_info *info);

/* Read and clear the plan's device status word (bounded waits and device
 * checks write it).  Synchronises with the plan's last use.  Returns FFTU_OK,
 * FFTU_ERR_TIMEOUT or FFTU_ERR_INTERNAL. */
fftu_status fftu_check_device_status(fftu_handle plan);

/*
 * fftu_exec_noalloc -- the whole transform with no device allocation at all.
 * The paper has no counterpart: this serves callers that cannot call
 * cudaMalloc where they run the FFT (code under CUDA graph capture, plugins
 * whose host owns all device memory, real-time loops that must not enter the
 * allocator).  No plan is needed; the arguments mean what they mean for
 * fftu_plan and fftu_exec, with these limits:
 *   - d = 3, FFTU_C64, p_0 = p_1 = p_2, and a shape with a fused kernel whose
 *     residue unit (n_0 n_1 n_2 / (p_0 p_1) elements) fits a 16 MiB slot.
 *     With the fused kernels this build has, that is 512^3 with p = 8^3 only;
 *     every other problem returns FFTU_ERR_UNSUPPORTED;
 *   - in != out (FFTU_ERR_ARG otherwise); both 16-byte aligned device pointers.
 * Scratch, counters, twiddle tables and a status word live in static device
 * arrays (about 32 MiB, held by every GPU that loads this part of the library
 * until the process exits).  Set-up: the first call on a device (with that
 * device current) looks up their addresses, and the first call with a given
 * axis length writes that length's twiddle table into a slot of its own (once
 * per device, then never rewritten) and waits for it; make those first calls
 * before any stream capture -- made under capture they return FFTU_ERR_ARG.
 * All calls share the arrays: calls that overlap on the GPU race and give
 * wrong results, so order them on one stream.  The counters are cleared on the
 * stream by each call.  A bounded device wait that expires leaves that call's
 * output invalid and sets the shared status word; read it with
 * fftu_noalloc_check_status.  Calls no cudaMalloc, cudaFree or allocating
 * library routine.
 */
fftu_status fftu_exec_noalloc(int d, const int64_t *n, const int64_t *p, fftu_dtype dtype, fftu_dir dir,
                              const void *in, void *out, void *stream);

/* fftu_noalloc_check_status -- read and clear the status word that fftu_exec_noalloc's kernels share
 * on the current device.  The read is ordered after the work queued on `stream` and the call waits
 * for it (not allowed while `stream` is capturing: FFTU_ERR_ARG).  Returns FFTU_OK if no device wait
 * has expired since the last check, FFTU_ERR_TIMEOUT if one has (the output of the call it belonged to
 * is invalid), FFTU_ERR_INTERNAL for any other recorded code.  No allocation.  The paper has no
 * counterpart (failure detection of the allocation-free entry point). */
fftu_status fftu_noalloc_check_status(void *stream);

/* fftu_noalloc_selftest_timeout -- failure-detection self-test of that status word: runs the library's
 * bounded device wait, on `stream`, on a static word nothing advances, with a budget of limit_s seconds
 * (0.001..2), so that the wait expires and records FFTU_ERR_TIMEOUT in the word
 * fftu_noalloc_check_status reads.  Waits for the stream.  Nothing traps; the context stays usable.
 * Returns FFTU_ERR_ARG for a budget out of range or a capturing stream. */
fftu_status fftu_noalloc_selftest_timeout(double limit_s, void *stream);

/*
 * Batches: many transforms of different shapes in one persistent kernel launch.
 * fftu_batch_create -- build a batch from `count` (1..128) existing plans with the same dtype,
 *   direction and device.  Every pass of every plan becomes a job (phase A's strided sub-FFT passes,
 *   then phase B, Algorithm 2.3); a persistent kernel takes their tiles in pass-major order and a tile
 *   of pass k waits (bounded) for pass k - 1 of the same transform.  Plans whose phase A alternates with
 *   a workspace (a line longer than a tile) are not batched (FFTU_ERR_UNSUPPORTED).  The batch reads the
 *   plans' twiddle tables: destroy the batch before its plans.  It owns a small device job table and
 *   counters.
 * fftu_batch_exec -- run the batch on `stream`: ins[i] -> outs[i] (device arrays of plan i's size,
 *   16-byte aligned; outs[i] may equal ins[i]; arrays of different transforms must not overlap).  No host
 *   synchronisation: the counters are cleared on the stream, so the call can be captured into a CUDA graph.
 *   One batch may run on one stream at a time.
 * fftu_batch_check_status -- read and clear the batch's device status word (bounded waits); synchronises.
 * fftu_batch_destroy -- synchronise the device and free the batch (NULL accepted).
 */
typedef struct fftu_batch_st *fftu_batch;
fftu_status fftu_batch_create(int count, const fftu_handle *plans, fftu_batch *out);
fftu_status fftu_batch_exec(fftu_batch batch, const void *const *ins, void *const *outs, void *stream);
fftu_status fftu_batch_check_status(fftu_batch batch);
fftu_status fftu_batch_destroy(fftu_batch batch);

/* Wisdom: the tuned choices as text lines "fftu-wisdom-v2 <key> <p_1,...,p_d> <schedule> <tile> <radix>"
 * with key "d:n_1,...,n_d:dtype:dir:schedule:precision:gpu_name" (lines "fftu-wisdom-v1 <key>
 * <p_1,...,p_d>", whose key has no precision field, are read as grids with the other choices left to
 * the defaults).  Export writes the process's table, import merges a file into it, forget clears it.
 * Import skips every line that no plan would accept (a grid with p_l^2 not dividing n_l, a shape that
 * is not a power of two, an unknown schedule, tile or radix, a malformed key) and lines of other
 * tools; FFTU_ERR_ARG only when the file cannot be opened. */
fftu_status fftu_wisdom_export(const char *path);
fftu_status fftu_wisdom_import(const char *path);
fftu_status fftu_wisdom_forget(void);

/* Bytes of device workspace the plan needs (0 for plans that need none).  Synchronous, host only. */
fftu_status fftu_workspace_size(fftu_handle plan, size_t *bytes);

/* Make the plan use `workspace` (device memory of at least fftu_workspace_size bytes, 256-byte
 * aligned, owned by the caller and kept alive until every exec that used it has completed) instead
 * of its own; a workspace the plan allocated itself is freed first (after a device synchronisation).
 * workspace == NULL detaches it (execs then fail with FFTU_ERR_ARG until another is set).  Execs of
 * one plan that overlap on the GPU must use different workspaces: give each stream its own plan, or
 * set a stream's workspace before its exec and order them. */
fftu_status fftu_set_workspace(fftu_handle plan, void *workspace, size_t bytes);

/* Failure-detection self-test (no counterpart in the paper): runs the bounded device wait the batch
 * kernel uses on a device word that nothing ever advances, with a budget of limit_s seconds
 * (0.001..2).  The wait must give up and report FFTU_ERR_TIMEOUT through its status word, as any
 * expired wait in this library does instead of trapping; *waited_s (may be NULL) receives the time
 * it waited.  Returns FFTU_OK when that happened, FFTU_ERR_INTERNAL if the status was not set.
 * Synchronises its own stream; the context stays usable. */
fftu_status fftu_selftest_bounded_wait(double limit_s, double *waited_s);

/* Measurement helper (not part of the method): the sustained FP64 fused multiply-add rate of the
 * current device in GFLOP/s (2 flops per FMA), from a kernel that keeps every SM's FP64 pipe busy with
 * independent FMA chains, timed with CUDA events; best of `reps` (1..100) timed launches after one
 * warm-up.  complex128 transforms are bound by this rate rather than by HBM bandwidth on GB300, so
 * their roofline is stated against it.  Allocates and frees 8 bytes of device memory and a stream;
 * synchronises that stream.  FFTU_ERR_ARG for a NULL gflops or reps out of range. */
fftu_status fftu_measure_fp64_rate(int reps, double *gflops);

/* Static string for a status code. */
const char *fftu_status_string(fftu_status s);

/* One-line detail about the last error on the calling thread ("" if none). */
const char *fftu_last_error(void);

/* Library version, e.g. "fftu 0.1.0 sm_103a". */
const char *fftu_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FFTU_H */
