// Phase-A pass along one axis with each sub-FFT held in registers (complex64).
//
// The operation is mode 0 of the strided pass (axis_pass.cu): Superstep 0 of Alg. 2.3 on one axis, i.e. a
// DFT of length len = n_l / p_l on every residue class s of every line, the axis' twiddle w_{n_l}^{k s} of
// Sec. 2.2, and the Put position s len + k of Superstep 1.  This kernel serves len = 16 T with T in
// {16, 32, 64, 128} (len 256 ... 2048).  It applies the radix split of Sec. 2.1.1 (eq. radix) twice,
//   len = 16 x T,  T = 16 x R3  (R3 = T / 16),
// with input index m = j + T r (j in [T], r in [16]) and output index k = k1 + 16 (k2 + 16 k3):
//   stage 1: thread j of the line: F_16 over r, times w_len^{j k1};
//   stage 2: thread (k1, j1) with j = j1 + R3 j2: F_16 over j2, times w_T^{j1 k2};
//   stage 3: F_R3 over j1 for each (k1, k2); then w_{n_l}^{k s} and the store.
// Each thread holds 16 values per stage; the input goes from HBM straight into registers and the output
// from registers straight to its Put position, with two shared-memory exchanges in between.  The strided
// pass instead keeps the whole tile in shared memory through every stage.
//
// In stage 1 thread t takes line t % W, so that the lanes of a warp load adjacent lines, whose elements are
// adjacent in memory (adjacent classes, or adjacent inner positions).  On a strided axis it keeps that line
// (adjacent inner positions are adjacent in the output too); on the contiguous axis, where adjacent classes
// land len apart in the output, stages 2 and 3 take line t / T instead, so that a warp stores runs of 16
// consecutive outputs of one class.
// Shared layout of a line's region (len elements, regions `pad` = 16 / W elements apart):
//   exchange 1: (k1, j) at k1 T + (j ^ k1);   exchange 2: (k1, j1, k2) at (j1 16 + k2) 16 + k1.
// A CPU count of the wavefronts of every access (tests/test_line_pass_maps.py) finds 2 per 32 lanes, the
// minimum for 8-byte elements, and 1 per half-warp.
#include <cuda_runtime.h>

#include "fft_device.cuh"
#include "fftu_internal.h"

namespace fftu {
namespace {

// At most 64 registers: two CTAs of 512 threads (or four of 256) per SM; 2048-point lines take eight lines
// per CTA, 1024 threads (one CTA per SM; measured faster than four lines per CTA).
constexpr int kLineMaxThreads = 1024;
template <int T> constexpr int line_max_threads() { return T == 128 ? 1024 : 512; }

template <int T, int DIR, bool CONTIG>
__global__ void __launch_bounds__(line_max_threads<T>(), line_max_threads<T>() == 1024 ? 1 : 2)
    line_pass_kernel(const __grid_constant__ LinePass a) {
    constexpr int LEN = 16 * T;
    constexpr int R3 = T / 16;
    extern __shared__ __align__(16) float2 line_sm[];
    const int t = threadIdx.x;
    const int w = t & (a.W - 1);  // line of this thread within the CTA
    const int q = t >> a.lg_W;    // role within the line, q in [T]
    const int w2 = CONTIG ? t / T : w;  // line of this thread in stages 2 and 3
    const int q2 = CONTIG ? t % T : q;
    const int64_t b = blockIdx.x;
    int64_t in_off, out_off;
    int c;  // residue class of the stage-2/3 line
    if constexpr (CONTIG) {
        const int lg_cgroups = __ffs(a.G) - 1 - a.lg_Wc;
        const int64_t cg = b & ((1ll << lg_cgroups) - 1), og = b >> lg_cgroups;
        const int64_t o = og * a.Wo + (w >> a.lg_Wc);
        in_off = o * a.nl + (cg << a.lg_Wc) + (w & (a.Wc - 1));
        const int64_t o2 = og * a.Wo + (w2 >> a.lg_Wc);
        c = (int)((cg << a.lg_Wc) + (w2 & (a.Wc - 1)));
        out_off = o2 * a.nl + (int64_t)c * LEN;
    } else {
        const int64_t vgroups = a.inner >> a.lg_W;
        const int64_t vg = b % vgroups, rest = b / vgroups;
        c = (int)(rest % a.G);
        const int64_t o = rest / a.G;
        const int64_t v = (vg << a.lg_W) + w;
        in_off = o * a.nl * a.inner + (int64_t)c * a.inner + v;
        out_off = o * a.nl * a.inner + (int64_t)c * LEN * a.inner + v;
    }
    const int64_t s_in = CONTIG ? (int64_t)a.G : (int64_t)a.G * a.inner;  // element stride of m
    float2 *reg = line_sm + w * (LEN + a.pad);
    const float2 *__restrict__ tw1 = static_cast<const float2 *>(a.tw1);
    float2 v[16];

    // stage 1: thread j loads x[j + T r], F_16 over r, twiddle w_len^{j k1}
    {
        const int j = q;
        const float2 *__restrict__ src = static_cast<const float2 *>(a.src) + in_off + j * s_in;
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = src[(int64_t)r * T * s_in];
        dft16<DIR>(v);
#pragma unroll
        for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], dirw<DIR>(tw1[k1 * T + j]));
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) reg[k1 * T + (j ^ k1)] = v[k1];
    }
    __syncthreads();

    // stage 2: thread (k1, j1): F_16 over j2 of the values j = j1 + R3 j2
    reg = line_sm + w2 * (LEN + a.pad);
    const int k1 = q2 & 15, j1 = q2 >> 4;
#pragma unroll
    for (int j2 = 0; j2 < 16; ++j2) {
        const int j = j1 + R3 * j2;
        v[j2] = reg[k1 * T + (j ^ k1)];
    }
    dft16<DIR>(v);
    // w_{nl}^{c k} of this line in Put order: entry c len + k (consecutive k of a class are adjacent, so a
    // warp's twiddle loads are runs like its stores).  For T = 16 the plain table w_nl^e at e = c k is kept:
    // it needs fewer registers there (four CTAs per SM; measured faster on 1024^3 at p = 4^3).
    const float2 *__restrict__ twp = static_cast<const float2 *>(T == 16 ? a.tw : a.twp) + (T == 16 ? 0 : c * LEN + k1);
    float2 *__restrict__ dst = static_cast<float2 *>(a.dst) + out_off;
    const int64_t s_out = CONTIG ? 1 : a.inner;  // element stride of the output index k
    if constexpr (R3 == 1) {
        // k = k1 + 16 k2: the axis twiddle w_{nl}^{k c} and the Put store
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
            const int k = k1 + 16 * k2;
            dst[(int64_t)k * s_out] = cmul(v[k2], dirw<DIR>(twp[T == 16 ? c * k : 16 * k2]));
        }
    } else {
        const float2 *__restrict__ tw2 = static_cast<const float2 *>(a.tw2);
#pragma unroll
        for (int k2 = 1; k2 < 16; ++k2) v[k2] = cmul(v[k2], dirw<DIR>(tw2[j1 * 16 + k2]));
        __syncthreads();  // every stage-2 read of the region is done before it is overwritten
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) reg[((j1 * 16 + k2) << 4) + k1] = v[k2];
        __syncthreads();

        // stage 3: thread (k1, h = j1) takes k2 = h + R3 i, i in [16 / R3]: F_R3 over j1
        const int h = j1;
#pragma unroll
        for (int i = 0; i < 16 / R3; ++i) {
            const int k2 = h + R3 * i;
            float2 y[R3];
#pragma unroll
            for (int jj = 0; jj < R3; ++jj) y[jj] = reg[((jj * 16 + k2) << 4) + k1];
            dft_small<R3, DIR>(y);
#pragma unroll
            for (int k3 = 0; k3 < R3; ++k3) {
                const int k = k1 + 16 * k2 + 256 * k3;
                dst[(int64_t)k * s_out] = cmul(y[k3], dirw<DIR>(twp[16 * k2 + 256 * k3]));
            }
        }
    }
}

// tw1[k1 T + j] = w_len^{(j k1) mod len}, then tw2[j1 16 + k2] = w_T^{(j1 k2) mod T}, then twp[c len + k] =
// w_nl^{(c k) mod nl}: forward roots in FP64, rounded to FP32 (the inverse conjugates them in the kernel).
__global__ void line_table_kernel(float2 *dst, int len, int nl) {
    const int T = len / 16;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < len + T + nl; e += gridDim.x * blockDim.x) {
        long long num, den;
        if (e >= len + T) {  // Put order: entry c len + k holds w_nl^{c k}
            const int f = e - len - T;
            num = ((long long)(f / len) * (f % len)) % nl;
            den = nl;
        } else if (e < len) {
            const int k1 = e / T, j = e % T;
            num = ((long long)j * k1) % len;
            den = len;
        } else {
            const int j1 = (e - len) / 16, k2 = (e - len) % 16;
            num = ((long long)j1 * k2) % T;
            den = T;
        }
        double s, co;
        sincospi(-2.0 * (double)num / (double)den, &s, &co);
        dst[e] = make_float2((float)co, (float)s);
    }
}

template <int T, int DIR>
cudaError_t launch_t(const LinePass &a, cudaStream_t st) {
    const dim3 grid((unsigned)a.ctas);
    if (a.contiguous)
        line_pass_kernel<T, DIR, true><<<grid, a.threads, a.smem, st>>>(a);
    else
        line_pass_kernel<T, DIR, false><<<grid, a.threads, a.smem, st>>>(a);
    return cudaGetLastError();
}

template <int DIR>
cudaError_t launch_dir(const LinePass &a, cudaStream_t st) {
    switch (a.T) {
        case 16: return launch_t<16, DIR>(a, st);
        case 32: return launch_t<32, DIR>(a, st);
        case 64: return launch_t<64, DIR>(a, st);
        case 128: return launch_t<128, DIR>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int T, int DIR>
cudaError_t prepare_t() {
    cudaError_t e = cudaFuncSetAttribute(line_pass_kernel<T, DIR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kMaxDynSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(line_pass_kernel<T, DIR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kMaxDynSmem);
    return e;
}

template <int DIR>
cudaError_t prepare_dir() {
    cudaError_t e = prepare_t<16, DIR>();
    if (e == cudaSuccess) e = prepare_t<32, DIR>();
    if (e == cudaSuccess) e = prepare_t<64, DIR>();
    if (e == cudaSuccess) e = prepare_t<128, DIR>();
    return e;
}

}  // namespace

cudaError_t prepare_line_pass(int dir) { return dir < 0 ? prepare_dir<-1>() : prepare_dir<1>(); }

cudaError_t launch_line_pass(const LinePass &a, int dir, cudaStream_t st) {
    if (a.ctas < 1 || a.threads < 32 || a.threads > kLineMaxThreads || a.threads != a.T * a.W ||
        (a.T != 128 && a.threads > 512) ||
        a.ctas > 0x7fffffffll || a.smem > (size_t)kMaxDynSmem)
        return cudaErrorInvalidValue;
    return dir < 0 ? launch_dir<-1>(a, st) : launch_dir<1>(a, st);
}

cudaError_t launch_line_tables(void *dst, int len, int nl, cudaStream_t st) {
    const int n = len + len / 16 + nl;
    line_table_kernel<<<(n + 255) / 256, 256, 0, st>>>(static_cast<float2 *>(dst), len, nl);
    return cudaGetLastError();
}

}  // namespace fftu
