// Generic strided sub-FFT pass along one axis, and the FP64 twiddle tables.
//
// One launch applies, to every line of one axis, a batch of independent
// length-len DFTs on the strided classes of that line (see AxisPass in
// fftu_internal.h).  Phase A of Algorithm 2.3 (Sec. 2.2) is one such pass per
// axis in mode 0 (local sub-FFT F_{n_l/p_l} on the residue class s_l, the
// twiddle w_{n_l}^{m_l s_l}, and the Put position m_l + s_l n_l/p_l of
// Superstep 1); phase B is one pass per axis in mode 1 (F_{p_l} on the class
// {m_l + s' n_l/p_l}, Superstep 2).  Applying the d-dim operators axis by axis
// is exact because they are tensor products (Sec. 2.2, Y = (F_{n_1} x ... x F_{n_d}) X).
//
// Inside a tile the DFTs run as a self-sorting (Stockham) mixed-radix
// sequence of radix-2/4/8/16 stages in shared memory: every thread reads its
// butterflies' inputs into registers, the block synchronises, then writes the
// outputs to their sorted positions.  Stage (radix R, span Ns) maps butterfly
// b of a column to inputs b + r len/R, twiddles w_{Ns R}^{r (b mod Ns)}, and
// outputs (b div Ns) Ns R + (b mod Ns) + r Ns.
#include <cuda_runtime.h>

#include "fft_device.cuh"
#include "fftu_internal.h"
#include "generic_tiles.cuh"

namespace fftu {

namespace {

constexpr int kAxisThreads = 512;

// R0: radix of the first stage (1 = none); every later stage is radix 8.  With TCK (split-precision
// tensor-core radix-16 stages, complex64 only), R0 is the radix of the last, CUDA-core stage.
template <typename C, int DIR, int R0, int TCK = 0>
__global__ void __launch_bounds__(kAxisThreads) axis_pass_kernel(const __grid_constant__ AxisPass a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw);
    const C *__restrict__ src = static_cast<const C *>(a.src);
    C *__restrict__ dst = static_cast<C *>(a.dst);
    const C *__restrict__ tw = static_cast<const C *>(a.tw);
    if constexpr (TCK == 1 || TCK == 2) {
        // tensor-core stages: operand tiles after the tile (128-byte aligned), TMEM for the block
        const uint32_t base = (uint32_t)__cvta_generic_to_shared(smem_raw + (size_t)a.tile * sizeof(C));
        unsigned char *raw = smem_raw + (size_t)a.tile * sizeof(C) + ((128 - (base & 127)) & 127);
        UmmaCtx u = umma_setup<DIR, TCK>(raw, reinterpret_cast<const float2 *>(tw), a.nl, a.status);
        for (int64_t t = blockIdx.x; t < a.tiles; t += gridDim.x) axis_tile<C, DIR, R0, TCK>(a, t, sm, src, dst, tw, &u);
        umma_teardown(u);
    } else {
        for (int64_t t = blockIdx.x; t < a.tiles; t += gridDim.x) axis_tile<C, DIR, R0, TCK>(a, t, sm, src, dst, tw);
    }
}

// w_n^e = exp(-2 pi i e / n) for e in [n], evaluated in FP64 by sincospi on the
// exactly reduced exponent, then rounded once to the table's precision.
template <typename C>
__global__ void twiddle_table_kernel(C *dst, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)e / (double)n, &s, &c);
        C w;
        w.x = (typename real_of<C>::type)c;
        w.y = (typename real_of<C>::type)s;
        dst[e] = w;
    }
}

template <typename C>
__global__ void pointwise_kernel(C *out, const C *mul, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = cmul(out[i], mul[i]);
}

template <typename C, int DIR, int TCK>
void launch_axis_tc(const AxisPass &a, unsigned grid, size_t smem, cudaStream_t st) {
    const int last = a.nstages > 0 ? a.radix[a.nstages - 1] : 1;
    switch (last) {
        case 2: axis_pass_kernel<C, DIR, 2, TCK><<<grid, a.threads, smem, st>>>(a); break;
        case 4: axis_pass_kernel<C, DIR, 4, TCK><<<grid, a.threads, smem, st>>>(a); break;
        case 8: axis_pass_kernel<C, DIR, 8, TCK><<<grid, a.threads, smem, st>>>(a); break;
        default: axis_pass_kernel<C, DIR, 1, TCK><<<grid, a.threads, smem, st>>>(a); break;
    }
}

template <typename C, int DIR>
cudaError_t launch_axis_t(const AxisPass &a, cudaStream_t st) {
    size_t smem = axis_pass_smem_bytes(a, sizeof(C) == 16);
    int64_t grid = a.tiles < (int64_t)1 << 30 ? a.tiles : (int64_t)1 << 30;
    if (a.tc == 3) {
        launch_axis_tc<C, DIR, 3>(a, (unsigned)grid, smem, st);
        return cudaGetLastError();
    }
    if constexpr (sizeof(C) == 8) {
        if (a.tc == 1) {
            launch_axis_tc<C, DIR, 1>(a, (unsigned)grid, smem, st);
            return cudaGetLastError();
        }
        if (a.tc == 2) {
            launch_axis_tc<C, DIR, 2>(a, (unsigned)grid, smem, st);
            return cudaGetLastError();
        }
    }
    const int r0 = a.nstages > 0 && a.radix[0] != 8 ? a.radix[0] : 1;
    switch (r0) {
        case 2: axis_pass_kernel<C, DIR, 2><<<(unsigned)grid, a.threads, smem, st>>>(a); break;
        case 4: axis_pass_kernel<C, DIR, 4><<<(unsigned)grid, a.threads, smem, st>>>(a); break;
        case 16: axis_pass_kernel<C, DIR, 16><<<(unsigned)grid, a.threads, smem, st>>>(a); break;
        default: axis_pass_kernel<C, DIR, 1><<<(unsigned)grid, a.threads, smem, st>>>(a); break;
    }
    return cudaGetLastError();
}

template <typename C, int DIR, int R0, int TCK = 0>
cudaError_t prepare_axis_r() {
    return cudaFuncSetAttribute(axis_pass_kernel<C, DIR, R0, TCK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kMaxDynSmem);
}

template <typename C, int DIR>
cudaError_t prepare_axis_t() {
    cudaError_t e = prepare_axis_r<C, DIR, 1>();
    if (e == cudaSuccess) e = prepare_axis_r<C, DIR, 2>();
    if (e == cudaSuccess) e = prepare_axis_r<C, DIR, 4>();
    if (e == cudaSuccess) e = prepare_axis_r<C, DIR, 16>();
    if (e == cudaSuccess) e = prepare_axis_r<C, DIR, 1, 3>();
    if (e == cudaSuccess) e = prepare_axis_r<C, DIR, 2, 3>();
    if (e == cudaSuccess) e = prepare_axis_r<C, DIR, 4, 3>();
    if (e == cudaSuccess) e = prepare_axis_r<C, DIR, 8, 3>();
    if constexpr (sizeof(C) == 8) {
        if (e == cudaSuccess) e = prepare_axis_r<C, DIR, 1, 1>();
        if (e == cudaSuccess) e = prepare_axis_r<C, DIR, 2, 1>();
        if (e == cudaSuccess) e = prepare_axis_r<C, DIR, 4, 1>();
        if (e == cudaSuccess) e = prepare_axis_r<C, DIR, 8, 1>();
        if (e == cudaSuccess) e = prepare_axis_r<C, DIR, 1, 2>();
        if (e == cudaSuccess) e = prepare_axis_r<C, DIR, 2, 2>();
        if (e == cudaSuccess) e = prepare_axis_r<C, DIR, 4, 2>();
        if (e == cudaSuccess) e = prepare_axis_r<C, DIR, 8, 2>();
    }
    return e;
}

}  // namespace

size_t axis_pass_smem_bytes(const AxisPass &a, int is_double) {
    const size_t tile = (size_t)a.tile * (is_double ? sizeof(double2) : sizeof(float2));
    if (!is_double && (a.tc == 1 || a.tc == 2)) return (tile + 127) / 128 * 128 + umma_smem_bytes(a.threads);
    return tile;
}

cudaError_t launch_axis_pass(const AxisPass &a, int is_double, int dir, cudaStream_t st) {
    if (is_double) return dir < 0 ? launch_axis_t<double2, -1>(a, st) : launch_axis_t<double2, 1>(a, st);
    return dir < 0 ? launch_axis_t<float2, -1>(a, st) : launch_axis_t<float2, 1>(a, st);
}

cudaError_t prepare_axis_pass(int is_double, int dir) {
    if (is_double) return dir < 0 ? prepare_axis_t<double2, -1>() : prepare_axis_t<double2, 1>();
    return dir < 0 ? prepare_axis_t<float2, -1>() : prepare_axis_t<float2, 1>();
}

cudaError_t launch_pointwise(void *out, const void *mul, int64_t n, int is_double, cudaStream_t st) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    if (is_double)
        pointwise_kernel<double2><<<(unsigned)blocks, 256, 0, st>>>(static_cast<double2 *>(out),
                                                                     static_cast<const double2 *>(mul), n);
    else
        pointwise_kernel<float2><<<(unsigned)blocks, 256, 0, st>>>(static_cast<float2 *>(out),
                                                                    static_cast<const float2 *>(mul), n);
    return cudaGetLastError();
}

cudaError_t launch_twiddle_table(void *dst, int64_t n, int is_double, cudaStream_t st) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    if (is_double)
        twiddle_table_kernel<double2><<<(unsigned)blocks, 256, 0, st>>>(static_cast<double2 *>(dst), n);
    else
        twiddle_table_kernel<float2><<<(unsigned)blocks, 256, 0, st>>>(static_cast<float2 *>(dst), n);
    return cudaGetLastError();
}

}  // namespace fftu
