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

namespace fftu {

namespace {

// complex values a thread holds per stage: 16 (c64) or 8 (c128)
template <typename C> __host__ __device__ constexpr int ept() { return sizeof(C) == 8 ? kEptMax : kEptMax / 2; }
constexpr int kAxisThreads = 512;

template <typename C, int DIR, int R>
__device__ __forceinline__ void stockham_stage(C *sm, const C *__restrict__ tw, const AxisPass &a, int Ns,
                                               int tid, int nthreads) {
    constexpr int B = ept<C>() / R > 0 ? ept<C>() / R : 1;  // butterflies per thread per stage
    const int lg_cols = a.lg_Gt + a.lg_V;
    const int cols = 1 << lg_cols;
    const int per_col = a.len / R;
    const int total = cols * per_col;
    const int twstep = a.nl / (Ns * R);
    const int lg_ns = 31 - __clz(Ns);
    C v[B][R];
#pragma unroll
    for (int q = 0; q < B; ++q) {
        const int w = tid + q * nthreads;
        if (w < total) {
            const int col = w & (cols - 1), b = w >> lg_cols;
            int base, js;
            if (a.contiguous) {
                base = ((col >> a.lg_Gt) << a.lg_nlt) + (col & (a.Gt - 1));
                js = a.Gt;
            } else {
                base = col;
                js = cols;
            }
            const int k = b & (Ns - 1);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                C x = sm[base + (b + r * per_col) * js];
                if (r > 0 && Ns > 1) x = cmul(x, dirw<DIR>(tw[r * k * twstep]));
                v[q][r] = x;
            }
            dft_small<R, DIR>(v[q]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < B; ++q) {
        const int w = tid + q * nthreads;
        if (w < total) {
            const int col = w & (cols - 1), b = w >> lg_cols;
            int base, js;
            if (a.contiguous) {
                base = ((col >> a.lg_Gt) << a.lg_nlt) + (col & (a.Gt - 1));
                js = a.Gt;
            } else {
                base = col;
                js = cols;
            }
            const int k = b & (Ns - 1);
            const int o = ((b >> lg_ns) << lg_ns) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) sm[base + (o + r * Ns) * js] = v[q][r];
        }
    }
    __syncthreads();
}

// R0: radix of the first stage (1 = none); every later stage is radix 8.
template <typename C, int DIR, int R0>
__global__ void __launch_bounds__(kAxisThreads) axis_pass_kernel(const __grid_constant__ AxisPass a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw);
    const C *__restrict__ src = static_cast<const C *>(a.src);
    C *__restrict__ dst = static_cast<C *>(a.dst);
    const C *__restrict__ tw = static_cast<const C *>(a.tw);
    using Rl = typename real_of<C>::type;
    const int tid = threadIdx.x, nt = blockDim.x;

    const int chunks = 1 << a.lg_chunks;  // class chunks per line
    for (int64_t t = blockIdx.x; t < a.tiles; t += gridDim.x) {
        const int cc = (int)(t & (chunks - 1));
        const int64_t tt = t >> a.lg_chunks;
        const int c0 = cc << a.lg_Gt;
        int64_t gbase;  // element offset of (first line or vector, line position 0)
        if (a.contiguous) {
            gbase = (tt << a.lg_V) * a.nl;
        } else {
            const int64_t tpo_mask = ((int64_t)1 << a.lg_tpo) - 1;
            gbase = (tt >> a.lg_tpo) * (int64_t)a.nl * a.inner + ((tt & tpo_mask) << a.lg_V);
        }
        // load: shared index e is the natural order of the tile (tile line position lp, vector v);
        // tile position lp = c_local + j Gt holds line position c0 + c_local + j G
        for (int e = tid; e < a.tile; e += nt) {
            int lp, v;
            if (a.contiguous) {
                v = e >> a.lg_nlt;
                lp = e & (a.nlt - 1);
            } else {
                lp = e >> a.lg_V;
                v = e & (a.V - 1);
            }
            const int64_t gp = c0 + (lp & (a.Gt - 1)) + ((int64_t)(lp >> a.lg_Gt) << a.lg_G);
            const int64_t g = a.contiguous ? gbase + (int64_t)v * a.nl + gp : gbase + gp * a.inner + v;
            sm[e] = src[g];
        }
        __syncthreads();

        int Ns = 1;
        if constexpr (R0 > 1) {
            stockham_stage<C, DIR, R0>(sm, tw, a, Ns, tid, nt);
            Ns = R0;
        }
        for (; Ns < a.len; Ns *= 8) stockham_stage<C, DIR, 8>(sm, tw, a, Ns, tid, nt);

        // store with the output permutation, twiddle and scale
        const Rl scale = (Rl)a.scale;
        for (int e = tid; e < a.tile; e += nt) {
            int lpo, v;  // tile output position and vector
            if (a.contiguous) {
                v = e >> a.lg_nlt;
                lpo = e & (a.nlt - 1);
            } else {
                lpo = e >> a.lg_V;
                v = e & (a.V - 1);
            }
            C val;
            int64_t gp;  // global line position of the output
            if (a.mode == 0) {
                const int cl = lpo >> a.lg_len, m = lpo & (a.len - 1);
                const int c = c0 + cl;
                const int src_lp = cl + (m << a.lg_Gt);
                val = sm[a.contiguous ? (v << a.lg_nlt) + src_lp : (src_lp << a.lg_V) + v];
                if (c != 0 && m != 0) val = cmul(val, dirw<DIR>(tw[c * m]));
                gp = ((int64_t)c << a.lg_len) + m;
            } else {
                val = sm[e];
                gp = c0 + (lpo & (a.Gt - 1)) + ((int64_t)(lpo >> a.lg_Gt) << a.lg_G);
            }
            if (a.scale != 1.0) val = cscale(val, scale);
            const int64_t g = a.contiguous ? gbase + (int64_t)v * a.nl + gp : gbase + gp * a.inner + v;
            dst[g] = val;
        }
        __syncthreads();
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

template <typename C, int DIR>
cudaError_t launch_axis_t(const AxisPass &a, cudaStream_t st) {
    size_t smem = (size_t)a.tile * sizeof(C);
    int64_t grid = a.tiles < (int64_t)1 << 30 ? a.tiles : (int64_t)1 << 30;
    const int r0 = a.nstages > 0 && a.radix[0] != 8 ? a.radix[0] : 1;
    switch (r0) {
        case 2: axis_pass_kernel<C, DIR, 2><<<(unsigned)grid, a.threads, smem, st>>>(a); break;
        case 4: axis_pass_kernel<C, DIR, 4><<<(unsigned)grid, a.threads, smem, st>>>(a); break;
        case 16: axis_pass_kernel<C, DIR, 16><<<(unsigned)grid, a.threads, smem, st>>>(a); break;
        default: axis_pass_kernel<C, DIR, 1><<<(unsigned)grid, a.threads, smem, st>>>(a); break;
    }
    return cudaGetLastError();
}

template <typename C, int DIR, int R0>
cudaError_t prepare_axis_r() {
    return cudaFuncSetAttribute(axis_pass_kernel<C, DIR, R0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kMaxDynSmem);
}

template <typename C, int DIR>
cudaError_t prepare_axis_t() {
    cudaError_t e = prepare_axis_r<C, DIR, 1>();
    if (e == cudaSuccess) e = prepare_axis_r<C, DIR, 2>();
    if (e == cudaSuccess) e = prepare_axis_r<C, DIR, 4>();
    if (e == cudaSuccess) e = prepare_axis_r<C, DIR, 16>();
    return e;
}

}  // namespace

size_t axis_pass_smem_bytes(const AxisPass &a, int is_double) {
    return (size_t)a.tile * (is_double ? sizeof(double2) : sizeof(float2));
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
