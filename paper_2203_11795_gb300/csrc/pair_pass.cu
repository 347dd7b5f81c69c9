// Phase A of two adjacent axes in one pass, each sub-FFT held in registers (complex64).
//
// For axes a and b = a + 1 with equal sub-FFT lengths L = n_a / p_a = n_b / p_b (8 or 16), every residue
// class (s_a, s_b) of every plane (a fixed position of the other axes) gets the two-dimensional DFT of its
// L x L elements x[m_a p_a + s_a][m_b p_b + s_b] (Superstep 0 of Alg. 2.3 on those two axes), the twiddles
// w_{n_a}^{k_a s_a} w_{n_b}^{k_b s_b} of Sec. 2.2, and the Put position (s_a L + k_a, s_b L + k_b) of
// Superstep 1.  Two strided passes (axis_pass.cu) would move the array through HBM twice; this pass moves it
// once:
//   stage 1: thread (s_b, s_a, m_a) loads its row of L values, F_L over m_b, times w_{n_b}^{s_b k_b};
//   stage 2: thread (k_b, s_b, s_a) takes its column from shared memory, F_L over m_a, times w_{n_a}^{s_a k_a},
//            and stores the column at its Put positions.
// The exchange stores element (m_a, k_b) of class c at c L^2 + ((m_a L + k_b) ^ sw(c)); the XOR swizzle
// (a bijection on each class block) and the 16 / W pad between the items' regions on a strided pair give
// 2 wavefronts per warp access (checked on the CPU in tests/test_pair_pass_maps.py).
//
// A CTA runs W items: W adjacent planes when b is the contiguous axis (stage-2 stores are runs of n_b
// elements), or W adjacent inner positions otherwise (thread t takes item t % W, so that a warp's loads and
// stores are runs of W elements).  Never in place: it reads src and writes dst.
#include <cuda_runtime.h>

#include "fft_device.cuh"
#include "fftu_internal.h"

namespace fftu {
namespace {

constexpr int kPairMaxThreads = 1024;

// XOR applied to (m_a L + k_b) within class c's block of the exchange.
template <int L> __device__ __forceinline__ int pair_sw(int c) {
    if constexpr (L == 16) return c & 15;
    else return (c & 7) | (((c ^ (c >> 3)) & 1) << 3);
}

template <int L, int DIR, bool CONTIG>
__global__ void __launch_bounds__(kPairMaxThreads) pair_pass_kernel(const __grid_constant__ PairPass a) {
    constexpr int LL = L * L;
    constexpr int LG_L = L == 8 ? 3 : 4;
    extern __shared__ __align__(16) float2 pair_sm[];
    const int t = threadIdx.x;
    const int lg_roles = a.lg_pa + a.lg_pb + LG_L;
    int it, r;  // item of the CTA and role within the item
    int64_t base;  // element offset of the item's plane origin
    if constexpr (CONTIG) {
        it = t >> lg_roles;
        r = t & ((1 << lg_roles) - 1);
        base = ((int64_t)blockIdx.x * a.W + it) * a.na * a.nb;
    } else {
        it = t & (a.W - 1);
        r = t >> a.lg_W;
        const int64_t vgroups = a.inner >> a.lg_W;
        const int64_t b = blockIdx.x;
        const int64_t vg = b % vgroups, o = b / vgroups;
        base = o * a.na * a.nb * a.inner + (vg << a.lg_W) + it;
    }
    const int64_t s = CONTIG ? 1 : a.inner;  // element stride within a plane's row
    float2 *reg = pair_sm + it * (a.pa * a.pb * LL + a.pad);
    float2 v[L];

    // stage 1: role (s_b, s_a, m_a): the row m_a p_a + s_a at columns m_b p_b + s_b
    {
        const int sb = r & (a.pb - 1), sa = (r >> a.lg_pb) & (a.pa - 1), ma = r >> (a.lg_pb + a.lg_pa);
        const int c = sa * a.pb + sb;
        const float2 *__restrict__ src =
            static_cast<const float2 *>(a.src) + base + ((int64_t)(ma * a.pa + sa) * a.nb + sb) * s;
#pragma unroll
        for (int mb = 0; mb < L; ++mb) v[mb] = src[(int64_t)mb * a.pb * s];
        dft_small<L, DIR>(v);
        const float2 *__restrict__ twb = static_cast<const float2 *>(a.twb);
#pragma unroll
        for (int kb = 1; kb < L; ++kb) v[kb] = cmul(v[kb], dirw<DIR>(twb[sb * kb]));
        const int sw = pair_sw<L>(c);
        float2 *blk = reg + c * LL;
#pragma unroll
        for (int kb = 0; kb < L; ++kb) blk[(ma * L + kb) ^ sw] = v[kb];
    }
    __syncthreads();

    // stage 2: role (k_b, s_b, s_a): column k_b of class (s_a, s_b), F_L over m_a, Put store
    {
        const int kb = r & (L - 1), sb = (r >> LG_L) & (a.pb - 1), sa = r >> (LG_L + a.lg_pb);
        const int c = sa * a.pb + sb;
        const int sw = pair_sw<L>(c);
        const float2 *blk = reg + c * LL;
#pragma unroll
        for (int ma = 0; ma < L; ++ma) v[ma] = blk[(ma * L + kb) ^ sw];
        dft_small<L, DIR>(v);
        const float2 *__restrict__ twa = static_cast<const float2 *>(a.twa);
#pragma unroll
        for (int ka = 1; ka < L; ++ka) v[ka] = cmul(v[ka], dirw<DIR>(twa[sa * ka]));
        float2 *__restrict__ dst =
            static_cast<float2 *>(a.dst) + base + ((int64_t)(sa * L) * a.nb + sb * L + kb) * s;
#pragma unroll
        for (int ka = 0; ka < L; ++ka) dst[(int64_t)ka * a.nb * s] = v[ka];
    }
}

template <int L, int DIR>
cudaError_t launch_l(const PairPass &a, cudaStream_t st) {
    const dim3 grid((unsigned)a.ctas);
    if (a.contiguous)
        pair_pass_kernel<L, DIR, true><<<grid, a.threads, a.smem, st>>>(a);
    else
        pair_pass_kernel<L, DIR, false><<<grid, a.threads, a.smem, st>>>(a);
    return cudaGetLastError();
}

template <int DIR>
cudaError_t launch_dir(const PairPass &a, cudaStream_t st) {
    return a.L == 8 ? launch_l<8, DIR>(a, st) : a.L == 16 ? launch_l<16, DIR>(a, st) : cudaErrorInvalidValue;
}

template <int L, int DIR>
cudaError_t prepare_l() {
    cudaError_t e = cudaFuncSetAttribute(pair_pass_kernel<L, DIR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kMaxDynSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(pair_pass_kernel<L, DIR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kMaxDynSmem);
    return e;
}

}  // namespace

cudaError_t prepare_pair_pass(int dir) {
    if (dir < 0) {
        cudaError_t e = prepare_l<8, -1>();
        return e == cudaSuccess ? prepare_l<16, -1>() : e;
    }
    cudaError_t e = prepare_l<8, 1>();
    return e == cudaSuccess ? prepare_l<16, 1>() : e;
}

cudaError_t launch_pair_pass(const PairPass &a, int dir, cudaStream_t st) {
    if (a.ctas < 1 || a.ctas > 0x7fffffffll || a.threads < 32 || a.threads > kPairMaxThreads ||
        a.threads != a.W * a.pa * a.pb * a.L || a.pa * a.pb < 16 || a.smem > (size_t)kMaxDynSmem)
        return cudaErrorInvalidValue;
    return dir < 0 ? launch_dir<-1>(a, st) : launch_dir<1>(a, st);
}

}  // namespace fftu
