// Phase A of the last three axes in one pass, each sub-FFT held in registers (complex64).
//
// For axes a, b, c = d - 3, d - 2, d - 1 with sub-FFT length 8 on each (n_l = 8 p_l) and p_b p_c = 16, every
// residue class (s_a, s_b, s_c) of every outer position gets the three-dimensional DFT of its 8 x 8 x 8
// elements x[m_a p_a + s_a][m_b p_b + s_b][m_c p_c + s_c] (Superstep 0 of Alg. 2.3 on those three axes), the
// twiddles w_{n_a}^{k_a s_a} w_{n_b}^{k_b s_b} w_{n_c}^{k_c s_c} of Sec. 2.2, and the Put position
// (s_a 8 + k_a, s_b 8 + k_b, s_c 8 + k_c) of Superstep 1: one HBM round trip where three strided passes
// (axis_pass.cu) take three.
//
// A CTA takes one outer position and one s_a: the 8 planes m_a p_a + s_a (8 n_b n_c elements, 64 KB at
// n_b n_c = 1024) in, the 8 planes s_a 8 + k_a out.  Its 1024 fibers per stage (16 classes x 64) go to 512
// threads, two each, one after the other (40 registers: three CTAs per SM; both at once took 63 registers, two
// CTAs per SM, and measured 3% slower):
//   stage 1: fiber (s_c, s_b, m_b, m_a) loads 8 values along c, F_8, times w_{n_c}^{s_c k_c};
//   stage 2: fiber (k_c, s_c, s_b, m_a), in place in shared memory: F_8 along b, times w_{n_b}^{s_b k_b};
//   stage 3: fiber (k_c, s_c, s_b, k_b): F_8 along a, times w_{n_a}^{s_a k_a}, stored at its Put positions
//            (a warp stores whole rows of n_c = 8 p_c consecutive elements).
// Shared layout: class q, position (x, y, z) at q 512 + ((x 64 + y 8 + z) ^ sw(q)); the swizzle gives 2
// wavefronts per warp access (checked on the CPU in tests/test_triple_pass_maps.py).  Never in place.
#include <cuda_runtime.h>

#include "fft_device.cuh"
#include "fftu_internal.h"

namespace fftu {
namespace {

constexpr int kTripleThreads = 512;

__device__ __forceinline__ int triple_sw(int q) { return ((q >> 1) & 7) | ((q & 1) << 3); }

template <int DIR>
__global__ void __launch_bounds__(kTripleThreads) triple_pass_kernel(const __grid_constant__ TriplePass a) {
    extern __shared__ __align__(16) float2 triple_sm[];
    const int64_t blk = blockIdx.x;
    const int sa = (int)(blk & (a.pa - 1));
    const int64_t o = blk >> a.lg_pa;
    const int64_t plane = (int64_t)a.nb * a.nc;
    const float2 *__restrict__ src = static_cast<const float2 *>(a.src) + o * a.na * plane;
    float2 *__restrict__ dst = static_cast<float2 *>(a.dst) + o * a.na * plane;
    const float2 *__restrict__ twa = static_cast<const float2 *>(a.twa);
    const float2 *__restrict__ twb = static_cast<const float2 *>(a.twb);
    const float2 *__restrict__ twc = static_cast<const float2 *>(a.twc);
    float2 v[8];

    // stage 1: fiber (s_c, s_b, m_b, m_a) along c
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        const int f = threadIdx.x + h * kTripleThreads;
        const int sc = f & (a.pc - 1), sb = (f >> a.lg_pc) & (a.pb - 1), mb = (f >> 4) & 7, ma = f >> 7;
        const int q = sb * a.pc + sc;
        const float2 *p = src + (int64_t)(ma * a.pa + sa) * plane + (int64_t)(mb * a.pb + sb) * a.nc + sc;
#pragma unroll
        for (int mc = 0; mc < 8; ++mc) v[mc] = p[mc * a.pc];
        dft8<DIR>(v);
#pragma unroll
        for (int kc = 1; kc < 8; ++kc) v[kc] = cmul(v[kc], dirw<DIR>(twc[sc * kc]));
        float2 *blkq = triple_sm + q * 512;
        const int sw = triple_sw(q);
#pragma unroll
        for (int kc = 0; kc < 8; ++kc) blkq[(ma * 64 + mb * 8 + kc) ^ sw] = v[kc];
    }
    __syncthreads();

    // stage 2: fiber (k_c, s_c, s_b, m_a) along b, in place
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        const int f = threadIdx.x + h * kTripleThreads;
        const int kc = f & 7, sc = (f >> 3) & (a.pc - 1), sb = (f >> (3 + a.lg_pc)) & (a.pb - 1), ma = f >> 7;
        const int q = sb * a.pc + sc;
        float2 *blkq = triple_sm + q * 512;
        const int sw = triple_sw(q);
#pragma unroll
        for (int mb = 0; mb < 8; ++mb) v[mb] = blkq[(ma * 64 + mb * 8 + kc) ^ sw];
        dft8<DIR>(v);
#pragma unroll
        for (int kb = 1; kb < 8; ++kb) v[kb] = cmul(v[kb], dirw<DIR>(twb[sb * kb]));
#pragma unroll
        for (int kb = 0; kb < 8; ++kb) blkq[(ma * 64 + kb * 8 + kc) ^ sw] = v[kb];
    }
    __syncthreads();

    // stage 3: fiber (k_c, s_c, s_b, k_b) along a, then the Put store
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        const int f = threadIdx.x + h * kTripleThreads;
        const int kc = f & 7, sc = (f >> 3) & (a.pc - 1), sb = (f >> (3 + a.lg_pc)) & (a.pb - 1), kb = f >> 7;
        const int q = sb * a.pc + sc;
        const float2 *blkq = triple_sm + q * 512;
        const int sw = triple_sw(q);
#pragma unroll
        for (int ma = 0; ma < 8; ++ma) v[ma] = blkq[(ma * 64 + kb * 8 + kc) ^ sw];
        dft8<DIR>(v);
#pragma unroll
        for (int ka = 1; ka < 8; ++ka) v[ka] = cmul(v[ka], dirw<DIR>(twa[sa * ka]));
        float2 *p = dst + (int64_t)(sa * 8) * plane + (int64_t)(sb * 8 + kb) * a.nc + sc * 8 + kc;
#pragma unroll
        for (int ka = 0; ka < 8; ++ka) p[(int64_t)ka * plane] = v[ka];
    }
}

}  // namespace

cudaError_t prepare_triple_pass(int dir) {
    return cudaFuncSetAttribute(dir < 0 ? triple_pass_kernel<-1> : triple_pass_kernel<1>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
}

cudaError_t launch_triple_pass(const TriplePass &a, int dir, cudaStream_t st) {
    if (a.ctas < 1 || a.ctas > 0x7fffffffll || a.pb * a.pc != 16 || a.na != 8 * a.pa || a.nb != 8 * a.pb ||
        a.nc != 8 * a.pc || a.smem != (size_t)8192 * sizeof(float2))
        return cudaErrorInvalidValue;
    const dim3 grid((unsigned)a.ctas);
    if (dir < 0)
        triple_pass_kernel<-1><<<grid, kTripleThreads, a.smem, st>>>(a);
    else
        triple_pass_kernel<1><<<grid, kTripleThreads, a.smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace fftu
