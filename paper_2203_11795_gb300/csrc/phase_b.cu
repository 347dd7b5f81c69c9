// Phase B in one pass: Superstep 2 of Algorithm 2.3 (Sec. 2.2) when every
// p_l <= 16.
//
// After the redistribution, the p = p_1 ... p_d values that one length-p DFT
// needs sit at the global positions m + s' (n/p), s' in [p_1] x ... x [p_d],
// for a fixed m in [n/p] (per axis m_l + s'_l n_l/p_l; Superstep 2 applies
// F_{p_1} x ... x F_{p_d} to W^{(s)}(t : n/p^2 : n/p), whose global positions
// are exactly these).  The output k is written back to m + k (n/p), so the
// pass is in place.
//
// A tile holds all p values for Mt consecutive m_d (the contiguous axis), so
// every global access is a run of Mt elements.  Two forms of the DFT stages:
// complex64 runs them in registers (phase_b_reg.cuh: each stage takes one
// group of at most 16 values per thread, the first loading from HBM and the
// last storing to it, shared memory in between); complex128, and complex64
// plans whose first pass is one axis over short runs, run one radix-p_l
// butterfly per group in a shared tile (generic_tiles.cuh).  Stages are
// separated by block barriers.  The inverse multiplies by 1/N in the store.
#include <cuda_runtime.h>

#include "fft_device.cuh"
#include "fftu_internal.h"
#include <cstring>

#include "generic_tiles.cuh"
#include "phase_b_reg.cuh"

namespace fftu {

namespace {

constexpr int kPairsPerThread = 16;  // complex64 tiles up to 16 x 2 x 256 elements take the offset path

// complex64: three CTAs of 256 threads per SM (64 KB tiles), the offsets of a thread held in 16 registers.
// SWZ: the tile's shared slots are swizzled (PhaseBFused::swz_*); a separate instantiation, so that the
// other plans run without the index arithmetic.
template <typename C, int DIR, bool SWZ>
__global__ void __launch_bounds__(256, sizeof(C) == 8 ? 3 : 1) phase_b_fused_kernel(const __grid_constant__ PhaseBFused b) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw);
    C *__restrict__ data = static_cast<C *>(b.data);
    if constexpr (sizeof(C) == 8) {
        if (b.Mt >= 2 && b.P * b.Mt <= 2 * kPairsPerThread * (int)blockDim.x &&
            phaseb_offset(b, b.P * b.Mt - 1) < (int64_t)INT32_MAX) {
            // every tile has the same offsets from its base (the largest is the last element's): compute
            // this thread's once, in 32 bits
            int off[kPairsPerThread];
#pragma unroll
            for (int k = 0; k < kPairsPerThread; ++k) {
                const int e = 2 * ((int)threadIdx.x + k * (int)blockDim.x);
                off[k] = e < b.P * b.Mt ? (int)phaseb_offset(b, e) : 0;
            }
            for (int64_t t = blockIdx.x; t < b.tiles; t += gridDim.x)
                phaseb_tile_pairs<DIR, kPairsPerThread, SWZ>(b, t, sm, data, off);
            return;
        }
    }
    for (int64_t t = blockIdx.x; t < b.tiles; t += gridDim.x) phaseb_tile<C, DIR, SWZ>(b, t, sm, data);
}

template <int DIR>
__global__ void __launch_bounds__(256) phase_b_reg_kernel(const __grid_constant__ PhaseBFused b,
                                                          const __grid_constant__ PBGroups g) {
    extern __shared__ __align__(16) float2 pbr_sm[];
    float2 *__restrict__ data = static_cast<float2 *>(b.data);
    const float scale = (float)b.scale;
    for (int64_t t = blockIdx.x; t < b.tiles; t += gridDim.x) {
        const int64_t base = phaseb_base(b, t);
        for (int gi = 0; gi < g.n; ++gi) {
            const bool first = gi == 0, last = gi == g.n - 1;
            switch (g.lo[gi] * 100 + g.hi[gi]) {
                case 201: pb_stage<DIR, 2, 1>(b, g, gi, base, pbr_sm, data, first, last, scale); break;
                case 401: pb_stage<DIR, 4, 1>(b, g, gi, base, pbr_sm, data, first, last, scale); break;
                case 801: pb_stage<DIR, 8, 1>(b, g, gi, base, pbr_sm, data, first, last, scale); break;
                case 1601: pb_stage<DIR, 16, 1>(b, g, gi, base, pbr_sm, data, first, last, scale); break;
                case 202: pb_stage<DIR, 2, 2>(b, g, gi, base, pbr_sm, data, first, last, scale); break;
                case 204: pb_stage<DIR, 2, 4>(b, g, gi, base, pbr_sm, data, first, last, scale); break;
                case 402: pb_stage<DIR, 4, 2>(b, g, gi, base, pbr_sm, data, first, last, scale); break;
                case 404: pb_stage<DIR, 4, 4>(b, g, gi, base, pbr_sm, data, first, last, scale); break;
                case 208: pb_stage<DIR, 2, 8>(b, g, gi, base, pbr_sm, data, first, last, scale); break;
                case 802: pb_stage<DIR, 8, 2>(b, g, gi, base, pbr_sm, data, first, last, scale); break;
                default: break;
            }
            __syncthreads();
        }
    }
}

// Axis groups of the register-resident phase B (the same grouping as phaseb_dfts); false if some axis has
// p_l > 16 or p_l = 1 between grouped axes is not representable.
bool pb_groups(const PhaseBFused &b, PBGroups &g) {
    std::memset(&g, 0, sizeof(g));
    int off = b.lg_Mt;
    for (int l = b.d - 1; l >= 0;) {
        if (b.p[l] == 1) {
            --l;
            continue;
        }
        const int pp = (l > 0 && b.p[l - 1] > 1) ? b.p[l] * b.p[l - 1] : 0;
        if (g.n >= FFTU_MAX_DIMS) return false;
        g.off[g.n] = off;
        g.lo[g.n] = b.p[l];
        g.lst_lo[g.n] = b.L[l] * b.stride[l];
        if (pp > 0 && pp <= 16) {
            g.hi[g.n] = b.p[l - 1];
            g.lst_hi[g.n] = b.L[l - 1] * b.stride[l - 1];
            off += b.lg_p[l] + b.lg_p[l - 1];
            l -= 2;
        } else {
            g.hi[g.n] = 1;
            g.lst_hi[g.n] = 0;
            off += b.lg_p[l];
            l -= 1;
        }
        ++g.n;
    }
    return g.n > 0;
}

template <typename C, int DIR>
cudaError_t launch_b_t(const PhaseBFused &b, cudaStream_t st) {
    if constexpr (sizeof(C) == 8) {
        // complex64: the register-resident stages, except where the swizzled shared tile applies (a single-axis
        // first pass over short runs), which measured faster there (64^4 at p = 8^4: 0.111 against 0.119 ms;
        // 32^5 at p = 4^5: 0.153 -> 0.134 ms and 16384^2 at p = 16^2: 0.830 -> 0.731 ms with the stages)
        PBGroups g;
        if (b.swz_mask == 0 && b.P * b.Mt <= 8192 && pb_groups(b, g)) {
            const size_t smem = (size_t)b.P * b.Mt * sizeof(C);
            int64_t grid = b.tiles < (int64_t)1 << 30 ? b.tiles : (int64_t)1 << 30;
            phase_b_reg_kernel<DIR><<<(unsigned)grid, 256, smem, st>>>(b, g);
            return cudaGetLastError();
        }
    }
    size_t smem = (size_t)b.P * b.Mt * sizeof(C);
    int64_t grid = b.tiles < (int64_t)1 << 30 ? b.tiles : (int64_t)1 << 30;
    if (sizeof(C) == 8 && b.swz_mask != 0)
        phase_b_fused_kernel<C, DIR, true><<<(unsigned)grid, b.threads, smem, st>>>(b);
    else
        phase_b_fused_kernel<C, DIR, false><<<(unsigned)grid, b.threads, smem, st>>>(b);
    return cudaGetLastError();
}

template <typename C, int DIR>
cudaError_t prepare_b_t() {
    if constexpr (sizeof(C) == 8) {
        cudaError_t e0 = cudaFuncSetAttribute(phase_b_reg_kernel<DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              kMaxDynSmem);
        if (e0 != cudaSuccess) return e0;
    }
    cudaError_t e = cudaFuncSetAttribute(phase_b_fused_kernel<C, DIR, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(phase_b_fused_kernel<C, DIR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kMaxDynSmem);
    return e;
}

}  // namespace

cudaError_t prepare_phase_b_fused(int is_double, int dir) {
    if (is_double) return dir < 0 ? prepare_b_t<double2, -1>() : prepare_b_t<double2, 1>();
    return dir < 0 ? prepare_b_t<float2, -1>() : prepare_b_t<float2, 1>();
}

size_t phase_b_fused_smem_bytes(const PhaseBFused &b, int is_double) {
    return (size_t)b.P * b.Mt * (is_double ? sizeof(double2) : sizeof(float2));
}

cudaError_t launch_phase_b_fused(const PhaseBFused &b, int is_double, int dir, cudaStream_t st) {
    if (is_double) return dir < 0 ? launch_b_t<double2, -1>(b, st) : launch_b_t<double2, 1>(b, st);
    return dir < 0 ? launch_b_t<float2, -1>(b, st) : launch_b_t<float2, 1>(b, st);
}

}  // namespace fftu
