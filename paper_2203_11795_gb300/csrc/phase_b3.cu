// Phase B for 3D arrays with a cubic-or-not p = P0 x P1 x P2 known at compile
// time: Superstep 2 of Algorithm 2.3 (Sec. 2.2), in place.
//
// For m in [n/p], the P0 P1 P2 values at m + s' (n/p) (per axis
// m_l + s'_l L_l, L_l = n_l / p_l) are replaced by their P0 x P1 x P2 DFT
// (F_{p_1} x F_{p_2} x F_{p_3}, the proof of Theorem 2.1 shows output k lands at
// m + k (n/p)).  One CTA takes fixed (m0, m1) and MT consecutive m2, i.e. all
// P values for MT contiguous elements of each of the P row segments.
//
//   1. thread (s0', s1', m2 pair) loads the P2 values along s2' straight from
//      HBM as 16-byte pairs (two consecutive m2), runs F_{P2} in registers and
//      parks the result in shared memory;
//   2. thread (s0', k2, m2 pair) runs F_{P1} along s1' in place in shared memory;
//   3. thread (k1, k2, m2 pair) runs F_{P0} along s0' and stores the result
//      (times 1/N for the inverse) straight back to HBM as 16-byte pairs.
// Every global access of a warp covers MT*8-byte contiguous runs.
#include <cuda_runtime.h>

#include "fft_device.cuh"
#include "fftu_internal.h"

namespace fftu {

namespace {

// Two consecutive elements per access: one 16-byte float4 for complex64,
// two 16-byte double2 for complex128.  Streaming cache hints: each element
// is touched once per pass.
__device__ __forceinline__ void load_pair(const float2 *p, float2 &a, float2 &b) {
    float4 v = __ldcs(reinterpret_cast<const float4 *>(p));
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void store_pair(float2 *p, float2 a, float2 b) {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(a.x, a.y, b.x, b.y));
}
__device__ __forceinline__ void load_pair(const double2 *p, double2 &a, double2 &b) {
    a = __ldcs(p);
    b = __ldcs(p + 1);
}
__device__ __forceinline__ void store_pair(double2 *p, double2 a, double2 b) {
    __stcs(p, a);
    __stcs(p + 1, b);
}

// Shared layout: [s0][s1][s2][m2] with m2 fastest, MT + pad per row of m2.
template <typename C, int DIR, int P0, int P1, int P2, int MT>
__global__ void __launch_bounds__(P0 * P1 * MT / 2) phase_b3_kernel(const __grid_constant__ PhaseBFused b) {
    constexpr int HALF = MT / 2;
    constexpr int NT = P0 * P1 * HALF;
    constexpr bool SINGLE = P0 >= 16 || P1 >= 16;  // phases 2 and 3 on single elements (register budget)
    constexpr int RS = MT;  // shared row (m2 run) stride
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sm = reinterpret_cast<C *>(smem_raw);
    C *__restrict__ data = static_cast<C *>(b.data);
    using Rl = typename real_of<C>::type;

    const int tid = threadIdx.x;
    const int64_t L0 = b.L[0], L1 = b.L[1], L2 = b.L[2];
    const int64_t st0 = b.stride[0], st1 = b.stride[1];
    const int64_t tiles2 = L2 / MT;
    const int hp = tid % HALF;  // m2 pair
    const int g = tid / HALF;   // (x, y) pair of the two slower indices

    for (int64_t t = blockIdx.x; t < b.tiles; t += gridDim.x) {
        const int64_t m2 = (t % tiles2) * MT + 2 * hp;
        const int64_t rest = t / tiles2;
        const int64_t m1 = rest % L1, m0 = rest / L1;
        const int64_t base = m0 * st0 + m1 * st1 + m2;
        {   // 1. F_{P2} along s2' from HBM
            const int s0 = g / P1, s1 = g % P1;
            C va[P2], vb[P2];
            const C *src = data + base + s0 * L0 * st0 + s1 * L1 * st1;
#pragma unroll
            for (int r = 0; r < P2; ++r) load_pair(src + r * L2, va[r], vb[r]);
            dft_small<P2, DIR>(va);
            dft_small<P2, DIR>(vb);
#pragma unroll
            for (int r = 0; r < P2; ++r) {
                C *q = sm + ((s0 * P1 + s1) * P2 + r) * RS + 2 * hp;
                q[0] = va[r];
                q[1] = vb[r];
            }
        }
        __syncthreads();
        // 2. F_{P1} along s1': thread (s0', k2, pair); P0*P2*HALF work items.  With a 16-point axis
        //    the pair would need 64 registers of values: single elements, P0*P2*MT items.
        if constexpr (SINGLE) {
            for (int w = tid; w < P0 * P2 * MT; w += NT) {
                const int e = w % MT, q = w / MT;
                const int k2 = q % P2, s0 = q / P2;
                C v[P1];
#pragma unroll
                for (int r = 0; r < P1; ++r) v[r] = sm[((s0 * P1 + r) * P2 + k2) * RS + e];
                dft_small<P1, DIR>(v);
#pragma unroll
                for (int r = 0; r < P1; ++r) sm[((s0 * P1 + r) * P2 + k2) * RS + e] = v[r];
            }
        } else
        for (int w = tid; w < P0 * P2 * HALF; w += NT) {
            const int h = w % HALF, q = w / HALF;
            const int k2 = q % P2, s0 = q / P2;
            C va[P1], vb[P1];
#pragma unroll
            for (int r = 0; r < P1; ++r) {
                const C *p = sm + ((s0 * P1 + r) * P2 + k2) * RS + 2 * h;
                va[r] = p[0];
                vb[r] = p[1];
            }
            dft_small<P1, DIR>(va);
            dft_small<P1, DIR>(vb);
#pragma unroll
            for (int r = 0; r < P1; ++r) {
                C *p = sm + ((s0 * P1 + r) * P2 + k2) * RS + 2 * h;
                p[0] = va[r];
                p[1] = vb[r];
            }
        }
        __syncthreads();
        // 3. F_{P0} along s0' and store: thread (k1, k2, pair); P1*P2*HALF items (single elements,
        //    P1*P2*MT items, with a 16-point axis)
        const Rl scale = (Rl)b.scale;
        if constexpr (SINGLE) {
            const C *mul = static_cast<const C *>(b.mul);
            for (int w = tid; w < P1 * P2 * MT; w += NT) {
                const int e = w % MT, q = w / MT;
                const int k2 = q % P2, k1 = q / P2;
                C v[P0];
#pragma unroll
                for (int r = 0; r < P0; ++r) v[r] = sm[((r * P1 + k1) * P2 + k2) * RS + e];
                dft_small<P0, DIR>(v);
                C *dst = data + (base - 2 * hp + e) + k1 * L1 * st1 + k2 * L2;
#pragma unroll
                for (int r = 0; r < P0; ++r) {
                    C a = v[r];
                    if (b.scale != 1.0) a = cscale(a, scale);
                    if (mul) a = cmul(a, mul[(dst - data) + r * L0 * st0]);
                    __stcs(dst + r * L0 * st0, a);
                }
            }
        } else
        for (int w = tid; w < P1 * P2 * HALF; w += NT) {
            const int h = w % HALF, q = w / HALF;
            const int k2 = q % P2, k1 = q / P2;
            C va[P0], vb[P0];
#pragma unroll
            for (int r = 0; r < P0; ++r) {
                const C *p = sm + ((r * P1 + k1) * P2 + k2) * RS + 2 * h;
                va[r] = p[0];
                vb[r] = p[1];
            }
            dft_small<P0, DIR>(va);
            dft_small<P0, DIR>(vb);
            C *dst = data + (base - 2 * hp + 2 * h) + k1 * L1 * st1 + k2 * L2;
            const C *mul = static_cast<const C *>(b.mul);
#pragma unroll
            for (int r = 0; r < P0; ++r) {
                C a = va[r], c = vb[r];
                if (b.scale != 1.0) {
                    a = cscale(a, scale);
                    c = cscale(c, scale);
                }
                if (mul) {  // pointwise product in the spectral domain, same natural index
                    C ma, mc;
                    load_pair(mul + (dst - data) + r * L0 * st0, ma, mc);
                    a = cmul(a, ma);
                    c = cmul(c, mc);
                }
                store_pair(dst + r * L0 * st0, a, c);
            }
        }
        __syncthreads();
    }
}

template <typename C, int DIR, int P0, int P1, int P2, int MT>
cudaError_t launch_t(const PhaseBFused &b, cudaStream_t st) {
    constexpr int NT = P0 * P1 * MT / 2;
    const size_t smem = (size_t)P0 * P1 * P2 * MT * sizeof(C);
    int64_t grid = b.tiles < (int64_t)1 << 30 ? b.tiles : (int64_t)1 << 30;
    phase_b3_kernel<C, DIR, P0, P1, P2, MT><<<(unsigned)grid, NT, smem, st>>>(b);
    return cudaGetLastError();
}

template <typename C, int DIR, int P0, int P1, int P2, int MT>
cudaError_t prepare_t() {
    return cudaFuncSetAttribute(phase_b3_kernel<C, DIR, P0, P1, P2, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kMaxDynSmem);
}

// Instantiated grids: p_0 = p_1 = p_2 = P (kind P), and p = 16 x 16 x 8 (kind 168, complex64),
// each with a fixed MT.
int b3_kind(int p0, int p1, int p2) {
    if (p0 == p1 && p1 == p2) return p0;
    if (p0 == 16 && p1 == 16 && p2 == 8) return 168;
    return 0;
}

template <typename C, int DIR, bool PREP>
cudaError_t dispatch(int P, const PhaseBFused *b, cudaStream_t st) {
    switch (P) {
        case 168:
            if constexpr (sizeof(C) == 8)
                return PREP ? prepare_t<C, DIR, 16, 16, 8, 8>() : launch_t<C, DIR, 16, 16, 8, 8>(*b, st);
            break;
        case 2: return PREP ? prepare_t<C, DIR, 2, 2, 2, 64>() : launch_t<C, DIR, 2, 2, 2, 64>(*b, st);
        case 4: return PREP ? prepare_t<C, DIR, 4, 4, 4, 32>() : launch_t<C, DIR, 4, 4, 4, 32>(*b, st);
        case 8: return PREP ? prepare_t<C, DIR, 8, 8, 8, 16>() : launch_t<C, DIR, 8, 8, 8, 16>(*b, st);
        case 16:
            if constexpr (sizeof(C) == 8)
                return PREP ? prepare_t<C, DIR, 16, 16, 16, 4>() : launch_t<C, DIR, 16, 16, 16, 4>(*b, st);
            break;
    }
    return cudaErrorInvalidValue;
}

}  // namespace

int phase_b3_tile_mt(int p0, int p1, int p2, int is_double) {
    switch (b3_kind(p0, p1, p2)) {
        case 2: return 64;
        case 4: return 32;
        case 8: return 16;
        case 16: return is_double ? 0 : 4;
        case 168: return is_double ? 0 : 8;
    }
    return 0;
}

cudaError_t prepare_phase_b3(int is_double, int dir) {
    for (int P : {2, 4, 8, 16, 168}) {
        const int q = P == 168 ? 16 : P;
        if (phase_b3_tile_mt(q, q, P == 168 ? 8 : q, is_double) == 0) continue;
        cudaError_t e;
        if (is_double)
            e = dir < 0 ? dispatch<double2, -1, true>(P, nullptr, 0) : dispatch<double2, 1, true>(P, nullptr, 0);
        else
            e = dir < 0 ? dispatch<float2, -1, true>(P, nullptr, 0) : dispatch<float2, 1, true>(P, nullptr, 0);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_phase_b3(const PhaseBFused &b, int is_double, int dir, cudaStream_t st) {
    const int P = b3_kind(b.p[0], b.p[1], b.p[2]);
    if (is_double) return dir < 0 ? dispatch<double2, -1, false>(P, &b, st) : dispatch<double2, 1, false>(P, &b, st);
    return dir < 0 ? dispatch<float2, -1, false>(P, &b, st) : dispatch<float2, 1, false>(P, &b, st);
}

}  // namespace fftu
