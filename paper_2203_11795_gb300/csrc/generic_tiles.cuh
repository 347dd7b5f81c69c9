// Per-tile bodies of the generic kernels, shared by the one-pass-per-launch kernels
// (axis_pass.cu, phase_b.cu) and the persistent batch kernel (batch.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "fft_device.cuh"
#include "fftu_internal.h"
#include "umma16.cuh"

namespace fftu {

// complex values a thread holds per stage: 16 (c64) or 8 (c128)
template <typename C> __host__ __device__ constexpr int ept() { return sizeof(C) == 8 ? kEptMax : kEptMax / 2; }

// Global -> shared copy of one element without a register round trip (cp.async): a thread can
// have all of its tile's loads in flight at once.  Completed by async_copy_wait() + __syncthreads().
template <typename C> __device__ __forceinline__ void async_copy(C *dst_shared, const C *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_shared);
    if constexpr (sizeof(C) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void async_copy_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Two adjacent complex64 elements in one 16-byte copy (both addresses 16-byte aligned).
__device__ __forceinline__ void async_copy_pair(float2 *dst_shared, const float2 *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_shared);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}


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
                C x = sm[smi(base + (b + r * per_col) * js, a.swz)];
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
            for (int r = 0; r < R; ++r) sm[smi(base + (o + r * Ns) * js, a.swz)] = v[q][r];
        }
    }
    __syncthreads();
}

// One tile of a generic strided pass (see AxisPass): load, Stockham stages, permuted store.
// TCK = 0: radix R0 first, then radix 8 (CUDA cores).  TCK = 1 / 2: radix-16 stages as split
// bfloat16 / float16 tcgen05 tensor-core contractions (umma16.cuh; `u` set up by the kernel), then
// one CUDA-core stage of radix R0 (the rest of len).  TCK = 3: radix-16 CUDA-core stages, then one
// stage of radix R0.
template <typename C, int DIR, int R0, int TCK = 0>
__device__ __forceinline__ void axis_tile(const AxisPass &a, int64_t t, C *sm, const C *__restrict__ src,
                                          C *__restrict__ dst, const C *__restrict__ tw, UmmaCtx *u = nullptr) {
    using Rl = typename real_of<C>::type;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int chunks = 1 << a.lg_chunks;  // class chunks per line
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
    // complex64 tiles whose elements 2k and 2k + 1 are adjacent in global memory (runs of Gt >= 2
    // classes along a line, or vectors of a strided axis): loads and stores go in 16-byte pairs with
    // one index computation per pair.
    const bool pairs = sizeof(C) == 8 && (a.contiguous ? a.Gt >= 2 && (a.mode == 1 || a.len >= 2) : a.V >= 2);
    // load: shared index e is the natural order of the tile (tile line position lp, vector v);
    // tile position lp = c_local + j Gt holds line position c0 + c_local + j G
    if (pairs) {
        const int half = a.tile >> 1;
        for (int e2 = tid; e2 < half; e2 += nt) {
            const int e = e2 << 1;
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
            async_copy_pair(reinterpret_cast<float2 *>(sm + smi(e, a.swz)), reinterpret_cast<const float2 *>(src + g));
        }
    } else
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
        async_copy(sm + smi(e, a.swz), src + g);
    }
    async_copy_wait();
    __syncthreads();

    int Ns = 1;
    if constexpr (TCK == 0) {
        if constexpr (R0 > 1) {
            stockham_stage<C, DIR, R0>(sm, tw, a, Ns, tid, nt);
            Ns = R0;
        }
        for (; Ns < a.len; Ns *= 8) stockham_stage<C, DIR, 8>(sm, tw, a, Ns, tid, nt);
    } else if constexpr (TCK == 3) {
        for (; Ns * 16 <= a.len; Ns *= 16) stockham_stage<C, DIR, 16>(sm, tw, a, Ns, tid, nt);
        if constexpr (R0 > 1) {
            if (Ns < a.len) stockham_stage<C, DIR, R0>(sm, tw, a, Ns, tid, nt);
        }
    } else {
        static_assert(sizeof(C) == 8, "split-precision stages are for complex64");
        for (; Ns * 16 <= a.len; Ns *= 16) stockham_stage_umma16<DIR, TCK>(sm, tw, a, Ns, *u);
        if constexpr (R0 > 1) {
            if (Ns < a.len) stockham_stage<C, DIR, R0>(sm, tw, a, Ns, tid, nt);
        }
    }

    // store with the output permutation, twiddle and scale
    const Rl scale = (Rl)a.scale;
    if (pairs) {
        const int half = a.tile >> 1;
        for (int e2 = tid; e2 < half; e2 += nt) {
            const int e = e2 << 1;
            int lpo, v;
            if (a.contiguous) {
                v = e >> a.lg_nlt;
                lpo = e & (a.nlt - 1);
            } else {
                lpo = e >> a.lg_V;
                v = e & (a.V - 1);
            }
            C v0, v1;
            int64_t gp;
            if (a.mode == 0) {
                const int cl = lpo >> a.lg_len, m = lpo & (a.len - 1);  // m even in the contiguous case
                const int c = c0 + cl;
                if (a.contiguous) {  // the pair is (m, m + 1) of class c
                    const int row = v << a.lg_nlt;
                    v0 = sm[smi(row + cl + (m << a.lg_Gt), a.swz)];
                    v1 = sm[smi(row + cl + ((m + 1) << a.lg_Gt), a.swz)];
                    if (c != 0) {
                        if (m != 0) v0 = cmul(v0, dirw<DIR>(tw[c * m]));
                        v1 = cmul(v1, dirw<DIR>(tw[c * (m + 1)]));
                    }
                } else {  // the pair is vectors (v, v + 1) of one output position
                    const int base = ((cl + (m << a.lg_Gt)) << a.lg_V) + v;
                    const float4 pv = *reinterpret_cast<const float4 *>(sm + smi(base, a.swz));  // base even
                    v0 = mk<C>(pv.x, pv.y);
                    v1 = mk<C>(pv.z, pv.w);
                    if (c != 0 && m != 0) {
                        const C w = dirw<DIR>(tw[c * m]);
                        v0 = cmul(v0, w);
                        v1 = cmul(v1, w);
                    }
                }
                gp = ((int64_t)c << a.lg_len) + m;
            } else {
                const float4 pv = *reinterpret_cast<const float4 *>(sm + smi(e, a.swz));
                v0 = mk<C>(pv.x, pv.y);
                v1 = mk<C>(pv.z, pv.w);
                gp = c0 + (lpo & (a.Gt - 1)) + ((int64_t)(lpo >> a.lg_Gt) << a.lg_G);
            }
            if (a.scale != 1.0) {
                v0 = cscale(v0, scale);
                v1 = cscale(v1, scale);
            }
            const int64_t g = a.contiguous ? gbase + (int64_t)v * a.nl + gp : gbase + gp * a.inner + v;
            *reinterpret_cast<float4 *>(dst + g) = make_float4(v0.x, v0.y, v1.x, v1.y);
        }
        __syncthreads();
        return;
    }
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
            val = sm[smi(a.contiguous ? (v << a.lg_nlt) + src_lp : (src_lp << a.lg_V) + v, a.swz)];
            if (c != 0 && m != 0) val = cmul(val, dirw<DIR>(tw[c * m]));
            gp = ((int64_t)c << a.lg_len) + m;
        } else {
            val = sm[smi(e, a.swz)];
            gp = c0 + (lpo & (a.Gt - 1)) + ((int64_t)(lpo >> a.lg_Gt) << a.lg_G);
        }
        if (a.scale != 1.0) val = cscale(val, scale);
        const int64_t g = a.contiguous ? gbase + (int64_t)v * a.nl + gp : gbase + gp * a.inner + v;
        dst[g] = val;
    }
    __syncthreads();
}

// Shared slot of phase-B tile element e (see PhaseBFused::swz_*; keeps the pairs (2k, 2k + 1) together).
// SWZ = false: the identity (no index arithmetic).
template <bool SWZ> __device__ __forceinline__ int pbs(const PhaseBFused &b, int e) {
    if constexpr (SWZ) return e ^ (((e >> b.swz_src) & b.swz_mask) << b.swz_dst);
    else return e;
}

template <typename C, int DIR, int R, bool SWZ = false>
__device__ __forceinline__ void axis_dft(const PhaseBFused &pb, C *sm, int total, int S, int tid, int nt) {
    // groups: total / R, group g -> base (g / S) * S * R + g % S, stride S (S a power of two)
    const int groups = total / R;
    const int lg_s = 31 - __clz(S);
    for (int g = tid; g < groups; g += nt) {
        const int base = ((g >> lg_s) << lg_s) * R + (g & (S - 1));
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = sm[pbs<SWZ>(pb, base + r * S)];
        dft_small<R, DIR>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) sm[pbs<SWZ>(pb, base + r * S)] = v[r];
    }
}

// F_{R1} along a stride-S axis and F_{R2} along the next (stride S R1) in one shared-memory pass: each group
// holds the R1 x R2 values of one fixed position of the other axes in registers.
template <typename C, int DIR, int R1, int R2, bool SWZ = false>
__device__ __forceinline__ void axis_dft2(const PhaseBFused &pb, C *sm, int total, int S, int tid, int nt) {
    const int groups = total / (R1 * R2);
    const int lg_s = 31 - __clz(S);
    for (int g = tid; g < groups; g += nt) {
        const int base = ((g >> lg_s) << lg_s) * (R1 * R2) + (g & (S - 1));
        C v[R1 * R2];
#pragma unroll
        for (int r = 0; r < R1 * R2; ++r) v[r] = sm[pbs<SWZ>(pb, base + r * S)];
#pragma unroll
        for (int r2 = 0; r2 < R2; ++r2) {
            C w[R1];
#pragma unroll
            for (int r1 = 0; r1 < R1; ++r1) w[r1] = v[r2 * R1 + r1];
            dft_small<R1, DIR>(w);
#pragma unroll
            for (int r1 = 0; r1 < R1; ++r1) v[r2 * R1 + r1] = w[r1];
        }
#pragma unroll
        for (int r1 = 0; r1 < R1; ++r1) {
            C w[R2];
#pragma unroll
            for (int r2 = 0; r2 < R2; ++r2) w[r2] = v[r2 * R1 + r1];
            dft_small<R2, DIR>(w);
#pragma unroll
            for (int r2 = 0; r2 < R2; ++r2) v[r2 * R1 + r1] = w[r2];
        }
#pragma unroll
        for (int r = 0; r < R1 * R2; ++r) sm[pbs<SWZ>(pb, base + r * S)] = v[r];
    }
}

// Offset of tile element e (e even when pairs) from the tile's base: the m_d position and the s'_l of every
// axis (shared by all tiles; the fused phase-B kernel computes a thread's offsets once).
__device__ __forceinline__ int64_t phaseb_offset(const PhaseBFused &b, int e) {
    const int d = b.d;
    const int mt = e & (b.Mt - 1);
    int sf = e >> b.lg_Mt;
    int64_t g = (int64_t)mt * b.stride[d - 1];
    for (int l = d - 1; l >= 0; --l) {
        const int sl = sf & (b.p[l] - 1);
        sf >>= b.lg_p[l];
        g += (int64_t)sl * b.L[l] * b.stride[l];
    }
    return g;
}

// Global element offset of tile t's first element (m_0 .. m_{d-2} and the first m_{d-1} of the tile).
__device__ __forceinline__ int64_t phaseb_base(const PhaseBFused &b, int64_t t) {
    const int d = b.d;
    const int lg_td = b.lg_L[d - 1] - b.lg_Mt;  // tiles along the last axis (log2)
    int64_t rem = t >> lg_td;
    int64_t base = ((t & (((int64_t)1 << lg_td) - 1)) << b.lg_Mt) * b.stride[d - 1];
    for (int l = d - 2; l >= 0; --l) {
        base += (rem & (b.L[l] - 1)) * b.stride[l];
        rem >>= b.lg_L[l];
    }
    return base;
}

// The DFT stages of a landed phase-B tile: F_{p_l} along every axis, last axis first, two adjacent axes per
// shared-memory pass where p_l p_{l-1} <= 16.
template <typename C, int DIR, bool SWZ = false>
__device__ __forceinline__ void phaseb_dfts(const PhaseBFused &b, C *sm) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int total = b.P * b.Mt;
    int S = b.Mt;
    for (int l = b.d - 1; l >= 0; --l) {
        const int pp = (l > 0 && b.p[l] > 1 && b.p[l - 1] > 1) ? b.p[l] * b.p[l - 1] : 0;
        if (pp > 0 && pp <= 16) {
            switch (b.p[l] * 100 + b.p[l - 1]) {
                case 202: axis_dft2<C, DIR, 2, 2, SWZ>(b, sm, total, S, tid, nt); break;
                case 204: axis_dft2<C, DIR, 2, 4, SWZ>(b, sm, total, S, tid, nt); break;
                case 208: axis_dft2<C, DIR, 2, 8, SWZ>(b, sm, total, S, tid, nt); break;
                case 402: axis_dft2<C, DIR, 4, 2, SWZ>(b, sm, total, S, tid, nt); break;
                case 404: axis_dft2<C, DIR, 4, 4, SWZ>(b, sm, total, S, tid, nt); break;
                case 802: axis_dft2<C, DIR, 8, 2, SWZ>(b, sm, total, S, tid, nt); break;
                default: break;
            }
            S *= pp;
            --l;
        } else {
            switch (b.p[l]) {
                case 2: axis_dft<C, DIR, 2, SWZ>(b, sm, total, S, tid, nt); break;
                case 4: axis_dft<C, DIR, 4, SWZ>(b, sm, total, S, tid, nt); break;
                case 8: axis_dft<C, DIR, 8, SWZ>(b, sm, total, S, tid, nt); break;
                case 16: axis_dft<C, DIR, 16, SWZ>(b, sm, total, S, tid, nt); break;
                default: break;
            }
            S *= b.p[l];
        }
        __syncthreads();
    }
}

// One complex64 phase-B tile with the thread's element offsets from the tile base precomputed (16-byte
// pairs; K pairs per thread at most): the per-element index arithmetic is one add.
template <int DIR, int K, bool SWZ = false>
__device__ __forceinline__ void phaseb_tile_pairs(const PhaseBFused &b, int64_t t, float2 *sm, float2 *__restrict__ data,
                                                  const int (&off)[K]) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int total = b.P * b.Mt;
    const int64_t base = phaseb_base(b, t);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int e = 2 * (tid + k * nt);
        if (e < total)
            async_copy_pair(sm + pbs<SWZ>(b, e), data + base + off[k]);
    }
    async_copy_wait();
    __syncthreads();
    phaseb_dfts<float2, DIR, SWZ>(b, sm);
    const float scale = (float)b.scale;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int e = 2 * (tid + k * nt);
        if (e < total) {
            float4 v = *reinterpret_cast<const float4 *>(sm + pbs<SWZ>(b, e));
            if (b.scale != 1.0) {
                v.x *= scale;
                v.y *= scale;
                v.z *= scale;
                v.w *= scale;
            }
            *reinterpret_cast<float4 *>(data + base + off[k]) = v;
        }
    }
    __syncthreads();
}

// One tile of the generic fused phase B (see PhaseBFused): all p values for Mt consecutive m_d.
template <typename C, int DIR, bool SWZ = false>
__device__ __forceinline__ void phaseb_tile(const PhaseBFused &b, int64_t t, C *sm, C *__restrict__ data) {
    using Rl = typename real_of<C>::type;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int d = b.d;
    const int total = b.P * b.Mt;
    const int64_t base = phaseb_base(b, t);  // fixed m_0..m_{d-2} and the first m_{d-1}
    // complex64 with Mt >= 2: elements mt and mt + 1 are adjacent along the last axis (stride 1),
    // so loads and stores go in 16-byte pairs with one index computation per pair
    const bool pairs = sizeof(C) == 8 && b.Mt >= 2;
    const int step = pairs ? 2 : 1;
    for (int e = tid * step; e < total; e += nt * step) {
        const int mt = e & (b.Mt - 1);
        int sf = e >> b.lg_Mt;
        int64_t g = base + (int64_t)mt * b.stride[d - 1];
        for (int l = d - 1; l >= 0; --l) {
            const int sl = sf & (b.p[l] - 1);
            sf >>= b.lg_p[l];
            g += (int64_t)sl * b.L[l] * b.stride[l];
        }
        if (pairs)
            async_copy_pair(reinterpret_cast<float2 *>(sm + pbs<SWZ>(b, e)), reinterpret_cast<const float2 *>(data + g));
        else
            async_copy(sm + pbs<SWZ>(b, e), data + g);
    }
    async_copy_wait();
    __syncthreads();
    phaseb_dfts<C, DIR, SWZ>(b, sm);
    const Rl scale = (Rl)b.scale;
    for (int e = tid * step; e < total; e += nt * step) {
        const int mt = e & (b.Mt - 1);
        int sf = e >> b.lg_Mt;
        int64_t g = base + (int64_t)mt * b.stride[d - 1];
        for (int l = d - 1; l >= 0; --l) {
            const int sl = sf & (b.p[l] - 1);
            sf >>= b.lg_p[l];
            g += (int64_t)sl * b.L[l] * b.stride[l];
        }
        C v = sm[pbs<SWZ>(b, e)];
        if (b.scale != 1.0) v = cscale(v, scale);
        if (pairs) {
            C w = sm[pbs<SWZ>(b, e + 1)];
            if (b.scale != 1.0) w = cscale(w, scale);
            *reinterpret_cast<float4 *>(data + g) = make_float4(v.x, v.y, w.x, w.y);
        } else {
            data[g] = v;
        }
    }
    __syncthreads();
}

}  // namespace fftu
