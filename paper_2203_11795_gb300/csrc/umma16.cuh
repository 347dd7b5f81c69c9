// Split-precision radix-16 DFT stages on the 5th-generation tensor cores (tcgen05.mma, TMEM
// accumulators, shared-memory operand descriptors), for the strided passes of complex64 plans.
//
// A radix-16 Stockham stage applies the 16-point DFT F (F[k][r] = w_16^{k r}, the radix split of
// Sec. 2.1.1, eq. radix) to every butterfly of the tile.  Written with one butterfly per row, the
// stage is one real contraction
//     y (rows x 32) = x (rows x 32) G,   x = [x_re(16), x_im(16)],  y = [y_re(16), y_im(16)],
//     G = [[F_re, F_im], [-F_im, F_re]]   (F is symmetric),
// which the tensor cores take in 16-bit operands: x and G are split as v = v_hi + v_lo in bfloat16
// (TCK 1) or float16 (TCK 2) and the product is taken as x_hi G_hi + x_lo G_hi + x_hi G_lo with FP32
// accumulation (the x_lo G_lo term is dropped).  For float16 every row (butterfly) is first scaled by
// a power of two that puts its largest magnitude in [2^13, 2^14), so neither part leaves float16's
// range; the result is scaled back.
//
// Mapping (one CTA): its warps form groups of at most four; group g owns 128 accumulator lanes of
// TMEM columns [32 g, 32 g + 32) and a pair of A tiles (x_hi, x_lo: 128 rows x 32 16-bit values).
// Per stage, group g takes butterflies [g R, (g + 1) R) with R = 32 x (warps in the group): thread r
// of the group loads butterfly g R + r (applying the stage's twiddles), splits it and writes row r
// of the A tiles; one elected thread issues the six MMAs (M = 128, N = 32, K = 16 each: three
// products, two K halves) and commits them to the group's mbarrier; every thread waits for it and
// reads its row of the accumulator with tcgen05.ld.  The block then writes the outputs back to the
// tile in Stockham order.  G_hi and G_lo (32 x 32 each) are built once per CTA.
//
// Operand layout (no swizzle, K-major canonical layout): element (row m, k) of a tile with K = 32 sits
// at byte (m % 8) 16 + (m / 8) 512 + (k % 8) 2 + (k / 8) 128, i.e. 8 x 16-byte core matrices, the
// leading-dimension byte offset (next core matrix along K) 128 and the stride byte offset (next 8
// rows) 512; the second K half of an MMA starts 256 bytes further.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bounded_wait.cuh"
#include "fft_device.cuh"
#include "fftu_internal.h"

namespace fftu {

constexpr int kUmmaRows = 128;             // M of every MMA (accumulator lanes of one group)
constexpr int kUmmaK = 32;                 // 16 real + 16 imaginary inputs per butterfly
constexpr int kUmmaTileBytes = kUmmaRows * kUmmaK * 2;   // one A tile, 8 KB
constexpr int kUmmaBBytes = 32 * kUmmaK * 2;             // one G tile (N = 32 rows), 2 KB
constexpr long long kUmmaWaitNs = 2000000000ll;          // bounded wait for an MMA's completion

// Groups of at most four warps in a block of `threads` threads.
__host__ __device__ constexpr int umma_groups(int threads) {
    return threads >= 128 ? threads / 128 : 1;
}
// Shared memory the tensor-core stages add after the tile (128-byte aligned start): G_hi, G_lo, the
// groups' A tiles, their mbarriers and the TMEM address slot.
__host__ __device__ constexpr size_t umma_smem_bytes(int threads) {
    return 128 + 2 * (size_t)kUmmaBBytes + 2 * (size_t)kUmmaTileBytes * umma_groups(threads) +
           8 * (size_t)umma_groups(threads) + 16;
}
// TMEM columns a block allocates: 32 per group, a power of two >= 32.
__host__ __device__ constexpr int umma_tmem_cols(int threads) {
    return umma_groups(threads) <= 1 ? 32 : umma_groups(threads) <= 2 ? 64 : umma_groups(threads) <= 4 ? 128 : 256;
}

struct UmmaCtx {
    uint32_t tmem;        // TMEM base address (lane 0, first allocated column)
    uint32_t g_hi, g_lo;  // shared addresses of G_hi, G_lo
    uint32_t a0;          // shared address of group 0's A_hi tile (A_lo follows; groups follow)
    uint64_t *bar;        // one mbarrier per group
    int *status;          // plan status word: FFTU_ERR_TIMEOUT if an MMA's completion never arrived
    unsigned phase;       // parity of the next completion of this thread's group's mbarrier
};

__device__ __forceinline__ uint32_t umma_smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading (K) and stride (8-row) byte offsets, the
// descriptor version of this architecture, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr) {
    constexpr uint64_t lbo = 128 >> 4, sbo = 512 >> 4;
    return (uint64_t)((addr >> 4) & 0x3FFF) | (lbo << 16) | (sbo << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, A and B both bfloat16 (TCK 1) or float16
// (TCK 2), both K-major, N = 32, M = 128.
template <int TCK> __device__ __forceinline__ uint32_t umma_idesc() {
    constexpr uint32_t fmt = TCK == 1 ? 1u : 0u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((32u >> 3) << 17) | ((uint32_t)(kUmmaRows >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     umma_smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ bool umma_bar_try(uint64_t *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(umma_smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// 32 consecutive FP32 accumulator columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// v = hi + lo, both rounded to the 16-bit type, two values packed per 32-bit word
template <int TCK> __device__ __forceinline__ uint32_t pack16(float a, float b) {
    if constexpr (TCK == 1) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}
template <int TCK> __device__ __forceinline__ float round16(float a) {
    if constexpr (TCK == 1) return __bfloat162float(__float2bfloat16_rn(a));
    else return __half2float(__float2half_rn(a));
}

// Byte offset of (row m, k) in a K = 32 operand tile (see the layout above).
__device__ __forceinline__ uint32_t umma_off(int m, int k) {
    return (uint32_t)((m & 7) * 16 + (m >> 3) * 512 + (k & 7) * 2 + (k >> 3) * 128);
}

// Write one row of 32 FP32 values as its hi and lo 16-bit parts (four 16-byte chunks each).
template <int TCK>
__device__ __forceinline__ void umma_write_row(unsigned char *hi_tile, unsigned char *lo_tile, int m,
                                               const float (&x)[32]) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float a = x[8 * c + 2 * j], b = x[8 * c + 2 * j + 1];
            const float ah = round16<TCK>(a), bh = round16<TCK>(b);
            h[j] = pack16<TCK>(ah, bh);
            l[j] = pack16<TCK>(a - ah, b - bh);
        }
        const uint32_t off = umma_off(m, 8 * c);
        *reinterpret_cast<uint4 *>(hi_tile + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4 *>(lo_tile + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// G_hi and G_lo of the 16-point DFT in this launch's direction, from the pass's table of w_{n_l}^e
// (w_16^j = w_{n_l}^{j n_l / 16}; 16 divides n_l whenever a radix-16 stage runs).  Row n of the B
// operand is output column n of G: G[k][n] for k in [32].
template <int DIR, int TCK>
__device__ __forceinline__ void umma_build_g(unsigned char *g_hi, unsigned char *g_lo, const float2 *__restrict__ tw,
                                             int nl) {
    const int step = nl >> 4;
    for (int n = threadIdx.x; n < 32; n += blockDim.x) {
        const int kk = n & 15;  // output index
        float col[32];
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const float2 w = dirw<DIR>(tw[((kk * r) & 15) * step]);  // F[kk][r]
            if (n < 16) {        // y_re[kk] = sum_r F_re x_re - F_im x_im
                col[r] = w.x;
                col[16 + r] = -w.y;
            } else {             // y_im[kk] = sum_r F_im x_re + F_re x_im
                col[r] = w.y;
                col[16 + r] = w.x;
            }
        }
        umma_write_row<TCK>(g_hi, g_lo, n, col);
    }
}

// Position of butterfly w of a Stockham stage: input r at base + (b + r per_col) js, output r at
// base + (o + r Ns) js.
struct UmmaBfly {
    int base, js, b, o, k;
};

__device__ __forceinline__ UmmaBfly umma_bfly(const AxisPass &a, int w, int lg_cols, int cols, int Ns, int lg_ns) {
    UmmaBfly p;
    const int col = w & (cols - 1);
    p.b = w >> lg_cols;
    if (a.contiguous) {
        p.base = ((col >> a.lg_Gt) << a.lg_nlt) + (col & (a.Gt - 1));
        p.js = a.Gt;
    } else {
        p.base = col;
        p.js = cols;
    }
    p.k = p.b & (Ns - 1);
    p.o = ((p.b >> lg_ns) << lg_ns) * 16 + p.k;
    return p;
}

// One radix-16 stage of the tile on the tensor cores (see the top of this file).  Every thread of the
// block calls it.
template <int DIR, int TCK>
__device__ __forceinline__ void stockham_stage_umma16(float2 *sm, const float2 *__restrict__ tw, const AxisPass &a,
                                                      int Ns, UmmaCtx &u) {
    const int tid = threadIdx.x, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int G = umma_groups(blockDim.x);
    const int g = nwarps >= 4 ? warp >> 2 : 0;               // this thread's group
    const int gwarps = nwarps >= 4 ? 4 : nwarps;             // warps per group
    const int R = 32 * gwarps;                                // butterflies per group
    const int r = tid - g * R;                                // row within the group
    const int lg_cols = a.lg_Gt + a.lg_V;
    const int cols = 1 << lg_cols;
    const int per_col = a.len >> 4;
    const int total = cols * per_col;
    const int twstep = a.nl / (Ns * 16);
    const int lg_ns = 31 - __clz(Ns);
    const int w = g * R + r;
    const bool active = g < G && w < total;
    unsigned char *tiles = reinterpret_cast<unsigned char *>(__cvta_shared_to_generic(u.a0)) +
                           (size_t)g * 2 * kUmmaTileBytes;
    unsigned char *a_hi = tiles, *a_lo = tiles + kUmmaTileBytes;
    // 1. load and twiddle the butterfly's 16 inputs, scale (float16), split into the A tiles
    float x[32];
    float inv = 1.f;
    UmmaBfly p{};
    if (active) {
        p = umma_bfly(a, w, lg_cols, cols, Ns, lg_ns);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            float2 v = sm[smi(p.base + (p.b + q * per_col) * p.js, a.swz)];
            if (Ns > 1) v = cmul(v, dirw<DIR>(tw[q * p.k * twstep]));
            x[q] = v.x;
            x[16 + q] = v.y;
        }
        if constexpr (TCK == 2) {
            float m = 0.f;
#pragma unroll
            for (int i = 0; i < 32; ++i) m = fmaxf(m, fabsf(x[i]));
            if (m > 0.f) {
                const int ex = (int)((__float_as_uint(m) >> 23) & 0xff) - 127;  // m in [2^ex, 2^(ex+1))
                int es = 127 + 13 - ex, ei = 127 - 13 + ex;
                es = es < 1 ? 1 : (es > 254 ? 254 : es);
                ei = ei < 1 ? 1 : (ei > 254 ? 254 : ei);
                const float sc = __uint_as_float((unsigned)es << 23);
                inv = __uint_as_float((unsigned)ei << 23);
#pragma unroll
                for (int i = 0; i < 32; ++i) x[i] *= sc;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) x[i] = 0.f;
    }
    if (g < G && r < kUmmaRows) umma_write_row<TCK>(a_hi, a_lo, r, x);
    fence_async_shared();  // the generic-proxy stores of the A rows before the tensor cores read them
    __syncthreads();       // every group's A rows written, every thread done with the previous stage
    // 2. one thread per group issues the three products (two K halves each) and commits them
    const uint32_t d = u.tmem + (uint32_t)(32 * g);
    if (g < G && r == 0) {
        tc_fence_after();
        const uint32_t idesc = umma_idesc<TCK>();
        const uint32_t ah = umma_smem_u32(a_hi), al = umma_smem_u32(a_lo);
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // K halves: k in [16 h, 16 h + 16), 256 bytes apart
            umma_f16(d, umma_desc(ah + 256 * h), umma_desc(u.g_hi + 256 * h), idesc, h);
            umma_f16(d, umma_desc(al + 256 * h), umma_desc(u.g_hi + 256 * h), idesc, 1);
            umma_f16(d, umma_desc(ah + 256 * h), umma_desc(u.g_lo + 256 * h), idesc, 1);
        }
        umma_commit(u.bar + g);
    }
    // 3. wait (bounded) for the group's products, read this thread's accumulator row
    if (g < G) {
        if (!umma_bar_try(u.bar + g, u.phase)) {
            const unsigned long long t0 = globaltimer_ns();
            while (!umma_bar_try(u.bar + g, u.phase)) {
                if ((long long)(globaltimer_ns() - t0) > kUmmaWaitNs) {
                    if (u.status) atomicCAS(u.status, 0, (int)FFTU_ERR_TIMEOUT);
                    break;
                }
            }
        }
        tc_fence_after();
    }
    u.phase ^= 1u;
    float y[32];
    // every warp of a group reads its 32 accumulator lanes (warp-collective), lane 32 (warp % 4) + lane id
    if (g < G) {
        tmem_ld32(d + ((uint32_t)(32 * (warp & 3)) << 16), y);
    } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) y[i] = 0.f;
    }
    tc_fence_before();
    __syncthreads();  // every input of the stage read before any output overwrites the tile
    // 4. outputs in Stockham order
    if (active) {
#pragma unroll
        for (int q = 0; q < 16; ++q)
            sm[smi(p.base + (p.o + q * Ns) * p.js, a.swz)] = make_float2(y[q] * inv, y[16 + q] * inv);
    }
    __syncthreads();
}

// Block set-up of the tensor-core stages: G tiles, mbarriers, TMEM allocation (warp 0).  `raw` is the
// 128-byte aligned shared region of umma_smem_bytes(blockDim.x) bytes.
template <int DIR, int TCK>
__device__ __forceinline__ UmmaCtx umma_setup(unsigned char *raw, const float2 *__restrict__ tw, int nl, int *status) {
    UmmaCtx u;
    const int G = umma_groups(blockDim.x);
    unsigned char *g_hi = raw, *g_lo = raw + kUmmaBBytes;
    unsigned char *a0 = raw + 2 * kUmmaBBytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(a0 + 2 * (size_t)kUmmaTileBytes * G);
    uint32_t *slot = reinterpret_cast<uint32_t *>(bar + G);
    umma_build_g<DIR, TCK>(g_hi, g_lo, tw, nl);
    if (threadIdx.x == 0) {
        for (int i = 0; i < G; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(umma_smem_u32(bar + i)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(umma_smem_u32(slot)),
                     "r"(umma_tmem_cols(blockDim.x))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_shared();  // G tiles visible to the tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    u.tmem = *slot;
    u.g_hi = umma_smem_u32(g_hi);
    u.g_lo = umma_smem_u32(g_lo);
    u.a0 = umma_smem_u32(a0);
    u.bar = bar;
    u.status = status;
    u.phase = 0;
    return u;
}

// Block tear-down: free the TMEM columns (warp 0, after every thread's last tcgen05 access).
__device__ __forceinline__ void umma_teardown(const UmmaCtx &u) {
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(u.tmem),
                     "r"(umma_tmem_cols(blockDim.x))
                     : "memory");
    }
}

}  // namespace fftu
