// Phase A for 3D complex64 arrays: Superstep 0 (local sub-FFTs of shape n/p
// and the twiddle) and the Superstep 1 redistribution of Algorithm 2.3
// (Sec. 2.2), in two stages that each read and write coalesced tiles.
//
// Axes are 0 (slowest), 1, 2 (contiguous); L_l = n_l / p_l.  The sub-FFT
// along axis 1 is split by the radix split of Sec. 2.1.1 (eq. radix) as
// L_1 = A * B, m_1 = a + A b:
//     Y[c + B e] = sum_a w_A^{a e} [ w_{L_1}^{a c} sum_b X[a + A b] w_B^{b c} ].
//
// Stage 1, task (s0, s1, m0, a): the B rows i0 = s0 + p0 m0,
//   i1 = s1 + p1 (a + A b), b in [B], read from HBM.
//   * each row: F_{L_2} on every residue class s2 (i2 = s2 + p2 j), as
//     L_2 = R1 * R2 (first radix-R1 stage straight from HBM in registers,
//     shared exchange, radix-R2 stage), twiddle w_{n_2}^{k2 s2} and the Put
//     position i2' = k2 + L_2 s2 (Superstep 1 along axis 2);
//   * across the B rows: F_B over b and w_{L_1}^{a c}.
//   The result T[c][i2'] goes to a scratch block laid out
//   [c][i2' / W][m0][a][i2' % W], so that each stage-2 tile is contiguous.
// Stage 2, task (s0, s1, c, chunk): the L_0 x A x W tile of T.
//   * F_A over a, k1 = c + B e, twiddle w_{n_1}^{k1 s1};
//   * F_{L_0} over m0 (L_0 = Q1 * Q2, two radix stages with one shared
//     exchange), twiddle w_{n_0}^{k0 s0};
//   * store at the Put position (k0 + L_0 s0, k1 + L_1 s1, i2') in HBM.
// The twiddles of the three axes multiply to prod_l w_{n_l}^{k_l s_l}
// (Algorithm 2.3, Superstep 0), and the three Put maps compose to the
// Superstep 1 map m + s (n/p).
//
// Scheduling: either two kernels through a workspace of N elements
// (stage 1 over all tasks, then stage 2), or one persistent kernel that walks
// the units (s0, s1) in order, interleaving stage 1 of unit u + 1 with stage
// 2 of unit u through a small ring of scratch slots meant to stay in L2; a
// unit's stage-2 tasks wait for its stage-1 completion counter, and a slot is
// reused only after the stage-2 tasks that read it have finished.  Waits are
// bounded: a wait that expires sets the plan's status word to FFTU_ERR_TIMEOUT
// and the task is skipped (the output is then invalid and the host reports it).
#include <cuda_runtime.h>

#include "fft_device.cuh"
#include "fftu_internal.h"

namespace fftu {

namespace {

template <int N2_, int P2_, int R1_, int B_, int A_, int L0_, int Q1_, int W_, int MINB_, int NS_, bool PP_,
          bool GT_ = false, int NT_ = 256>
struct Cfg {
    static constexpr int N2 = N2_, P2 = P2_, L2 = N2 / P2, R1 = R1_, R2 = L2 / R1;
    static constexpr int B = B_, A = A_, L1 = A * B;
    static constexpr int L0 = L0_, Q1 = Q1_, Q2 = L0 / Q1;
    static constexpr int W = W_, NCH = N2 / W;
    static constexpr int NT = NT_;              // consumer threads (plus one producer warp)
    static constexpr int MINB = MINB_;          // resident CTAs per SM the register budget targets
    static constexpr int TILE1 = B * N2;        // stage-1 elements
    static constexpr int TILE2 = L0 * A * W;    // stage-2 elements
    static constexpr int TILE = TILE1 > TILE2 ? TILE1 : TILE2;
    static constexpr int UNIT = L0 * L1 * N2;   // elements of one residue unit (s0, s1)
    static constexpr int S1_TASKS = L0 * A;     // stage-1 tasks per unit
    static constexpr int S2_TASKS = B * NCH;    // stage-2 tasks per unit
    // shared swizzle widths (8-byte words per 128-byte wavefront = 16)
    static constexpr int SW1 = (16 / P2) < R2 ? (16 / P2) : R2;
    static constexpr int SW2 = (16 / W) < Q2 ? (16 / W) : Q2;
    static constexpr int SWA = ((16 / W) < A ? (16 / W) : A) - 1;  // scratch row swizzle mask
    static constexpr int NS = NS_;               // shared input buffers (pipeline depth)
    static constexpr bool PINGPONG = PP_;        // passes alternate with a work buffer (else in place)
    static constexpr bool GLOBAL_T = GT_;        // the broadcast twiddles (t1, te) stay in global memory
};

// Run-time geometry shared by every task.
struct Geo {
    const float2 *in;
    float2 *out;
    float2 *scratch;       // workspace (two-kernel mode: N elements; ring mode: ring slots)
    const float2 *tw0, *tw1, *tw2;  // w_{n_l}^e tables
    int *status;
    unsigned *counters;    // ring mode: [0] task counter, [1..U] stage-1 done, [U+1..2U] stage-2 done
    int P0, P1;            // p_0, p_1
    int n0, n1;            // n_0 = P0 L0, n1 = P1 L1
    int units;             // P0 * P1
    int ring;              // ring slots (ring mode)
    int lag;               // ring mode: stage 2 of unit u runs after stage 1 of unit u + lag (lag < ring)
    long long spin_limit;  // bounded-wait budget in nanoseconds
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int DIR> __device__ __forceinline__ float2 tw_at(const float2 *t, int e) { return dirw<DIR>(t[e]); }

// Per-CTA twiddle tables in shared memory, already conjugated for the inverse
// and laid out so that the lanes of a warp read consecutive entries (or one
// broadcast entry) in every pass.
struct Tabs {
    float4 *tb;  // [k2][s2 / 2]: (w_{n2}^{k2 s2}, w_{n2}^{k2 (s2 + 1)})        stage 1b
    float2 *ta;  // [u][q]: w_{L2}^{q u}                                         stage 1a
    float2 *td;  // [u'][q']: w_{L0}^{q' u'}                                     stage 2b
    float2 *t1;  // [e]: w_{n1}^e (read as a broadcast)                          stages 1c, 2a
    float2 *te;  // [s0][k0]: w_{n0}^{k0 s0}                                     stage 2c
    float2 *tile;
};

template <class K>
__host__ __device__ constexpr size_t table_elems(int n0, int n1) {
    return (size_t)K::L2 * K::P2 + K::R1 * K::R2 + K::Q1 * K::Q2 + (K::GLOBAL_T ? 0 : n1 + n0);
}

template <class K, int DIR>
__device__ __forceinline__ Tabs build_tables(const Geo &g, unsigned char *raw) {
    Tabs T;
    T.tile = nullptr;
    T.tb = reinterpret_cast<float4 *>(raw);
    T.ta = reinterpret_cast<float2 *>(T.tb + K::L2 * K::P2 / 2);
    T.td = T.ta + K::R1 * K::R2;
    T.t1 = T.td + K::Q1 * K::Q2;
    T.te = T.t1 + (K::GLOBAL_T ? 0 : g.n1);
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < K::L2 * K::P2 / 2; i += nt) {
        const int k2 = i / (K::P2 / 2), s2 = 2 * (i % (K::P2 / 2));
        const float2 w0 = tw_at<DIR>(g.tw2, k2 * s2), w1 = tw_at<DIR>(g.tw2, k2 * (s2 + 1));
        T.tb[i] = make_float4(w0.x, w0.y, w1.x, w1.y);
    }
    for (int i = tid; i < K::R1 * K::R2; i += nt)
        T.ta[i] = tw_at<DIR>(g.tw2, ((i % K::R2) * (i / K::R2) * K::P2) & (K::N2 - 1));
    for (int i = tid; i < K::Q1 * K::Q2; i += nt)
        T.td[i] = tw_at<DIR>(g.tw0, ((i % K::Q2) * (i / K::Q2) * g.P0) & (g.n0 - 1));
    if (!K::GLOBAL_T)
        for (int i = tid; i < g.n1; i += nt) T.t1[i] = tw_at<DIR>(g.tw1, i);
    for (int i = tid; i < (K::GLOBAL_T ? 0 : g.n0); i += nt) {
        const int s0 = i / K::L0, k0 = i % K::L0;
        T.te[i] = tw_at<DIR>(g.tw0, (k0 * s0) & (g.n0 - 1));
    }
    __syncthreads();
    return T;
}

// The broadcast-style twiddles: w_{n1}^e (all lanes read one entry) and w_{n0}^{k0 s0} (lanes read
// consecutive k0), from shared memory or, with GLOBAL_T, through the read-only L1 path.
template <class K, int DIR>
__device__ __forceinline__ float2 t1_at(const Geo &g, const Tabs &T, int e) {
    if constexpr (K::GLOBAL_T) return dirw<DIR>(__ldg(g.tw1 + e));
    return T.t1[e];
}
template <class K, int DIR>
__device__ __forceinline__ float2 te_at(const Geo &g, const Tabs &T, int s0, int k0) {
    if constexpr (K::GLOBAL_T) return dirw<DIR>(__ldg(g.tw0 + ((k0 * s0) & (g.n0 - 1))));
    return T.te[s0 * K::L0 + k0];
}

// Scratch stores of the ring keep their lines in L2 (evict-last policy); the
// stage-2 reader discards them after use so dead lines are never written back.
__device__ __forceinline__ unsigned long long l2_keep_policy() {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void st_keep(float2 *p, float2 a, float2 b, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(a.x), "f"(a.y),
                 "f"(b.x), "f"(b.y), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void discard_l2_line(const void *p) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

// Two adjacent complex64 values moved as one 16-byte access.
struct Pair {
    float2 a, b;
};
__device__ __forceinline__ Pair unpack(float4 v) { return {make_float2(v.x, v.y), make_float2(v.z, v.w)}; }
__device__ __forceinline__ float4 pack(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
__device__ __forceinline__ Pair ld_sh(const float2 *p) { return unpack(*reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ void st_sh(float2 *p, float2 a, float2 b) { *reinterpret_cast<float4 *>(p) = pack(a, b); }
__device__ __forceinline__ void st_stream(float2 *p, float2 a, float2 b) {
    __stcs(reinterpret_cast<float4 *>(p), pack(a, b));
}
__device__ __forceinline__ void st_l2(float2 *p, float2 a, float2 b) { *reinterpret_cast<float4 *>(p) = pack(a, b); }

// ---- pipeline primitives: mbarriers and bulk copies ----------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity; false when the budget runs out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, long long limit_ns) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try(bar, parity))
        if ((long long)(global_ns() - t0) > limit_ns) return false;
    return true;
}
// One-dimensional bulk copy global -> shared, completing on an mbarrier.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// The same bulk copy with an L2 eviction-priority hint.
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, unsigned bytes, uint64_t *bar,
                                              unsigned long long pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ unsigned long long l2_first_policy() {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// Order this thread's earlier generic-proxy acquires before its later bulk-copy reads of global memory.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
template <int N> __device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(N) : "memory"); }

// ---- stage 1: compute on a landed tile of B rows ------------------------------------------------
// buf: the B rows of the task, natural order [b][i2] as the bulk copies left them.
// In place, shared layouts after the first exchange:
//   X1[b][u][q'][s2] with q' = q ^ (u mod SW1)        (exchange inside each row FFT)
//   X2[b][i2''] with i2'' = L2 s2 + (k2 ^ sigma(s2))    (Put order, swizzled; sigma is even so
//                                                       pairs of adjacent k2 stay adjacent)
// Output: the scratch block of unit `dst_unit`, element (c, i2', m0, a) at
//   block (c, i2' / W), row m0 * A + (a ^ (m0 & SWA)), column i2' % W
// (the row swizzle makes the stage-2 reads of the landed block conflict-free).
template <class K>
__device__ __forceinline__ int x2_index(int b, int k2, int s2) {
    constexpr int sig = 16 / K::P2 > 1 ? 16 / K::P2 : 2;  // even, so k2 pairs stay adjacent
    const int sw = (s2 * sig) & (K::L2 - 1) & 15;
    return b * K::N2 + K::L2 * s2 + (k2 ^ sw);
}

template <class K, int DIR, bool RING>
__device__ __forceinline__ void stage1_compute(const Geo &g, const Tabs &T, float2 *buf, float2 *work, int m0, int a,
                                               float2 *dst_unit) {
    const int tid = threadIdx.x;
    constexpr int HP2 = K::P2 / 2;
    // S1a (buf -> X1): items (b, s2 pair, q); inputs j = q + R2 r -> i2 = s2 + P2 q + (N2 / R1) r;
    // F_{R1} over r -> u; twiddle w_{L2}^{q u}.  X1 goes to `work` (ping-pong) or back into `buf`.
    float2 *x1 = K::PINGPONG ? work : buf;
    constexpr int IA = K::B * HP2 * K::R2;
    constexpr int NA = (IA + K::NT - 1) / K::NT;
    {
        float2 ha[NA][K::R1], hb[NA][K::R1];
#pragma unroll
        for (int h = 0; h < NA; ++h) {
            const int it = tid + h * K::NT;
            if (it < IA) {
                const int sp = it % HP2, q = (it / HP2) % K::R2, b = it / (HP2 * K::R2);
#pragma unroll
                for (int r = 0; r < K::R1; ++r) {
                    const Pair pr = ld_sh(buf + b * K::N2 + 2 * sp + K::P2 * q + (K::N2 / K::R1) * r);
                    ha[h][r] = pr.a;
                    hb[h][r] = pr.b;
                }
                dft_small<K::R1, DIR>(ha[h]);
                dft_small<K::R1, DIR>(hb[h]);
            }
            if (K::PINGPONG && it < IA) {
                const int sp = it % HP2, q = (it / HP2) % K::R2, b = it / (HP2 * K::R2);
#pragma unroll
                for (int u = 0; u < K::R1; ++u) {
                    const float2 w = T.ta[u * K::R2 + q];
                    st_sh(x1 + ((b * K::R1 + u) * K::R2 + (q ^ (u % K::SW1))) * K::P2 + 2 * sp, cmul(ha[h][u], w),
                          cmul(hb[h][u], w));
                }
            }
        }
        if (!K::PINGPONG) {
            consumer_sync<K::NT>();
#pragma unroll
            for (int h = 0; h < NA; ++h) {
                const int it = tid + h * K::NT;
                if (it < IA) {
                    const int sp = it % HP2, q = (it / HP2) % K::R2, b = it / (HP2 * K::R2);
#pragma unroll
                    for (int u = 0; u < K::R1; ++u) {
                        const float2 w = T.ta[u * K::R2 + q];
                        st_sh(x1 + ((b * K::R1 + u) * K::R2 + (q ^ (u % K::SW1))) * K::P2 + 2 * sp,
                              cmul(ha[h][u], w), cmul(hb[h][u], w));
                    }
                }
            }
        }
    }
    consumer_sync<K::NT>();
    // S1b (X1 -> buf): items (b, s2 pair, u); F_{R2} over q -> v; k2 = u + R1 v; twiddle w_{n2}^{k2 s2};
    // Put order (X2 layout)
    constexpr int IB = K::B * HP2 * K::R1;
    constexpr int NB = (IB + K::NT - 1) / K::NT;
    {
        float2 ha[NB][K::R2], hb[NB][K::R2];
#pragma unroll
        for (int h = 0; h < NB; ++h) {
            const int it = tid + h * K::NT;
            if (it < IB) {
                const int sp = it % HP2, u = (it / HP2) % K::R1, b = it / (HP2 * K::R1);
#pragma unroll
                for (int q = 0; q < K::R2; ++q) {
                    const Pair pr = ld_sh(x1 + ((b * K::R1 + u) * K::R2 + (q ^ (u % K::SW1))) * K::P2 + 2 * sp);
                    ha[h][q] = pr.a;
                    hb[h][q] = pr.b;
                }
                dft_small<K::R2, DIR>(ha[h]);
                dft_small<K::R2, DIR>(hb[h]);
            }
        }
        if (!K::PINGPONG) consumer_sync<K::NT>();
#pragma unroll
        for (int h = 0; h < NB; ++h) {
            const int it = tid + h * K::NT;
            if (it < IB) {
                const int sp = it % HP2, u = (it / HP2) % K::R1, b = it / (HP2 * K::R1);
                const int s2 = 2 * sp;
#pragma unroll
                for (int vv = 0; vv < K::R2; ++vv) {
                    const int k2 = u + K::R1 * vv;
                    const float4 tt = T.tb[k2 * HP2 + sp];
                    buf[x2_index<K>(b, k2, s2)] = cmul(ha[h][vv], make_float2(tt.x, tt.y));
                    buf[x2_index<K>(b, k2, s2 + 1)] = cmul(hb[h][vv], make_float2(tt.z, tt.w));
                }
            }
        }
    }
    consumer_sync<K::NT>();
    // S1c (buf -> scratch): items (pair of adjacent i2' in Put order); F_B over b -> c; twiddle w_{L1}^{a c}
    constexpr int IC = K::N2 / 2;
    const int arow = m0 * K::A + (a ^ (m0 & K::SWA));
    unsigned long long pol = 0;
    if constexpr (RING) pol = l2_keep_policy();
    for (int it = tid; it < IC; it += K::NT) {
        const int ip = 2 * it;
        const int s2 = ip / K::L2, k2 = ip % K::L2;
        float2 va[K::B], vb[K::B];
#pragma unroll
        for (int b = 0; b < K::B; ++b) {
            const Pair pr = ld_sh(buf + x2_index<K>(b, k2, s2));
            va[b] = pr.a;
            vb[b] = pr.b;
        }
        dft_small<K::B, DIR>(va);
        dft_small<K::B, DIR>(vb);
        float2 *d = dst_unit + (size_t)(ip / K::W) * K::TILE2 + arow * K::W + ip % K::W;
#pragma unroll
        for (int c = 0; c < K::B; ++c) {
            const float2 t = t1_at<K, DIR>(g, T, (a * c * g.P1) & (g.n1 - 1));
            float2 *dc = d + (size_t)c * K::NCH * K::TILE2;
            if constexpr (RING)
                st_keep(dc, cmul(va[c], t), cmul(vb[c], t), pol);
            else
                st_l2(dc, cmul(va[c], t), cmul(vb[c], t));
        }
    }
}

// ---- stage 2: compute on a landed block --------------------------------------------------------
// buf: the L0 x A x W block of one (c, chunk), rows swizzled as stage 1 wrote them.
// In place, shared layouts: Y1[e][m0][w]; Y2[e][u'][q''][w] with q'' = q' ^ (u' mod SW2).
template <class K, int DIR>
__device__ __forceinline__ void stage2_compute(const Geo &g, const Tabs &T, float2 *buf, float2 *work, int s0, int s1,
                                               int c, int chunk) {
    const int tid = threadIdx.x;
    constexpr int HW = K::W / 2;
    // S2a (buf -> Y1): items (m0, w pair); F_A over a -> e; k1 = c + B e; twiddle w_{n1}^{k1 s1}.
    // Y1 goes to `work` (ping-pong) or back into `buf`.
    float2 *y1 = K::PINGPONG ? work : buf;
    constexpr int IA = K::L0 * HW;
    constexpr int NA = (IA + K::NT - 1) / K::NT;
    {
        float2 ha[NA][K::A], hb[NA][K::A];
#pragma unroll
        for (int h = 0; h < NA; ++h) {
            const int it = tid + h * K::NT;
            if (it < IA) {
                const int wp = it % HW, m0 = it / HW;
#pragma unroll
                for (int a = 0; a < K::A; ++a) {
                    const Pair pr = ld_sh(buf + (m0 * K::A + (a ^ (m0 & K::SWA))) * K::W + 2 * wp);
                    ha[h][a] = pr.a;
                    hb[h][a] = pr.b;
                }
                dft_small<K::A, DIR>(ha[h]);
                dft_small<K::A, DIR>(hb[h]);
            }
        }
        if (!K::PINGPONG) consumer_sync<K::NT>();
#pragma unroll
        for (int h = 0; h < NA; ++h) {
            const int it = tid + h * K::NT;
            if (it < IA) {
                const int wp = it % HW, m0 = it / HW;
#pragma unroll
                for (int e = 0; e < K::A; ++e) {
                    const float2 t = t1_at<K, DIR>(g, T, ((c + K::B * e) * s1) & (g.n1 - 1));
                    st_sh(y1 + (e * K::L0 + m0) * K::W + 2 * wp, cmul(ha[h][e], t), cmul(hb[h][e], t));
                }
            }
        }
    }
    consumer_sync<K::NT>();
    // S2b (Y1 -> buf): items (e, q', w pair); m0 = q' + Q2 r; F_{Q1} over r -> u'; twiddle w_{L0}^{q' u'}
    constexpr int IB = K::A * K::Q2 * HW;
    constexpr int NB = (IB + K::NT - 1) / K::NT;
    {
        float2 ha[NB][K::Q1], hb[NB][K::Q1];
#pragma unroll
        for (int h = 0; h < NB; ++h) {
            const int it = tid + h * K::NT;
            if (it < IB) {
                const int wp = it % HW, q = (it / HW) % K::Q2, e = it / (HW * K::Q2);
#pragma unroll
                for (int r = 0; r < K::Q1; ++r) {
                    const Pair pr = ld_sh(y1 + (e * K::L0 + q + K::Q2 * r) * K::W + 2 * wp);
                    ha[h][r] = pr.a;
                    hb[h][r] = pr.b;
                }
                dft_small<K::Q1, DIR>(ha[h]);
                dft_small<K::Q1, DIR>(hb[h]);
            }
        }
        if (!K::PINGPONG) consumer_sync<K::NT>();
#pragma unroll
        for (int h = 0; h < NB; ++h) {
            const int it = tid + h * K::NT;
            if (it < IB) {
                const int wp = it % HW, q = (it / HW) % K::Q2, e = it / (HW * K::Q2);
#pragma unroll
                for (int u = 0; u < K::Q1; ++u) {
                    const float2 t = T.td[u * K::Q2 + q];
                    st_sh(buf + ((e * K::Q1 + u) * K::Q2 + (q ^ (u % K::SW2))) * K::W + 2 * wp, cmul(ha[h][u], t),
                          cmul(hb[h][u], t));
                }
            }
        }
    }
    consumer_sync<K::NT>();
    // S2c (buf -> HBM): items (e, u', w pair); F_{Q2} over q' -> v'; k0 = u' + Q1 v'; twiddle w_{n0}^{k0 s0}
    constexpr int IC = K::A * K::Q1 * HW;
    for (int it = tid; it < IC; it += K::NT) {
        const int wp = it % HW, u = (it / HW) % K::Q1, e = it / (HW * K::Q1);
        float2 va[K::Q2], vb[K::Q2];
#pragma unroll
        for (int q = 0; q < K::Q2; ++q) {
            const Pair pr = ld_sh(buf + ((e * K::Q1 + u) * K::Q2 + (q ^ (u % K::SW2))) * K::W + 2 * wp);
            va[q] = pr.a;
            vb[q] = pr.b;
        }
        dft_small<K::Q2, DIR>(va);
        dft_small<K::Q2, DIR>(vb);
        float2 *dst = g.out + ((size_t)(c + K::B * e + K::L1 * s1) * K::N2 + (size_t)chunk * K::W + 2 * wp);
#pragma unroll
        for (int vv = 0; vv < K::Q2; ++vv) {
            const int k0 = u + K::Q1 * vv;
            const float2 t = te_at<K, DIR>(g, T, s0, k0);
            st_stream(dst + (size_t)(k0 + K::L0 * s0) * g.n1 * K::N2, cmul(va[vv], t), cmul(vb[vv], t));
        }
    }
}

// ---- the pipelined kernel --------------------------------------------------------------------------
// MODE 0: stage 1 of every task (two-kernel schedule, scratch = workspace of N elements)
// MODE 1: stage 2 of every task (two-kernel schedule)
// MODE 2: persistent ring, task order S1(0), S1(1), S2(0), S1(2), S2(1), ..., S2(U-1)
//
// Warp roles: NT consumer threads compute; one producer warp (lane 0) takes tasks, waits for their
// dependencies (ring), and lands each task's input in one of NS shared buffers with bulk copies
// (B rows of N2 elements for stage 1, one contiguous block for stage 2), completing the buffer's
// `full` mbarrier.  Consumers release a buffer through its `empty` mbarrier.
// Ring order: group j = S1(j) (if j < U) followed by S2(j - lag) (if j >= lag), j = 0 .. U + lag - 1.
template <class K>
__device__ __forceinline__ void decode_task(int t, int U, int mode, int lag, int &unit, int &lt, int &is_s1) {
    constexpr int S1 = K::S1_TASKS, S2 = K::S2_TASKS;
    if (mode == 0) {
        unit = t / S1;
        lt = t % S1;
        is_s1 = 1;
    } else if (mode == 1) {
        unit = t / S2;
        lt = t % S2;
        is_s1 = 0;
    } else if (t < lag * S1) {  // groups 0 .. lag-1: stage 1 only
        unit = t / S1;
        lt = t % S1;
        is_s1 = 1;
    } else if (t < lag * S1 + (U - lag) * (S1 + S2)) {  // groups lag .. U-1: both
        const int r = t - lag * S1;
        const int j = r / (S1 + S2) + lag, o = r % (S1 + S2);
        if (o < S1) {
            unit = j;
            lt = o;
            is_s1 = 1;
        } else {
            unit = j - lag;
            lt = o - S1;
            is_s1 = 0;
        }
    } else {  // groups U .. U+lag-1: stage 2 only
        const int r = t - lag * S1 - (U - lag) * (S1 + S2);
        unit = U - lag + r / S2;
        lt = r % S2;
        is_s1 = 0;
    }
}

template <class K>
__host__ __device__ constexpr size_t pipe_smem_bytes(int n0, int n1) {
    return (size_t)(K::NS + (K::PINGPONG ? 1 : 0)) * K::TILE * sizeof(float2) + table_elems<K>(n0, n1) * sizeof(float2) +
           2 * K::NS * sizeof(uint64_t) + K::NS * sizeof(int) + 16;
}

template <class K, int DIR, int MODE>
__global__ void __launch_bounds__(K::NT + 32, K::MINB) pipe_kernel(const __grid_constant__ Geo g) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2 *bufs = reinterpret_cast<float2 *>(smem_raw);
    float2 *work = bufs + (size_t)K::NS * K::TILE;  // ping-pong partner of the landed buffer
    const Tabs T =
        build_tables<K, DIR>(g, smem_raw + (size_t)(K::NS + (K::PINGPONG ? 1 : 0)) * K::TILE * sizeof(float2));
    uint64_t *full = reinterpret_cast<uint64_t *>(
        (reinterpret_cast<uintptr_t>(T.te + (K::GLOBAL_T ? 0 : g.n0)) + 7) & ~static_cast<uintptr_t>(7));
    uint64_t *empty = full + K::NS;
    int *task = reinterpret_cast<int *>(empty + K::NS);
    if (threadIdx.x == 0) {
        for (int s = 0; s < K::NS; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int U = g.units;
    const int total = MODE == 0 ? U * K::S1_TASKS : MODE == 1 ? U * K::S2_TASKS : U * (K::S1_TASKS + K::S2_TASKS);
    unsigned *task_ctr = g.counters;
    unsigned *s1_done = g.counters + 1;
    unsigned *s2_done = g.counters + 1 + U;

    if (threadIdx.x >= K::NT) {
        // ---------------- producer ----------------
        // Besides landing inputs, the producer publishes task completion for the ring: once the
        // consumers release a buffer (its `empty` phase completes, which orders every consumer
        // store of that task before it), a gpu-scope fence and a counter increment make the task's
        // output visible to the other CTAs.  Completed tasks are also published while the producer
        // waits on a dependency, so a CTA never waits on its own unpublished work.
        if (threadIdx.x != K::NT) return;
        // pend[s]: task in buffer s not yet published (its consumers may still be running);
        // unpub: released tasks waiting to be published (at most 2 NS entries are ever held).
        int pend_task[K::NS];
        unsigned pend_par[K::NS];
        int unpub[2 * K::NS];
        int n_unpub = 0;
        for (int s = 0; s < K::NS; ++s) {
            pend_task[s] = -1;
            pend_par[s] = 0;
        }
        auto release = [&](int s, bool block) -> bool {  // move a finished buffer's task to unpub
            if (pend_task[s] < 0) return true;
            const bool done =
                block ? mbar_wait(empty + s, pend_par[s], g.spin_limit) : mbar_try(empty + s, pend_par[s]);
            if (!done) return false;
            unpub[n_unpub++] = pend_task[s];
            pend_task[s] = -1;
            return true;
        };
        auto publish = [&]() {
            if (MODE != 2 || n_unpub == 0) {
                n_unpub = 0;
                return;
            }
            __threadfence();
            for (int k = 0; k < n_unpub; ++k) {
                int unit, lt, is_s1;
                decode_task<K>(unpub[k], U, MODE, g.lag, unit, lt, is_s1);
                atomicAdd(is_s1 ? s1_done + unit : s2_done + unit, 1u);
            }
            n_unpub = 0;
        };
        bool abort = false;
        const unsigned long long in_pol = l2_first_policy();
        constexpr bool kPrefetchTask = false;  // claim the next task one step early
        int next_t = MODE == 2 ? (kPrefetchTask ? (int)atomicAdd(task_ctr, 1u) : -1) : (int)blockIdx.x;
        for (int i = 0;; ++i) {
            const int s = i % K::NS;
            const unsigned ph = (unsigned)(i / K::NS) & 1u;
            if (i >= K::NS && !release(s, true)) {  // buffer s free again
                atomicCAS(g.status, 0, (int)FFTU_ERR_TIMEOUT);
                abort = true;
            }
            publish();  // dependents in other CTAs are waiting for it: publish right away
            int t = abort ? total : next_t;
            if (MODE == 2 && !kPrefetchTask && !abort) t = (int)atomicAdd(task_ctr, 1u);
            if (t < total)
                next_t = MODE == 2 ? (kPrefetchTask ? (int)atomicAdd(task_ctr, 1u) : -1)
                                   : (int)blockIdx.x + (i + 1) * (int)gridDim.x;
            if (t >= total) {
                task[s] = -1;
                mbar_arrive(full + s);
                break;
            }
            int unit, lt, is_s1;
            decode_task<K>(t, U, MODE, g.lag, unit, lt, is_s1);
            if (MODE == 2) {
                const unsigned *ctr = nullptr;
                unsigned target = 0;
                if (is_s1 && unit >= g.ring) {
                    ctr = s2_done + (unit - g.ring);
                    target = K::S2_TASKS;
                } else if (!is_s1) {
                    ctr = s1_done + unit;
                    target = K::S1_TASKS;
                }
                if (ctr) {
                    const unsigned long long t0 = global_ns();
                    for (;;) {
                        unsigned v;
                        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
                        if (v >= target) break;
                        // never wait on our own finished but unpublished work
                        for (int o = 0; o < K::NS; ++o) release(o, false);
                        publish();
                        if ((long long)(global_ns() - t0) > g.spin_limit) {
                            atomicCAS(g.status, 0, (int)FFTU_ERR_TIMEOUT);
                            abort = true;
                            break;
                        }
                        __nanosleep(32);
                    }
                    if (abort) {
                        task[s] = -1;
                        mbar_arrive(full + s);
                        break;
                    }
                }
                fence_proxy_async_global();
            }
            task[s] = t;
            pend_task[s] = t;
            pend_par[s] = ph;
            float2 *dst = bufs + (size_t)s * K::TILE;
            const int s0 = unit / g.P1, s1 = unit % g.P1;
            if (is_s1) {
                const int m0 = lt / K::A, a = lt % K::A;
                const float2 *plane = g.in + (size_t)(s0 + g.P0 * m0) * g.n1 * K::N2;
                mbar_arrive_tx(full + s, K::B * K::N2 * (unsigned)sizeof(float2));
#pragma unroll 1
                for (int b = 0; b < K::B; ++b) {
                    const float2 *row = plane + (size_t)(s1 + g.P1 * (a + K::A * b)) * K::N2;
                    // with ring units above 16 MiB the ring competes with the input for L2: the input,
                    // read once, goes in with evict-first priority (1024^3 at p = 16 x 16 x 8: phase A
                    // 6.71 against 6.85 ms; no effect at 16 MiB units)
                    if (MODE == 2 && (size_t)K::UNIT * sizeof(float2) > ((size_t)16 << 20))
                        bulk_g2s_hint(dst + b * K::N2, row, K::N2 * (unsigned)sizeof(float2), full + s, in_pol);
                    else
                        bulk_g2s(dst + b * K::N2, row, K::N2 * (unsigned)sizeof(float2), full + s);
                }
            } else {
                const float2 *slot = g.scratch + (size_t)(MODE == 2 ? unit % g.ring : unit) * K::UNIT;
                mbar_arrive_tx(full + s, K::TILE2 * (unsigned)sizeof(float2));
                bulk_g2s(dst, slot + (size_t)lt * K::TILE2, K::TILE2 * (unsigned)sizeof(float2), full + s);
            }
            publish();
        }
        // publish the tasks still in flight (the consumers finish them before seeing the sentinel)
        for (int s = 0; s < K::NS; ++s)
            if (!release(s, true)) atomicCAS(g.status, 0, (int)FFTU_ERR_TIMEOUT);
        publish();
        return;
    }
    // ---------------- consumers ----------------
    for (int i = 0;; ++i) {
        const int s = i % K::NS;
        const unsigned ph = (unsigned)(i / K::NS) & 1u;
        if (!mbar_wait(full + s, ph, g.spin_limit)) {
            if (threadIdx.x == 0) atomicCAS(g.status, 0, (int)FFTU_ERR_TIMEOUT);
            break;
        }
        const int t = task[s];
        if (t < 0) break;
        int unit, lt, is_s1;
        decode_task<K>(t, U, MODE, g.lag, unit, lt, is_s1);
        const int s0 = unit / g.P1, s1 = unit % g.P1;
        float2 *buf = bufs + (size_t)s * K::TILE;
        if (is_s1) {
            float2 *slot = g.scratch + (size_t)(MODE == 2 ? unit % g.ring : unit) * K::UNIT;
            stage1_compute<K, DIR, MODE == 2>(g, T, buf, work, lt / K::A, lt % K::A, slot);
        } else {
            stage2_compute<K, DIR>(g, T, buf, work, s0, s1, lt / K::NCH, lt % K::NCH);
            if (MODE == 2) {
                // the block has been read: drop its L2 lines without write-back
                const float2 *blk = g.scratch + (size_t)(unit % g.ring) * K::UNIT + (size_t)lt * K::TILE2;
                constexpr int LINES = K::TILE2 * (int)sizeof(float2) / 128;
                for (int l = threadIdx.x; l < LINES; l += K::NT)
                    discard_l2_line(reinterpret_cast<const char *>(blk) + 128 * l);
            }
        }
        consumer_sync<K::NT>();
        if (threadIdx.x == 0) mbar_arrive(empty + s);  // releases the buffer; the producer publishes the task
    }
}

// ---- host side --------------------------------------------------------------------------------

template <class K, int DIR>
cudaError_t launch_k(const Phase3Launch &l, cudaStream_t st) {
    Geo g;
    g.in = static_cast<const float2 *>(l.in);
    g.out = static_cast<float2 *>(l.out);
    g.scratch = static_cast<float2 *>(l.scratch);
    g.tw0 = static_cast<const float2 *>(l.tw[0]);
    g.tw1 = static_cast<const float2 *>(l.tw[1]);
    g.tw2 = static_cast<const float2 *>(l.tw[2]);
    g.status = l.status;
    g.counters = l.counters;
    g.P0 = l.p0;
    g.P1 = l.p1;
    g.n0 = l.n0;
    g.n1 = l.n1;
    g.units = l.p0 * l.p1;
    g.ring = l.ring;
    g.lag = l.lag;
    g.spin_limit = l.spin_limit_ns;
    const size_t smem = pipe_smem_bytes<K>(l.n0, l.n1);
    if (l.mode == 0) {
        int grid1 = g.units * K::S1_TASKS, grid2 = g.units * K::S2_TASKS;
        if (grid1 > l.grid1) grid1 = l.grid1;
        if (grid2 > l.grid2) grid2 = l.grid2;
        pipe_kernel<K, DIR, 0><<<grid1, K::NT + 32, smem, st>>>(g);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        pipe_kernel<K, DIR, 1><<<grid2, K::NT + 32, smem, st>>>(g);
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(l.counters, 0, sizeof(unsigned) * (1 + 2 * (size_t)g.units), st);
    if (e != cudaSuccess) return e;
    pipe_kernel<K, DIR, 2><<<l.grid, K::NT + 32, smem, st>>>(g);
    return cudaGetLastError();
}

// Raise the dynamic shared-memory limit, prefer the largest shared carveout,
// and return SMs x resident CTAs per SM for one kernel.
template <typename F>
cudaError_t setup_kernel(F *fn, int nt, size_t smem, int *grid_out) {
    // The limit belongs to the kernel and is shared by every plan that uses it (the table part of
    // the shared memory depends on n_0 and n_1): set the device's opt-in maximum, never one plan's size.
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (smem > (size_t)optin) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nt, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *grid_out = sms * per_sm;
    return cudaSuccess;
}

template <class K, int DIR>
cudaError_t prepare_k(int n0, int n1, int *grids) {
    const size_t smem = pipe_smem_bytes<K>(n0, n1);
    cudaError_t e = setup_kernel(pipe_kernel<K, DIR, 0>, K::NT + 32, smem, &grids[0]);
    if (e == cudaSuccess) e = setup_kernel(pipe_kernel<K, DIR, 1>, K::NT + 32, smem, &grids[1]);
    if (e == cudaSuccess) e = setup_kernel(pipe_kernel<K, DIR, 2>, K::NT + 32, smem, &grids[2]);
    return e;
}

// Instantiated configurations (complex64):
//   512^3, p = 8^3: L = 64, rows 64 = 8 x 8, axis 1 = 8 x 8, axis 0 = 8 x 8, W = 8;
//                   two input buffers and a work buffer, 2 CTAs/SM (measured fastest among
//                   {2, 3} buffers x {in place, ping-pong} x {2, 3} CTAs/SM)
//   512^3, p = 4^3: L = 128, rows 128 = 8 x 16, axis 1 = 16 x 8, axis 0 = 8 x 16, W = 4;
//                   two input buffers and a work buffer, 1 CTA/SM
//   1024^3, p = 8^3: L = 128, rows 128 = 8 x 16, axis 1 = 8 x 16, axis 0 = 8 x 16, W = 4;
//                   64 KB tiles, 512 consumer threads, 1 CTA/SM (residue units of 128 MiB: two kernels)
//   1024^3, p = 16^3: L = 64, rows 64 = 8 x 8, axis 1 = 8 x 8, axis 0 = 8 x 8, W = 16; 64 KB tiles,
//                   512 consumer threads, 1 CTA/SM; residue units of 32 MiB, so the ring (3 units)
//                   is meant to stay in L2
//   1024^3, p = 16 x 16 x 8: rows 128 = 8 x 16, axis 1 = 8 x 8, axis 0 = 8 x 8, W = 16; 32 MiB
//                   residue units as for p = 16^3, with the 16 x 16 x 8 phase B (runs of 8)
using K512p8 = Cfg<512, 8, 8, 8, 8, 64, 8, 8, 2, 2, true, false>;
using K512p4 = Cfg<512, 4, 8, 8, 16, 128, 8, 4, 1, 2, true>;
using K1024p8 = Cfg<1024, 8, 8, 8, 16, 128, 8, 4, 1, 2, true, true, 512>;
using K1024p16 = Cfg<1024, 16, 8, 8, 8, 64, 8, 16, 1, 2, true, true, 512>;
using K1024p16x8 = Cfg<1024, 8, 8, 8, 8, 64, 8, 16, 1, 2, true, true, 512>;

// dispatch() below handles exactly the configurations 0 .. kPhaseA3Configs - 1.
static_assert(kPhaseA3Configs == 5, "phase_a3_select / dispatch and kPhaseA3Configs disagree");

template <int DIR, bool PREP>
cudaError_t dispatch(int which, const Phase3Launch *l, cudaStream_t st, int n0, int n1, int *grid, size_t *smem) {
    switch (which) {
        case 0:
            if (smem) *smem = pipe_smem_bytes<K512p8>(n0, n1);
            return PREP ? prepare_k<K512p8, DIR>(n0, n1, grid) : launch_k<K512p8, DIR>(*l, st);
        case 1:
            if (smem) *smem = pipe_smem_bytes<K512p4>(n0, n1);
            return PREP ? prepare_k<K512p4, DIR>(n0, n1, grid) : launch_k<K512p4, DIR>(*l, st);
        case 2:
            if (smem) *smem = pipe_smem_bytes<K1024p8>(n0, n1);
            return PREP ? prepare_k<K1024p8, DIR>(n0, n1, grid) : launch_k<K1024p8, DIR>(*l, st);
        case 3:
            if (smem) *smem = pipe_smem_bytes<K1024p16>(n0, n1);
            return PREP ? prepare_k<K1024p16, DIR>(n0, n1, grid) : launch_k<K1024p16, DIR>(*l, st);
        case 4:
            if (smem) *smem = pipe_smem_bytes<K1024p16x8>(n0, n1);
            return PREP ? prepare_k<K1024p16x8, DIR>(n0, n1, grid) : launch_k<K1024p16x8, DIR>(*l, st);
    }
    return cudaErrorInvalidValue;
}

template <class K>
bool matches(const int64_t *n, const int64_t *p) {
    return n[2] == K::N2 && p[2] == K::P2 && n[1] / p[1] == K::L1 && n[0] / p[0] == K::L0;
}

template <class K>
void fill(Phase3Info &info) {
    info.unit_elems = K::UNIT;
    info.s1_tasks = K::S1_TASKS;
    info.s2_tasks = K::S2_TASKS;
}

}  // namespace

int phase_a3_select(int d, const int64_t *n, const int64_t *p, int is_double, Phase3Info *info) {
    if (d != 3 || is_double) return -1;
    if (n[0] > (1 << 20) || n[1] > (1 << 20)) return -1;
    if (matches<K512p8>(n, p)) {
        fill<K512p8>(*info);
        return 0;
    }
    if (matches<K512p4>(n, p)) {
        fill<K512p4>(*info);
        return 1;
    }
    if (matches<K1024p8>(n, p)) {
        fill<K1024p8>(*info);
        return 2;
    }
    if (matches<K1024p16>(n, p)) {
        fill<K1024p16>(*info);
        return 3;
    }
    if (matches<K1024p16x8>(n, p)) {
        fill<K1024p16x8>(*info);
        return 4;
    }
    return -1;
}

cudaError_t prepare_phase_a3(int which, int dir, int n0, int n1, int *grid, size_t *smem) {
    return dir < 0 ? dispatch<-1, true>(which, nullptr, 0, n0, n1, grid, smem)
                   : dispatch<1, true>(which, nullptr, 0, n0, n1, grid, smem);
}

cudaError_t launch_phase_a3(const Phase3Launch &l, cudaStream_t st) {
    return l.dir < 0 ? dispatch<-1, false>(l.which, &l, st, l.n0, l.n1, nullptr, nullptr)
                     : dispatch<1, false>(l.which, &l, st, l.n0, l.n1, nullptr, nullptr);
}

}  // namespace fftu
