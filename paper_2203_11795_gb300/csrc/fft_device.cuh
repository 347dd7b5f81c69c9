// Device building blocks: complex arithmetic and small DFT butterflies.
//
// A butterfly of radix R computes y_t = sum_q x_q w_R^{q t} in registers, with
// w_R = exp(DIR * 2 pi i / R) and DIR = -1 (forward) or +1 (inverse), i.e. the
// 1D DFT of Sec. 1 (eq. dft) at R points.  Radix 8 and 16 are built from the
// radix split of Sec. 2.1.1 (eq. radix): F_R from two or four smaller DFTs and
// the weights w_R^{q k}.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fftu {

template <typename C> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

template <typename C> __device__ __forceinline__ C mk(typename real_of<C>::type re,
                                                      typename real_of<C>::type im) {
    C c;
    c.x = re;
    c.y = im;
    return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cscale(C a, typename real_of<C>::type s) {
    return mk<C>(a.x * s, a.y * s);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
// a * (DIR * i): the quarter-turn w_4 = -i (forward) or +i (inverse).
template <int DIR, typename C> __device__ __forceinline__ C mul_w4(C a) {
    return DIR < 0 ? mk<C>(a.y, -a.x) : mk<C>(-a.y, a.x);
}
// Table entries hold the forward root w_n^e = exp(-2 pi i e / n); the inverse
// conjugates them.
template <int DIR, typename C> __device__ __forceinline__ C dirw(C w) { return DIR < 0 ? w : cconj(w); }

template <int DIR, typename C> __device__ __forceinline__ void bfly2(C &a, C &b) {
    C t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <int DIR, typename C> __device__ __forceinline__ void bfly4(C &x0, C &x1, C &x2, C &x3) {
    C a = cadd(x0, x2), b = csub(x0, x2);
    C c = cadd(x1, x3), d = mul_w4<DIR>(csub(x1, x3));
    x0 = cadd(a, c);
    x2 = csub(a, c);
    x1 = cadd(b, d);
    x3 = csub(b, d);
}

// In-place radix-8 DFT on v[0..7] (natural order in and out).
template <int DIR, typename C> __device__ __forceinline__ void dft8(C *v) {
    using R = typename real_of<C>::type;
    const R h = R(0.70710678118654752440);
    // even and odd halves
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    bfly4<DIR>(e0, e1, e2, e3);
    bfly4<DIR>(o0, o1, o2, o3);
    // o_k *= w_8^k
    o1 = mk<C>(h * (o1.x - DIR * o1.y), h * (o1.y + DIR * o1.x));   // (1 + DIR i)/sqrt2
    o2 = mul_w4<DIR>(o2);
    o3 = mk<C>(h * (-o3.x - DIR * o3.y), h * (-o3.y + DIR * o3.x)); // (-1 + DIR i)/sqrt2
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}

template <int DIR, typename C> __device__ __forceinline__ void dft4(C *v) { bfly4<DIR>(v[0], v[1], v[2], v[3]); }
template <int DIR, typename C> __device__ __forceinline__ void dft2(C *v) { bfly2<DIR>(v[0], v[1]); }

// Radix 16 as 4 x 4, in place: column DFTs F_4 over x[q + 4j] (q in [4]),
// weights w_16^{q k}, then row DFTs F_4 over q; output k + 4t.
template <int DIR, typename C> __device__ __forceinline__ void dft16(C *v) {
    using R = typename real_of<C>::type;
    const R c1 = R(0.92387953251128675613), s1 = R(0.38268343236508977173);
    const R h = R(0.70710678118654752440);
#pragma unroll
    for (int q = 0; q < 4; ++q) bfly4<DIR>(v[q], v[q + 4], v[q + 8], v[q + 12]);
    // v[q + 4k] now holds column q, frequency k; multiply by w_16^{q k}
    const C w1 = mk<C>(c1, DIR * s1), w2 = mk<C>(h, DIR * h), w3 = mk<C>(s1, DIR * c1);
    const C w6 = mk<C>(-h, DIR * h), w9 = mk<C>(-c1, -DIR * s1);
    v[1 + 4 * 1] = cmul(v[1 + 4 * 1], w1);
    v[1 + 4 * 2] = cmul(v[1 + 4 * 2], w2);
    v[1 + 4 * 3] = cmul(v[1 + 4 * 3], w3);
    v[2 + 4 * 1] = cmul(v[2 + 4 * 1], w2);
    v[2 + 4 * 2] = mul_w4<DIR>(v[2 + 4 * 2]);
    v[2 + 4 * 3] = cmul(v[2 + 4 * 3], w6);
    v[3 + 4 * 1] = cmul(v[3 + 4 * 1], w3);
    v[3 + 4 * 2] = cmul(v[3 + 4 * 2], w6);
    v[3 + 4 * 3] = cmul(v[3 + 4 * 3], w9);
#pragma unroll
    for (int k = 0; k < 4; ++k) bfly4<DIR>(v[0 + 4 * k], v[1 + 4 * k], v[2 + 4 * k], v[3 + 4 * k]);
    // v[t + 4k] holds output k + 4t: transpose the 4 x 4 block (register renaming)
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int t = k + 1; t < 4; ++t) {
            C tmp = v[t + 4 * k];
            v[t + 4 * k] = v[k + 4 * t];
            v[k + 4 * t] = tmp;
        }
}

// Physical shared-memory slot of tile index i of the strided passes: bits 1-3 XORed with bits 4-6 when
// the pass asks for it (swz = 14, contiguous passes; 0: identity).  A bijection on every 16-element group
// that keeps the pairs (2k, 2k + 1) together, so that the class-strided accesses of contiguous lines
// (strides of Gt elements, Gt = 4, 8, 16) spread over all 32 banks instead of piling on 2 to 8 of them.
__device__ __forceinline__ int smi(int i, int swz) { return i ^ ((i >> 3) & swz); }

template <int R, int DIR, typename C> __device__ __forceinline__ void dft_small(C *v) {
    if constexpr (R == 1) {
    } else if constexpr (R == 2) {
        dft2<DIR>(v);
    } else if constexpr (R == 4) {
        dft4<DIR>(v);
    } else if constexpr (R == 8) {
        dft8<DIR>(v);
    } else if constexpr (R == 16) {
        dft16<DIR>(v);
    }
}

}  // namespace fftu
