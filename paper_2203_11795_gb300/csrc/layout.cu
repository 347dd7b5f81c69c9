// The CYCLIC storage layout: the local arrays X^{(s)} of the virtual processors, concatenated in
// row-major order of s, each local array row-major over its own shape n/p.
//
// Sec. 1.1 distributes a d-dim array cyclically: element x_j goes to processor s with
// s_l = j_l mod p_l, at local index r_l = j_l div p_l.  With processor-major storage that is
// element (s, r) at offset s_lin (N/P) + r_lin.  These kernels move an array between that layout
// and the natural row-major one (one HBM round trip each); the transform itself always runs on
// the natural view.
#include <cuda_runtime.h>

#include "fftu_internal.h"

namespace fftu {

namespace {

// Shifts and masks of the power-of-two shape: per axis log2 n_l and log2 p_l.
struct CyclicMap {
    int d;
    int lg_n[FFTU_MAX_DIMS];
    int lg_p[FFTU_MAX_DIMS];
    int lg_local;  // log2 (N / P): elements per local array
    int64_t N;
};

// Offset of natural element g in the CYCLIC layout.
__device__ __forceinline__ int64_t cyclic_offset(const CyclicMap &m, int64_t g) {
    int64_t s_lin = 0, r_lin = 0;
    int shift = 0;
    int64_t s_parts[FFTU_MAX_DIMS], r_parts[FFTU_MAX_DIMS];
    for (int l = m.d - 1; l >= 0; --l) {  // decompose g into per-axis indices, last axis first
        const int64_t j = (g >> shift) & (((int64_t)1 << m.lg_n[l]) - 1);
        shift += m.lg_n[l];
        s_parts[l] = j & (((int64_t)1 << m.lg_p[l]) - 1);
        r_parts[l] = j >> m.lg_p[l];
    }
    for (int l = 0; l < m.d; ++l) {
        s_lin = (s_lin << m.lg_p[l]) | s_parts[l];
        r_lin = (r_lin << (m.lg_n[l] - m.lg_p[l])) | r_parts[l];
    }
    return (s_lin << m.lg_local) | r_lin;
}

// TO_CYCLIC: dst[cyclic(g)] = src[g]; else dst[g] = src[cyclic(g)].  g runs over the natural order,
// so one side of every access is coalesced.
template <typename C, bool TO_CYCLIC>
__global__ void cyclic_permute_kernel(const C *__restrict__ src, C *__restrict__ dst, const CyclicMap m) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < m.N; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = cyclic_offset(m, g);
        if (TO_CYCLIC)
            dst[c] = src[g];
        else
            dst[g] = src[c];
    }
}

int ilog2_64(int64_t v) {
    int k = 0;
    while (((int64_t)1 << k) < v) ++k;
    return k;
}

}  // namespace

cudaError_t launch_cyclic_permute(const void *src, void *dst, int d, const int64_t *n, const int64_t *p,
                                  int is_double, int to_cyclic, cudaStream_t st) {
    CyclicMap m;
    m.d = d;
    m.N = 1;
    int lg_P = 0;
    for (int l = 0; l < d; ++l) {
        m.lg_n[l] = ilog2_64(n[l]);
        m.lg_p[l] = ilog2_64(p[l]);
        m.N *= n[l];
        lg_P += m.lg_p[l];
    }
    m.lg_local = ilog2_64(m.N) - lg_P;
    int64_t blocks = (m.N + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    const unsigned b = (unsigned)blocks;
    if (is_double) {
        if (to_cyclic)
            cyclic_permute_kernel<double2, true><<<b, 256, 0, st>>>(static_cast<const double2 *>(src),
                                                                    static_cast<double2 *>(dst), m);
        else
            cyclic_permute_kernel<double2, false><<<b, 256, 0, st>>>(static_cast<const double2 *>(src),
                                                                     static_cast<double2 *>(dst), m);
    } else {
        if (to_cyclic)
            cyclic_permute_kernel<float2, true><<<b, 256, 0, st>>>(static_cast<const float2 *>(src),
                                                                   static_cast<float2 *>(dst), m);
        else
            cyclic_permute_kernel<float2, false><<<b, 256, 0, st>>>(static_cast<const float2 *>(src),
                                                                    static_cast<float2 *>(dst), m);
    }
    return cudaGetLastError();
}

}  // namespace fftu
