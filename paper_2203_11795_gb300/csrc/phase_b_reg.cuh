// Register-resident form of the generic fused phase B (complex64): the tile's axes are grouped from the last
// one down into groups of at most 16 values (two adjacent axes where p_l p_{l-1} <= 16); each group is one
// stage in which a thread holds one fiber (all values of the group's axes for fixed other tile indices):
// the first stage loads its fibers from HBM, the last one stores them, the others go through shared memory.
#pragma once

#include "fft_device.cuh"
#include "fftu_internal.h"
#include "generic_tiles.cuh"

namespace fftu {

struct PBGroups {
    int n;
    int off[FFTU_MAX_DIMS], lo[FFTU_MAX_DIMS], hi[FFTU_MAX_DIMS];
    int64_t lst_lo[FFTU_MAX_DIMS], lst_hi[FFTU_MAX_DIMS];
};

template <int DIR, int LO, int HI>
__device__ __forceinline__ void pb_stage(const PhaseBFused &b, const PBGroups &g, int gi, int64_t base, float2 *sm,
                                         float2 *__restrict__ data, bool first, bool last, float scale) {
    constexpr int PG = LO * HI;
    constexpr int LG = PG == 2 ? 1 : PG == 4 ? 2 : PG == 8 ? 3 : 4;
    const int off = g.off[gi];
    const int fibers = (b.P * b.Mt) >> LG;
    const int64_t slo = g.lst_lo[gi], shi = g.lst_hi[gi];
    for (int phi = threadIdx.x; phi < fibers; phi += blockDim.x) {
        const int e0 = ((phi >> off) << (off + LG)) | (phi & ((1 << off) - 1));
        float2 v[PG];
        int64_t go = 0;
        if (first || last) go = base + phaseb_offset(b, e0);
        if (first) {
#pragma unroll
            for (int j = 0; j < PG; ++j) v[j] = data[go + (j % LO) * slo + (j / LO) * shi];
        } else {
#pragma unroll
            for (int j = 0; j < PG; ++j) v[j] = sm[e0 + (j << off)];
        }
        if constexpr (LO > 1) {
#pragma unroll
            for (int jh = 0; jh < HI; ++jh) dft_small<LO, DIR>(v + jh * LO);
        }
        if constexpr (HI > 1) {
#pragma unroll
            for (int jl = 0; jl < LO; ++jl) {
                float2 w[HI];
#pragma unroll
                for (int jh = 0; jh < HI; ++jh) w[jh] = v[jh * LO + jl];
                dft_small<HI, DIR>(w);
#pragma unroll
                for (int jh = 0; jh < HI; ++jh) v[jh * LO + jl] = w[jh];
            }
        }
        if (last) {
#pragma unroll
            for (int j = 0; j < PG; ++j) {
                float2 x = v[j];
                if (scale != 1.f) x = cscale(x, scale);
                data[go + (j % LO) * slo + (j / LO) * shi] = x;
            }
        } else {
#pragma unroll
            for (int j = 0; j < PG; ++j) sm[e0 + (j << off)] = v[j];
        }
    }
}

}  // namespace fftu
