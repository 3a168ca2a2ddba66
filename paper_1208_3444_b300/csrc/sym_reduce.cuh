// sym_reduce.cuh -- the consumer side of the pair-once plans (force_sym.cuh):
// the fixed-order sums of a body's row segments and column slots that the
// step and output epilogues take in place of a segment sum.
#pragma once

#include "force_sym.cuh"

namespace colatus {

// Sum of cnt float4 entries stride apart from p (x, y, z; with the low words
// `lo` float4 further on when COMP, folded as reduce_f32 does), in order,
// B independent loads at a time (the last batch predicated).
template <bool COMP, int B = 8>
__device__ __forceinline__ void sym_sum_run(const float4 *__restrict__ p, long long stride, int cnt, int lo,
                                            float &hx, float &hy, float &hz, float &lx, float &ly, float &lz) {
    for (int s = 0; s < cnt; s += B) {
        float4 h[B], l[B];
#pragma unroll
        for (int k = 0; k < B; ++k) {
            if (s + k < cnt) {
                h[k] = __ldg(p + (s + k) * stride);
                if (COMP) l[k] = __ldg(p + (s + k) * stride + lo);
            }
        }
#pragma unroll
        for (int k = 0; k < B; ++k) {
            if (s + k < cnt) {
                if (COMP) {
                    acc2_add(hx, lx, h[k].x);
                    acc2_add(hy, ly, h[k].y);
                    acc2_add(hz, lz, h[k].z);
                    lx += l[k].x;
                    ly += l[k].y;
                    lz += l[k].z;
                } else {
                    hx += h[k].x;
                    hy += h[k].y;
                    hz += h[k].z;
                }
            }
        }
    }
}

// Epilogue side: the force on body i (FP32 partial sums of a symmetric plan),
// its row segments then the column slots on its tile, in that fixed order,
// B loads at a time; COMP adds the low words separately, as reduce_f32 does.
template <bool COMP, int B>
__device__ __forceinline__ float3 reduce_sym_f32(const float4 *__restrict__ part, const ForceLaunch &L,
                                                 int T, long long i) {
    const SymTab S(L.sym);
    const long long t = i / T, il = i - t * T;
    const long long step = (COMP ? 2LL : 1LL) * T;
    float hx = 0.f, hy = 0.f, hz = 0.f, lx = 0.f, ly = 0.f, lz = 0.f;
    sym_sum_run<COMP, B>(part + t * L.S_max * step + il, step, S.row_ns[t], T, hx, hy, hz, lx, ly, lz);
    const int k0 = S.col_start[t];
    sym_sum_run<COMP, B>(part + L.col_off + (long long)k0 * step + il, step, S.col_start[t + 1] - k0, T, hx, hy,
                         hz, lx, ly, lz);
    return COMP ? make_float3(hx + lx, hy + ly, hz + lz) : make_float3(hx, hy, hz);
}

}  // namespace colatus
