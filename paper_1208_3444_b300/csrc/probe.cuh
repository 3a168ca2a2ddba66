// probe.cuh -- microbenchmarks of the issue rates the force roofline rests on:
// scalar FFMA, packed FFMA2 (f32x2) and MUFU.RSQ throughput per SM per clock.
//
// Each thread runs K independent dependency chains of one instruction kind,
// so the pipe, not latency, bounds the loop.  The kernel fills every SM with
// `blocks_per_sm` blocks; the host divides the executed lane-operations by
// (SMs x elapsed SM cycles).  The results seed nothing: they are reported
// next to the roofline that assumes 128 FP32 lane-ops and 16 MUFU.RSQ per SM
// per clock.
#pragma once

#include "common.cuh"

namespace colatus {

constexpr int kProbeChains = 8;

// kind 0: FFMA, 1: FFMA2 (two lane-ops each), 2: MUFU.RSQ
template <int KIND>
__global__ void probe_pipe_kernel(int iters, float seed, float *sink, long long *cycles) {
    const long long t0 = clock64();
    if (KIND == 1) {
        float2 a[kProbeChains];
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) a[c] = make_float2(seed + c, seed - c);
        const float2 m = make_float2(0.999f, 0.998f), b = make_float2(1e-3f, 2e-3f);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int c = 0; c < kProbeChains; ++c) a[c] = __ffma2_rn(a[c], m, b);
        }
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) s += a[c].x + a[c].y;
        if (s == 12345.f) sink[threadIdx.x] = s;
    } else {
        float a[kProbeChains];
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) a[c] = seed + c;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int c = 0; c < kProbeChains; ++c) {
                if (KIND == 0)
                    a[c] = fmaf(a[c], 0.999f, 1e-3f);
                else
                    a[c] = rsqrt_approx(a[c] + 1.5f);
            }
        }
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) s += a[c];
        if (s == 12345.f) sink[threadIdx.x] = s;
    }
    const long long t1 = clock64();
    if (threadIdx.x == 0) atomicMax(reinterpret_cast<unsigned long long *>(&cycles[blockIdx.x]),
                                    static_cast<unsigned long long>(t1 - t0));
}

}  // namespace colatus
