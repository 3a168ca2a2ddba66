// force.cuh -- the all-pairs softened force of Eq. 1 on sm_103a.
//
//   F_k = sum_{j != k} m_j (x_j - x_k) / (|x_j - x_k|^2 + eps^2)^{3/2}
//
// (attractive orientation; G and a^-3 are applied by the caller).  With
// eps > 0 the self pair contributes exactly zero (x_j - x_k = 0), so no mask
// is needed, as the Appendix A kernel's `idx != i` test intends.
//
// Work decomposition ("stream-K"): the N_pad x N_pad interaction matrix is cut
// into units of (one i-tile of ITILE bodies) x (one j-tile of JT bodies),
// ordered i-major.  A persistent grid of G CTAs (a multiple of the SM count)
// takes contiguous, equal-sized ranges of units, so every SM gets the same
// work whatever N is.  A CTA that covers several j-tiles of one i-tile sums
// them in registers and writes one partial "segment"; the epilogue kernel
// adds the segments of an i-tile in CTA order (fixed order: deterministic).
//
// Pipeline: j-tiles are streamed into shared memory by the bulk-copy engine
// (cp.async.bulk, one elected thread) through STAGES buffers, each completed
// on its own mbarrier; every wait is bounded (FLAG_TIMEOUT, no hang).
//
// FP32 arithmetic: bodies are stored pair-interleaved in HBM,
// [x0 x1 y0 y1 z0 z1 m0 m1] per pair of consecutive bodies, so two j-bodies
// arrive in two 16-byte shared-memory broadcasts as ready-made float2 pairs.
// Each thread holds IPT i-bodies as duplicated float2 pairs and runs the pair
// arithmetic as packed f32x2 FADD/FFMA/FMUL (half the issue slots of scalar
// FP32), with one MUFU.RSQ per interaction: 12 FP32 lane-ops + 1 MUFU per
// interaction, which is the floor for this expression.
//
// Accumulation: the j-sum is blocked.  Each group of FOLD j-pairs is summed
// in an FP32 partial that is then folded into the running total -- plainly
// (COLATUS_FP32) or by TwoSum into a two-float (hi, lo) total
// (COLATUS_FP32_COMP).  The SFU's rsqrt.approx error (~1e-7 relative,
// unbiased to ~2e-8) then dominates: both modes stay within 1e-6 of the FP64
// sum; the compensated one also keeps that at N = 128^3 and beyond.
//
// Equal masses (EQM): when every body has the same mass m, the sum is taken
// as m * sum_j (x_j - x_k)/s^3, which drops one multiply per interaction
// (11 FP32 lane-ops instead of 12).
#pragma once

#include "common.cuh"

namespace colatus {

// ------------------------------------------------------------ stream-K split
// Units [sk_begin(g), sk_begin(g+1)) belong to CTA g; W >= G is required so
// that no CTA is empty.
__host__ __device__ inline long long sk_begin(long long g, long long W, long long G) {
    return (g * W) / G;
}
// The CTA whose range contains unit u: the largest g with sk_begin(g) <= u.
__host__ __device__ inline long long sk_owner(long long u, long long W, long long G) {
    return ((u + 1) * G - 1) / W;
}

struct ForceLaunch {
    long long W;    // units = n_it * n_jt
    int n_it;       // i-tiles
    int n_jt;       // j-tiles
    int S_max;      // max segments any i-tile has
    int G;          // CTAs
    // symmetric plans (force_sym.cuh) only, else null / 0: the plan's tables
    // (device ints) and the float4 offset of the column slots in the
    // segment buffer
    const int *sym;
    long long col_off;
    int fine;       // the symmetric tables are in sub-phases (force_sym.cuh)
};

// ---------------------------------------------------------------- FP32 kernel
template <int NT, int IPT, int JT, int STAGES, int FOLD, bool COMP, bool EQM>
struct F32Kernel {
    static constexpr int ITILE = NT * IPT;
    static constexpr int JPAIRS = JT / 2;
    static constexpr uint32_t TILE_BYTES = JT * 16;  // JT bodies x 16 B
    static constexpr int SMEM = STAGES * TILE_BYTES + STAGES * 8;
    static_assert(JT % 2 == 0 && JPAIRS % FOLD == 0, "FOLD must divide the j-pairs of a tile");
    static_assert(TILE_BYTES % 16 == 0, "bulk copies move multiples of 16 bytes");
};

// Sum one j-tile (JT bodies, pair-interleaved in shared memory) into the
// totals of the IPT i-bodies of this thread.
template <int IPT, int JT, int FOLD, bool COMP, bool EQM, int UNR, int NRCP = 0>
__device__ __forceinline__ void f32_tile(const float4 *__restrict__ t, const float2 (&nx)[IPT],
                                         const float2 (&ny)[IPT], const float2 (&nz)[IPT],
                                         const float2 e2, float (&hx)[IPT], float (&hy)[IPT],
                                         float (&hz)[IPT], float (&lx)[IPT], float (&ly)[IPT],
                                         float (&lz)[IPT]) {
    constexpr int JPAIRS = JT / 2;
#pragma unroll 1
    for (int q0 = 0; q0 < JPAIRS; q0 += FOLD) {
        float2 px[IPT], py[IPT], pz[IPT];
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            px[k] = make_float2(0.f, 0.f);
            py[k] = make_float2(0.f, 0.f);
            pz[k] = make_float2(0.f, 0.f);
        }
#pragma unroll (UNR)
        for (int q = q0; q < q0 + FOLD; ++q) {
            const float4 A = t[2 * q];      // x0 x1 y0 y1
            const float4 B = t[2 * q + 1];  // z0 z1 m0 m1
            const float2 xj = make_float2(A.x, A.y);
            const float2 yj = make_float2(A.z, A.w);
            const float2 zj = make_float2(B.x, B.y);
            const float2 mj = make_float2(B.z, B.w);
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                const float2 dx = __fadd2_rn(xj, nx[k]);
                const float2 dy = __fadd2_rn(yj, ny[k]);
                const float2 dz = __fadd2_rn(zj, nz[k]);
                float2 r2 = __ffma2_rn(dx, dx, e2);
                r2 = __ffma2_rn(dy, dy, r2);
                r2 = __ffma2_rn(dz, dz, r2);
                const float2 inv = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                const float2 inv2 = k < NRCP ? make_float2(rcp_approx(r2.x), rcp_approx(r2.y))
                                             : __fmul2_rn(inv, inv);
                const float2 s = EQM ? __fmul2_rn(inv, inv2) : __fmul2_rn(__fmul2_rn(mj, inv), inv2);
                px[k] = __ffma2_rn(dx, s, px[k]);
                py[k] = __ffma2_rn(dy, s, py[k]);
                pz[k] = __ffma2_rn(dz, s, pz[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            if (COMP) {
                acc2_add(hx[k], lx[k], px[k].x + px[k].y);
                acc2_add(hy[k], ly[k], py[k].x + py[k].y);
                acc2_add(hz[k], lz[k], pz[k].x + pz[k].y);
            } else {
                hx[k] += px[k].x + px[k].y;
                hy[k] += py[k].x + py[k].y;
                hz[k] += pz[k].x + pz[k].y;
            }
        }
    }
}

// Persistent stream-K force kernel, FP32.  pk: pair-interleaved bodies
// (N_pad bodies, N_pad a multiple of ITILE and JT).  part: segments laid out
// [n_it][S_max][COMP ? 2 : 1][ITILE] float4 (x, y, z, 0); for COMP the
// second plane holds the low words.  EQM: segments are scaled by mass_eq.
// UNR: unroll depth of the j-pair loop (a tuning knob).
template <int NT, int IPT, int JT, int STAGES, int FOLD, bool COMP, bool EQM, int MINB, int UNR,
          int NRCP = 0>
__global__ void __launch_bounds__(NT, MINB)
    force_f32_kernel(const float *__restrict__ pk, float4 *__restrict__ part, int *__restrict__ flags,
                     ForceLaunch L, float eps2, float mass_eq) {
    using K = F32Kernel<NT, IPT, JT, STAGES, FOLD, COMP, EQM>;
    extern __shared__ __align__(128) unsigned char smem[];
    float4 *tiles = reinterpret_cast<float4 *>(smem);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * K::TILE_BYTES);

    const int tid = threadIdx.x;
    const long long G = gridDim.x, g = blockIdx.x;
    const long long W = L.W;
    const long long u0 = sk_begin(g, W, G), u1 = sk_begin(g + 1, W, G);
    const int n_jt = L.n_jt;

    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < STAGES && u0 + s < u1; ++s) {
            const long long jt = (u0 + s) % n_jt;
            mbar_arrive_expect_tx(&full[s], K::TILE_BYTES);
            bulk_load(tiles + s * JT, pk + jt * (long long)JT * 4, K::TILE_BYTES, &full[s]);
        }
    }

    const float2 e2 = make_float2(eps2, eps2);
    long long u = u0;
    bool bad = false;
    int stage = 0;
    uint32_t parity = 0;
    while (u < u1) {
        const long long it = u / n_jt;
        const long long uend = min(u1, (it + 1) * (long long)n_jt);
        float2 nx[IPT], ny[IPT], nz[IPT];
        float hx[IPT], hy[IPT], hz[IPT], lx[IPT], ly[IPT], lz[IPT];
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const long long i = it * K::ITILE + tid + k * NT;
            const float *p = pk + (i >> 1) * 8 + (i & 1);
            const float x = __ldg(p), y = __ldg(p + 2), z = __ldg(p + 4);
            nx[k] = make_float2(-x, -x);
            ny[k] = make_float2(-y, -y);
            nz[k] = make_float2(-z, -z);
            hx[k] = hy[k] = hz[k] = 0.f;
            lx[k] = ly[k] = lz[k] = 0.f;
        }
        for (; u < uend; ++u) {
            const bool ok = mbar_wait_bounded(&full[stage], parity);
            if (ok)
                f32_tile<IPT, JT, FOLD, COMP, EQM, UNR, NRCP>(tiles + stage * JT, nx, ny, nz, e2, hx, hy,
                                                         hz, lx, ly, lz);
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
            if (tid == 0 && u + STAGES < u1) {
                const long long jt = (u + STAGES) % n_jt;
                mbar_arrive_expect_tx(&full[stage], K::TILE_BYTES);
                bulk_load(tiles + stage * JT, pk + jt * (long long)JT * 4, K::TILE_BYTES,
                          &full[stage]);
            }
            if (++stage == STAGES) {
                stage = 0;
                parity ^= 1u;
            }
        }
        if (bad) break;
        const long long sidx = g - sk_owner(it * n_jt, W, G);
        float4 *dst = part + (it * L.S_max + sidx) * (COMP ? 2 : 1) * (long long)K::ITILE;
        const float ms = EQM ? mass_eq : 1.f;
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            dst[tid + k * NT] = make_float4(ms * hx[k], ms * hy[k], ms * hz[k], 0.f);
            if (COMP) dst[K::ITILE + tid + k * NT] = make_float4(ms * lx[k], ms * ly[k], ms * lz[k], 0.f);
        }
    }
    if (bad && tid == 0) {
        atomicOr(&flags[FLAG_TIMEOUT], 1);
        // drain the copies still in flight (units u .. u+STAGES-1), bounded
        for (long long v = u; v < u1 && v < u + STAGES; ++v) {
            mbar_wait_bounded(&full[stage], parity);
            if (++stage == STAGES) {
                stage = 0;
                parity ^= 1u;
            }
        }
    }
}

// ---------------------------------------------------------------- FP64 kernel
// Same decomposition and pipeline; bodies are double4 (x, y, z, m), one
// i-body per register set, plain double arithmetic with the library rsqrt.
template <int NT, int IPT, int JT, int STAGES>
struct F64Kernel {
    static constexpr int ITILE = NT * IPT;
    static constexpr uint32_t TILE_BYTES = JT * 32;
    static constexpr int SMEM = STAGES * TILE_BYTES + STAGES * 8;
};

template <int NT, int IPT, int JT, int STAGES>
__global__ void __launch_bounds__(NT)
    force_f64_kernel(const double4 *__restrict__ pos, double4 *__restrict__ part,
                     int *__restrict__ flags, ForceLaunch L, double eps2) {
    using K = F64Kernel<NT, IPT, JT, STAGES>;
    extern __shared__ __align__(128) unsigned char smem[];
    double4 *tiles = reinterpret_cast<double4 *>(smem);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * K::TILE_BYTES);

    const int tid = threadIdx.x;
    const long long G = gridDim.x, g = blockIdx.x;
    const long long W = L.W;
    const long long u0 = sk_begin(g, W, G), u1 = sk_begin(g + 1, W, G);
    const int n_jt = L.n_jt;

    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < STAGES && u0 + s < u1; ++s) {
            const long long jt = (u0 + s) % n_jt;
            mbar_arrive_expect_tx(&full[s], K::TILE_BYTES);
            bulk_load(tiles + s * JT, pos + jt * (long long)JT, K::TILE_BYTES, &full[s]);
        }
    }
    long long u = u0;
    bool bad = false;
    int stage = 0;
    uint32_t parity = 0;
    while (u < u1) {
        const long long it = u / n_jt;
        const long long uend = min(u1, (it + 1) * (long long)n_jt);
        double xi[IPT], yi[IPT], zi[IPT], ax[IPT], ay[IPT], az[IPT];
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const double4 p = pos[it * K::ITILE + tid + k * NT];
            xi[k] = p.x;
            yi[k] = p.y;
            zi[k] = p.z;
            ax[k] = ay[k] = az[k] = 0.0;
        }
        for (; u < uend; ++u) {
            const bool ok = mbar_wait_bounded(&full[stage], parity);
            if (ok) {
                const double4 *t = tiles + stage * JT;
#pragma unroll 4
                for (int j = 0; j < JT; ++j) {
                    const double4 b = t[j];
#pragma unroll
                    for (int k = 0; k < IPT; ++k) {
                        const double dx = b.x - xi[k], dy = b.y - yi[k], dz = b.z - zi[k];
                        const double r2 = dx * dx + dy * dy + dz * dz + eps2;
                        const double inv = rsqrt(r2);
                        const double s = b.w * inv * inv * inv;
                        ax[k] += s * dx;
                        ay[k] += s * dy;
                        az[k] += s * dz;
                    }
                }
            }
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
            if (tid == 0 && u + STAGES < u1) {
                const long long jt = (u + STAGES) % n_jt;
                mbar_arrive_expect_tx(&full[stage], K::TILE_BYTES);
                bulk_load(tiles + stage * JT, pos + jt * (long long)JT, K::TILE_BYTES,
                          &full[stage]);
            }
            if (++stage == STAGES) {
                stage = 0;
                parity ^= 1u;
            }
        }
        if (bad) break;
        const long long sidx = g - sk_owner(it * n_jt, W, G);
        double4 *dst = part + (it * L.S_max + sidx) * (long long)K::ITILE;
#pragma unroll
        for (int k = 0; k < IPT; ++k) dst[tid + k * NT] = make_double4(ax[k], ay[k], az[k], 0.0);
    }
    if (bad && tid == 0) {
        atomicOr(&flags[FLAG_TIMEOUT], 1);
        for (long long v = u; v < u1 && v < u + STAGES; ++v) {
            mbar_wait_bounded(&full[stage], parity);
            if (++stage == STAGES) {
                stage = 0;
                parity ^= 1u;
            }
        }
    }
}

}  // namespace colatus
