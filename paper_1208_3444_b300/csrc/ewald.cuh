// ewald.cuh -- periodic boundaries (Sec. II) by Ewald summation on the
// all-pairs path.
//
// The force on body k in a box of side L is the pull of every image of every
// body with the uniform mean density removed (the k = 0 mode left out), the
// nearest image Plummer-softened with eps:
//
//   F_k = sum_j m_j [ sum_n N(d_j + n L) - N(d_j) + P(d_j) ],
//   d_j = minimum image of x_j - x_k,  N(d) = d/|d|^3,  P(d) = d/(|d|^2+eps^2)^{3/2}.
//
// Ewald's split with parameter alpha turns the image sum into
//   real space:  sum_j m_j d [ (r^2+eps^2)^{-3/2} - erf(alpha r)/r^3
//                              + (2 alpha/sqrt(pi)) exp(-alpha^2 r^2)/r^2 ]
//                over minimum images only (r = |d|; the other images carry
//                erfc(alpha r) with r >= L/2, below the chosen tolerance),
//   k space:     -(4 pi / L^3) sum_{k != 0} exp(-k^2/(4 alpha^2))/k^2 k
//                 [sin(k.x_k) C(k) - cos(k.x_k) S(k)],
//                C + i S = sum_j m_j exp(i k.x_j),  k = 2 pi n / L, |n| <= nk.
//
// The real-space bracket is finite at r -> 0 (its limit is
// -(4/3) alpha^3/sqrt(pi)) but its terms cancel there, so below alpha r = 0.05
// it is taken from its series (2 alpha^3/sqrt(pi)) sum_k (-1)^{k+1} 2 x^{2k} /
// (k! (2k+3)), x = alpha r: two terms in FP32 (the next is 1e-6 of it), four
// in FP64 (4e-13).  The self pair (d = 0) then contributes 0.
//
// Real space reuses the force kernel's decomposition: a persistent stream-K
// grid over (i-tile x j-tile) units, j-tiles staged by bulk copies through
// bounded mbarrier waits, segments in [i-tile][segment][plane][ITILE] float4
// that the step epilogues sum in CTA order.  FP32 arithmetic runs on the
// pair-interleaved bodies as packed f32x2 where the operation allows; erfc is
// Abramowitz & Stegun 7.1.26 (|error| <= 1.5e-7, its exp shared with the
// Gaussian term); FP64 uses the library erfc.
//
// k space: every body's tables exp(2 pi i n x_c/L), n = 0..nk, are computed
// once per force evaluation (ewald_phase_kernel; n x_c/L reduced exactly in
// FP64 before sincospi).  The k-vectors come in pencils of consecutive nz at
// fixed (nx, ny); the x-y phase product is formed once per pencil and body.
// The structure factors are one pass over (k, body) pairs (partial sums per
// body split, added in order), and the force pass evaluates the k-sum at every
// body from its own tables.
#pragma once

#include "common.cuh"
#include "force.cuh"
#include "force_sym.cuh"

namespace colatus {

struct EwaldArgs {
    double L, alpha;
    float Lf, invLf;          // box and 1/box
    float alpha2_log2e;       // alpha^2 log2(e): exp(-alpha^2 r^2) = 2^(-this r^2)
    float alpha_f, cg;        // alpha; 2 alpha / sqrt(pi)
    float p_alpha;            // A&S 7.1.26 p times alpha
    float s0, s1;             // series of the bracket: s0 + s1 r^2 for alpha r < 0.05
    float x2_series;          // (0.05 / alpha)^2: r^2 below which the series is used
    int nk;                   // |n| <= nk in each table
    // derivatives (adjoint and tangent): 2 alpha^2 cg, and the series of minus
    // the bracket's f'(r)/r, -(cs0 + cs1 r^2), for alpha r < 0.05
    float c2ag, ncs0, ncs1;
};

// ---------------------------------------------------------------- FP32 real space
template <int NT, int IPT, int JT, int STAGES, int FOLD, bool COMP>
struct EwaldF32Kernel {
    static constexpr int ITILE = NT * IPT;
    static constexpr int JPAIRS = JT / 2;
    static constexpr uint32_t TILE_BYTES = JT * 16;
    static constexpr int SMEM = STAGES * TILE_BYTES + STAGES * 8;
    static_assert(JPAIRS % FOLD == 0, "FOLD must divide the j-pairs of a tile");
};

// Abramowitz & Stegun 7.1.26 coefficients (Hastings): erfc(x) ~ t P(t) e^{-x^2},
// t = 1 / (1 + p x), x >= 0.
constexpr float kAsP = 0.3275911f;
constexpr float kAsA1 = 0.254829592f, kAsA2 = -0.284496736f, kAsA3 = 1.421413741f,
                kAsA4 = -1.453152027f, kAsA5 = 1.061405429f;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Minimum image of a pair-packed separation on the FMA pipe: fma(d, 1/L, M)
// with M = 1.5 * 2^23 rounds d/L to the nearest integer (ties to even) in
// its single rounding, for |d/L| < 2^22; subtracting M leaves that integer n,
// and d - L n is the minimum image.  (rintf runs on the XU pipe, which the
// pair body already loads with four MUFU results.)
__device__ __forceinline__ float2 min_image2(float2 d, float2 iL, float2 Lm) {
    const float2 magic = make_float2(12582912.f, 12582912.f);
    const float2 n = __fadd2_rn(__ffma2_rn(d, iL, magic), make_float2(-12582912.f, -12582912.f));
    return __ffma2_rn(Lm, n, d);
}

// Real-space bracket times m_j for two j-bodies at once (packed f32x2):
//   m_j [ (r^2+eps^2)^{-3/2} + (1/r^2) (e (q_erfc / r + cg) - 1/r) ],
// e = exp(-alpha^2 r^2), q_erfc = erfc(alpha r) / e from A&S 7.1.26 with
// t = 1 / (1 + p alpha r); 36 FP32 lane-ops and 4 MUFU results per pair
// including the minimum image and the accumulation.  EQM (every body has
// the same mass): the bracket alone, m folded into the segments (35 ops).
template <bool EQM>
__device__ __forceinline__ float2 ewald_pair2(const float2 dx, const float2 dy, const float2 dz,
                                              const float2 mj, const EwaldArgs &A, const float2 e2) {
    float2 r2 = __fmul2_rn(dx, dx);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dz, dz, r2);
    const float2 s2 = __fadd2_rn(r2, e2);
    const float2 ip = make_float2(rsqrt_approx(s2.x), rsqrt_approx(s2.y));
    const float2 ip3 = __fmul2_rn(__fmul2_rn(ip, ip), ip);
    const float2 ir = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
    const float2 pr2 = __fmul2_rn(make_float2(A.p_alpha, A.p_alpha), r2);
    const float2 den = __ffma2_rn(pr2, ir, make_float2(1.f, 1.f));           // 1 + p alpha r
    const float2 t = make_float2(rcp_approx(den.x), rcp_approx(den.y));
    const float2 ea = __fmul2_rn(make_float2(-A.alpha2_log2e, -A.alpha2_log2e), r2);
    const float2 ex = make_float2(ex2_approx(ea.x), ex2_approx(ea.y));       // exp(-alpha^2 r^2)
    float2 poly = __ffma2_rn(make_float2(kAsA5, kAsA5), t, make_float2(kAsA4, kAsA4));
    poly = __ffma2_rn(poly, t, make_float2(kAsA3, kAsA3));
    poly = __ffma2_rn(poly, t, make_float2(kAsA2, kAsA2));
    poly = __ffma2_rn(poly, t, make_float2(kAsA1, kAsA1));
    const float2 qe = __fmul2_rn(poly, t);                                   // erfc(x) / exp(-x^2)
    const float2 q = __ffma2_rn(qe, ir, make_float2(A.cg, A.cg));
    const float2 h = __ffma2_rn(ex, q, make_float2(-ir.x, -ir.y));
    float2 f = __fmul2_rn(h, __fmul2_rn(ir, ir));         // -erf(x)/r^3 + cg e / r^2
    const float2 fs = __ffma2_rn(make_float2(A.s1, A.s1), r2, make_float2(A.s0, A.s0));
    f.x = r2.x < A.x2_series ? fs.x : f.x;
    f.y = r2.y < A.x2_series ? fs.y : f.y;
    const float2 br = __fadd2_rn(ip3, f);
    return EQM ? br : __fmul2_rn(mj, br);
}

// The real-space term as a pair policy of the pair-once kernel
// (force_sym.cuh): the minimum image of the separation, then the mass-free
// bracket of ewald_pair2.  The term is antisymmetric: the minimum image of
// x_k - x_j is exactly minus that of x_j - x_k (the FMA-pipe rounding is odd,
// ties at half a box go to the even integer 0 both ways) and the bracket
// depends on |d| only.  35 FP32 lane-ops and 4 MUFU results per pair with one
// side's accumulation, 38 with both.
struct EwaldPair {
    using Args = EwaldArgs;
    __device__ __forceinline__ static float2 weight(float2 &dx, float2 &dy, float2 &dz, const float2 e2,
                                                    const EwaldArgs &A) {
        const float2 Lm = make_float2(-A.Lf, -A.Lf), iL = make_float2(A.invLf, A.invLf);
        dx = min_image2(dx, iL, Lm);
        dy = min_image2(dy, iL, Lm);
        dz = min_image2(dz, iL, Lm);
        return ewald_pair2<true>(dx, dy, dz, make_float2(0.f, 0.f), A, e2);
    }
};

// pk: the bodies with positions wrapped into [0, L] (ewald_phase_kernel
// writes them), so every separation rounds once from coordinates of the
// box's own size, whatever box the bodies have drifted to.  EQM: every body
// has mass mass_eq (and no zero-mass padding enters): the pair term drops m_j
// and the segments are scaled by mass_eq.
template <int NT, int IPT, int JT, int STAGES, int FOLD, bool COMP, int MINB, bool EQM>
__global__ void __launch_bounds__(NT, MINB)
    ewald_f32_kernel(const float *__restrict__ pk, float4 *__restrict__ part, int *__restrict__ flags,
                     ForceLaunch L, float eps2, EwaldArgs A, float mass_eq) {
    using K = EwaldF32Kernel<NT, IPT, JT, STAGES, FOLD, COMP>;
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
    const float2 Lm = make_float2(-A.Lf, -A.Lf), iL = make_float2(A.invLf, A.invLf);
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
            if (ok) {
                const float4 *t = tiles + stage * JT;
#pragma unroll 1
                for (int q0 = 0; q0 < K::JPAIRS; q0 += FOLD) {
                    float2 px[IPT], py[IPT], pz[IPT];
#pragma unroll
                    for (int k = 0; k < IPT; ++k)
                        px[k] = py[k] = pz[k] = make_float2(0.f, 0.f);
#pragma unroll 2
                    for (int q = q0; q < q0 + FOLD; ++q) {
                        const float4 Aq = t[2 * q], Bq = t[2 * q + 1];
                        const float2 xj = make_float2(Aq.x, Aq.y), yj = make_float2(Aq.z, Aq.w);
                        const float2 zj = make_float2(Bq.x, Bq.y), mj = make_float2(Bq.z, Bq.w);
#pragma unroll
                        for (int k = 0; k < IPT; ++k) {
                            float2 dx = __fadd2_rn(xj, nx[k]);
                            float2 dy = __fadd2_rn(yj, ny[k]);
                            float2 dz = __fadd2_rn(zj, nz[k]);
                            dx = min_image2(dx, iL, Lm);
                            dy = min_image2(dy, iL, Lm);
                            dz = min_image2(dz, iL, Lm);
                            const float2 s = ewald_pair2<EQM>(dx, dy, dz, mj, A, e2);
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
        for (long long v = u; v < u1 && v < u + STAGES; ++v) {
            mbar_wait_bounded(&full[stage], parity);
            if (++stage == STAGES) {
                stage = 0;
                parity ^= 1u;
            }
        }
    }
}

// ---------------------------------------------------------------- FP64 real space
template <int NT, int JT, int STAGES>
struct EwaldF64Kernel {
    static constexpr int ITILE = NT;
    static constexpr uint32_t TILE_BYTES = JT * 32;
    static constexpr int SMEM = STAGES * TILE_BYTES + STAGES * 8;
};

template <int NT, int JT, int STAGES>
__global__ void __launch_bounds__(NT)
    ewald_f64_kernel(const double4 *__restrict__ pos, double4 *__restrict__ part,
                     int *__restrict__ flags, ForceLaunch L, double eps2, EwaldArgs A) {
    using K = EwaldF64Kernel<NT, JT, STAGES>;
    extern __shared__ __align__(128) unsigned char smem[];
    double4 *tiles = reinterpret_cast<double4 *>(smem);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * K::TILE_BYTES);

    const int tid = threadIdx.x;
    const long long G = gridDim.x, g = blockIdx.x;
    const long long W = L.W;
    const long long u0 = sk_begin(g, W, G), u1 = sk_begin(g + 1, W, G);
    const int n_jt = L.n_jt;
    const double Lb = A.L, invL = 1.0 / A.L, al = A.alpha, al2 = A.alpha * A.alpha;
    const double cg = 2.0 * A.alpha * rsqrt(acos(-1.0));
    const double x2s = (0.05 / A.alpha) * (0.05 / A.alpha);
    // series of the bracket to (alpha r)^6: relative error 4e-13 at alpha r = 0.05
    const double sc = 2.0 * al * al2 * rsqrt(acos(-1.0));

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
        const double4 pi = pos[it * K::ITILE + tid];
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (; u < uend; ++u) {
            const bool ok = mbar_wait_bounded(&full[stage], parity);
            if (ok) {
                const double4 *t = tiles + stage * JT;
#pragma unroll 2
                for (int j = 0; j < JT; ++j) {
                    const double4 b = t[j];
                    double dx = b.x - pi.x, dy = b.y - pi.y, dz = b.z - pi.z;
                    dx -= Lb * rint(dx * invL);
                    dy -= Lb * rint(dy * invL);
                    dz -= Lb * rint(dz * invL);
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    const double ip = rsqrt(r2 + eps2);
                    double f;
                    if (r2 < x2s) {
                        const double x2 = al2 * r2;
                        f = sc * (-2.0 / 3.0 + x2 * (0.4 + x2 * (-1.0 / 7.0 + x2 * (1.0 / 27.0))));
                    } else {
                        const double ir = rsqrt(r2), r = r2 * ir;
                        f = -erf(al * r) * ir * ir * ir + cg * exp(-al2 * r2) * ir * ir;
                    }
                    const double s = b.w * (ip * ip * ip + f);
                    ax += s * dx;
                    ay += s * dy;
                    az += s * dz;
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
        part[(it * L.S_max + sidx) * (long long)K::ITILE + tid] = make_double4(ax, ay, az, 0.0);
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

// ---------------------------------------------------------------- k space
// Half of the k-space: n = (nx, ny, nz) with nx > 0, or nx = 0 and ny > 0, or
// nx = ny = 0 and nz > 0, and |n|^2 <= nk^2.  The -n terms equal the n terms,
// so w carries a factor 2: w = 2 (4 pi / L^3) exp(-k^2/(4 alpha^2)) / k^2.
struct KVec {
    int nx, ny, nz, pad;
};

// Where the k-space kernels read bodies.  FP32: pair-interleaved records of
// `rec` floats per pair of bodies (8: [x0 x1 y0 y1 z0 z1 m0 m1], the force
// input; 16: the VJP input, whose co-vector follows at 8, 10, 12).  FP64:
// `rec` double4 per body (1: (x, y, z, m); 2: then (wx, wy, wz, 0)).  The
// structure factors weigh each body by entry `widx` of its record: the mass
// (6 in FP32, 3 in FP64) or a co-vector component (8/10/12; 4/5/6).
struct BodySrc {
    const float *pk;
    const double4 *pos;
    int rec, widx;
};

__host__ __device__ inline BodySrc masses_of(const float *pk, const double4 *pos) {
    return BodySrc{pk, pos, pos ? 1 : 8, pos ? 3 : 6};
}

// Body position as FP64 from either layout.
__device__ __forceinline__ double3 body_pos(const BodySrc &b, long long i) {
    if (b.pos) {
        const double4 p = b.pos[i * b.rec];
        return make_double3(p.x, p.y, p.z);
    }
    const float *p = b.pk + (i >> 1) * b.rec + (i & 1);
    return make_double3((double)p[0], (double)p[2], (double)p[4]);
}

// Record entry k of body i (FP32: float k of the pair record's lane; FP64:
// component k of the double4 record, 0..7).
__device__ __forceinline__ double body_entry(const BodySrc &b, long long i, int k) {
    if (b.pos) {
        const double4 p = b.pos[i * b.rec + (k >> 2)];
        const int c = k & 3;
        return c == 0 ? p.x : (c == 1 ? p.y : (c == 2 ? p.z : p.w));
    }
    return (double)b.pk[(i >> 1) * b.rec + (i & 1) + k];
}

__device__ __forceinline__ double body_weight(const BodySrc &b, long long i) {
    return body_entry(b, i, b.widx);
}

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// Phase tables of every body, once per force evaluation:
//   ph[(3 i + c) (nk + 1) + n] = exp(2 pi i n x_c / L),  n = 0..nk,
// with n x_c / L reduced exactly (FP64: exact for |n| < 2^20, minus its
// nearest integer) before sincospi.  One thread per (body, axis).
//
// wrap (FP32 pair-packed bodies only, else null): the same bodies with each
// coordinate wrapped into [0, L] as x - L floor(x / L) in FP64, rounded once
// (exact for a coordinate already in [0, L)), the input of ewald_f32_kernel.
template <typename T>
__global__ void ewald_phase_kernel(BodySrc src, long long N, EwaldArgs A,
                                   typename Vec2<T>::type *__restrict__ ph, float *__restrict__ wrap) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= 3 * N) return;
    const long long i = q / 3;
    const int c = (int)(q - 3 * i);
    const double3 p = body_pos(src, i);
    const double xc = c == 0 ? p.x : (c == 1 ? p.y : p.z);
    const double u = xc / A.L;
    if (wrap) {
        const long long o = (i >> 1) * 8 + (i & 1);
        wrap[o + 2 * c] = (float)(xc - A.L * floor(u));
        if (c == 0) wrap[o + 6] = src.pk[o + 6];
    }
    typename Vec2<T>::type *o = ph + q * (A.nk + 1);
    for (int n = 0; n <= A.nk; ++n) {
        double f = (double)n * u;
        f -= rint(f);
        T sn, cs;
        sincospi((T)(2.0 * f), &sn, &cs);
        o[n].x = cs;
        o[n].y = sn;
    }
}

// The k-vectors of the half space are ordered (nx, ny, nz) with nz fastest, so
// those sharing (nx, ny) form a "pencil" of consecutive nz.  exp(i k.x) is the
// product of the x and y phases, once per pencil and body, with the z phase.
struct KPencil {
    int nx, ny, nz0, len;         // k = (nx, ny, nz0 .. nz0 + len - 1)
    int koff, pad0, pad1, pad2;   // index of the pencil's first k-vector
};

// exp(i n 2 pi x_c / L) of one body for -nk <= n <= nk from its table of
// n = 0 .. nk (entries `stride` apart): negative n take the conjugate.
template <typename T, typename T2>
__device__ __forceinline__ T2 axis_phase(const T2 *row, int n, int stride) {
    T2 v = row[(n < 0 ? -n : n) * stride];
    if (n < 0) v.y = -v.y;
    return v;
}

constexpr int kEwKThreads = 256;  // k-vectors per block of the structure-factor kernel

// bodies per shared-memory batch of the structure-factor kernel
template <typename T>
__host__ __device__ constexpr int ew_bodies() { return sizeof(T) == 4 ? 64 : 32; }

// Partial structure factors: rho_part[split][k] = sum over the split's bodies
// of m_j exp(i k.x_j) (m_j: the weight src names, the mass by default).  Grid
// (k chunks, body splits); a chunk is a run of whole
// pencils with at most kEwKThreads k-vectors (rchunk: first pencil of chunk c;
// np_max pencils at most), one k per thread.  Per batch of kEwBodies bodies the
// block stages their tables, then the per-(body, pencil) base
// m_j exp(i (kx x_j + ky y_j)), so a k costs one z-table read and one complex
// multiply-add per body.  ewald_rho_sum_kernel adds the splits in order
// (deterministic).
template <typename T>
__global__ void __launch_bounds__(kEwKThreads)
    ewald_rho_kernel(BodySrc src, long long N,
                     const typename Vec2<T>::type *__restrict__ ph, const KPencil *__restrict__ pen,
                     const int *__restrict__ rchunk, int np_max, int nkv, EwaldArgs A,
                     double2 *__restrict__ rho_part) {
    using T2 = typename Vec2<T>::type;
    constexpr int kEwBodies = ew_bodies<T>();
    extern __shared__ __align__(16) unsigned char sm[];
    const int nt = A.nk + 1;
    T2 *tab = reinterpret_cast<T2 *>(sm);                       // [kEwBodies][3][nt]
    T2 *base = tab + kEwBodies * 3 * nt;                        // [kEwBodies][np_max]
    T *tm = reinterpret_cast<T *>(base + kEwBodies * np_max);   // [kEwBodies]
    int2 *sp = reinterpret_cast<int2 *>(tm + kEwBodies);        // [np_max] (nx, ny) of the chunk
    const int p0 = rchunk[blockIdx.x], np = rchunk[blockIdx.x + 1] - p0;
    const int k0 = pen[p0].koff;
    const int nkc = pen[p0 + np - 1].koff + pen[p0 + np - 1].len - k0;
    const int t = threadIdx.x;
    for (int l = t; l < np; l += kEwKThreads) sp[l] = make_int2(pen[p0 + l].nx, pen[p0 + l].ny);
    // this thread's k: its pencil (lp) and nz
    int lp = 0;
    while (lp + 1 < np && pen[p0 + lp + 1].koff <= k0 + t) ++lp;
    const int nz = pen[p0 + lp].nz0 + (k0 + t - pen[p0 + lp].koff);
    const int zrow = 2 * nt + (nz < 0 ? -nz : nz);
    const T zs = nz < 0 ? (T)-1 : (T)1;
    const long long per = (N + gridDim.y - 1) / gridDim.y;
    const long long b0 = (long long)blockIdx.y * per, b1 = min(N, b0 + per);
    double cr = 0.0, ci = 0.0;
    for (long long j0 = b0; j0 < b1; j0 += kEwBodies) {
        const int nb = (int)min((long long)kEwBodies, b1 - j0);
        __syncthreads();
        const T2 *tsrc = ph + j0 * 3 * nt;
        for (int q = t; q < nb * 3 * nt; q += kEwKThreads) tab[q] = tsrc[q];
        for (int b = t; b < nb; b += kEwKThreads) tm[b] = (T)body_weight(src, j0 + b);
        __syncthreads();
        for (int q = t; q < nb * np; q += kEwKThreads) {
            const int b = q / np, l = q - b * np;
            const int2 P = sp[l];
            const T2 *tb = tab + b * 3 * nt;
            const T2 x = tb[P.x];
            const T2 y = axis_phase<T, T2>(tb + nt, P.y, 1);
            const T m = tm[b];
            T2 v;
            v.x = m * (x.x * y.x - x.y * y.y);
            v.y = m * (x.x * y.y + x.y * y.x);
            base[q] = v;
        }
        __syncthreads();
        if (t < nkc) {
            T pr = 0, pi = 0;
#pragma unroll 4
            for (int b = 0; b < nb; ++b) {
                const T2 z = tab[b * 3 * nt + zrow];
                const T2 w = base[b * np + lp];
                const T zi = zs * z.y;
                pr += w.x * z.x - w.y * zi;
                pi += w.x * zi + w.y * z.x;
            }
            cr += (double)pr;
            ci += (double)pi;
        }
    }
    if (t < nkc) rho_part[(long long)blockIdx.y * nkv + k0 + t] = make_double2(cr, ci);
}

// Shared memory of ewald_rho_kernel.
template <typename T>
__host__ inline size_t ew_rho_smem(int nk, int np_max) {
    using T2 = typename Vec2<T>::type;
    constexpr int nb = ew_bodies<T>();
    return ((size_t)nb * 3 * (nk + 1) + (size_t)nb * np_max) * sizeof(T2) + nb * sizeof(T) +
           (size_t)np_max * sizeof(int2);
}

// rho[k] = sum of the splits in order; wcs[k] = (w_k C(k), w_k S(k)) for the
// long-range force (C, S the real and imaginary parts of rho).
template <typename T>
__global__ void ewald_rho_sum_kernel(const double2 *__restrict__ rho_part, int splits, int nkv,
                                     const double *__restrict__ w, double2 *__restrict__ rho,
                                     typename Vec2<T>::type *__restrict__ wcs) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nkv) return;
    double r = 0.0, i = 0.0;
    for (int s = 0; s < splits; ++s) {
        const double2 v = rho_part[(long long)s * nkv + k];
        r += v.x;
        i += v.y;
    }
    rho[k] = make_double2(r, i);
    wcs[k].x = (T)(w[k] * r);
    wcs[k].y = (T)(w[k] * i);
}

// Long-range acceleration (G-less) at every body:
//   lr_i = -sum_k w_k k [sin(k.x_i) C(k) - cos(k.x_i) S(k)].
// A block holds kEwFThreads bodies' tables in shared memory as
// [3 nt][kEwFThreads] (a warp reads consecutive entries) and runs
// kEwFSlices threads per body, each taking every kEwFSlices-th pencil.  Per
// pencil a thread forms the x-y phase once, then walks nz: one z-table read,
// one complex multiply and the weights (w C, w S) read as a broadcast per k.
// The sum over a pencil is scaled by (nx, ny) once.  Pencils arrive in chunks
// of at most ew_fk<T>() k-vectors (fchunk), whose weights are staged first.
// The slices' sums are added in slice order at the end (deterministic).
constexpr int kEwFThreads = 64;    // bodies per block
constexpr int kEwFSlices = 4;      // threads per body
constexpr int kEwFKBytes = 16384;  // staged weights per chunk

template <typename T>
__host__ __device__ constexpr int ew_fk() { return kEwFKBytes / (2 * (int)sizeof(T)); }

template <typename T, typename T4>
__global__ void __launch_bounds__(kEwFThreads * kEwFSlices)
    ewald_kforce_kernel(long long N, const typename Vec2<T>::type *__restrict__ ph,
                        const KPencil *__restrict__ pen, const int *__restrict__ fchunk, int nfchunk,
                        const typename Vec2<T>::type *__restrict__ wcs, EwaldArgs A,
                        T4 *__restrict__ lr) {
    using T2 = typename Vec2<T>::type;
    constexpr int NT = kEwFThreads * kEwFSlices;
    constexpr int FK = ew_fk<T>();
    extern __shared__ __align__(16) unsigned char sm[];
    const int nt = A.nk + 1;
    T2 *sw = reinterpret_cast<T2 *>(sm);   // [FK] weights of the chunk
    T2 *tab = sw + FK;                     // [3 nt][kEwFThreads]
    const long long i0 = (long long)blockIdx.x * kEwFThreads;
    const int nb = (int)min((long long)kEwFThreads, N - i0);
    for (int q = threadIdx.x; q < nb * 3 * nt; q += NT) {
        const int b = q / (3 * nt), r = q - b * 3 * nt;
        tab[r * kEwFThreads + b] = ph[i0 * 3 * nt + q];
    }
    const int bi = threadIdx.x % kEwFThreads, sl = threadIdx.x / kEwFThreads;
    const long long i = i0 + bi;
    const T2 *mine = tab + bi;
    const T2 *zt = mine + 2 * nt * kEwFThreads;
    const double tpl = 2.0 * acos(-1.0) / A.L;
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int c = 0; c < nfchunk; ++c) {
        const int p0 = fchunk[c], p1 = fchunk[c + 1];
        const int k0 = pen[p0].koff, nkc = pen[p1 - 1].koff + pen[p1 - 1].len - k0;
        __syncthreads();
        for (int q = threadIdx.x; q < nkc; q += NT) sw[q] = wcs[k0 + q];
        __syncthreads();
        if (i < N) {
            T px = 0, py = 0, pz = 0;
            for (int p = p0 + sl; p < p1; p += kEwFSlices) {
                const KPencil P = pen[p];
                const T2 x = mine[P.nx * kEwFThreads];
                const T2 y = axis_phase<T, T2>(mine + nt * kEwFThreads, P.ny, kEwFThreads);
                const T er = x.x * y.x - x.y * y.y, ei = x.x * y.y + x.y * y.x;
                const T2 *wk = sw + (P.koff - k0 - P.nz0);   // weights indexed by nz
                T B = 0, Bz = 0;
                const int nz1 = P.nz0 + P.len;
                int nz = P.nz0;
                for (; nz < 0 && nz < nz1; ++nz) {           // negative nz: conjugate z phase
                    const T2 z = zt[-nz * kEwFThreads];
                    const T cr = er * z.x + ei * z.y, si = ei * z.x - er * z.y;
                    const T2 w = wk[nz];
                    const T b = si * w.x - cr * w.y;
                    B += b;
                    Bz += b * (T)nz;
                }
                for (; nz < nz1; ++nz) {
                    const T2 z = zt[nz * kEwFThreads];
                    const T cr = er * z.x - ei * z.y, si = er * z.y + ei * z.x;
                    const T2 w = wk[nz];
                    const T b = si * w.x - cr * w.y;
                    B += b;
                    Bz += b * (T)nz;
                }
                px += (T)P.nx * B;
                py += (T)P.ny * B;
                pz += Bz;
            }
            ax += (double)px;
            ay += (double)py;
            az += (double)pz;
        }
    }
    // add the slices in order; the weight staging area holds the partial sums
    __syncthreads();
    double *red = reinterpret_cast<double *>(sm);   // [3][kEwFSlices][kEwFThreads]
    static_assert(3 * NT * sizeof(double) <= kEwFKBytes, "reduction fits");
    red[(0 * kEwFSlices + sl) * kEwFThreads + bi] = ax;
    red[(1 * kEwFSlices + sl) * kEwFThreads + bi] = ay;
    red[(2 * kEwFSlices + sl) * kEwFThreads + bi] = az;
    __syncthreads();
    if (sl == 0 && i < N) {
        double sx = 0.0, sy = 0.0, sz = 0.0;
#pragma unroll
        for (int t = 0; t < kEwFSlices; ++t) {
            sx += red[(0 * kEwFSlices + t) * kEwFThreads + bi];
            sy += red[(1 * kEwFSlices + t) * kEwFThreads + bi];
            sz += red[(2 * kEwFSlices + t) * kEwFThreads + bi];
        }
        lr[i].x = (T)(-tpl * sx);
        lr[i].y = (T)(-tpl * sy);
        lr[i].z = (T)(-tpl * sz);
        lr[i].w = (T)0;
    }
}

}  // namespace colatus
