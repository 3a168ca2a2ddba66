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
// FP64 before sincospi); the structure factors are one pass over (k, body)
// pairs with those tables staged in shared memory, and the force pass
// evaluates the k-sum at every body from its own tables.
#pragma once

#include "common.cuh"
#include "force.cuh"

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

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
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
// including the minimum image and the accumulation.
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
    return __fmul2_rn(mj, __fadd2_rn(ip3, f));
}

template <int NT, int IPT, int JT, int STAGES, int FOLD, bool COMP, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    ewald_f32_kernel(const float *__restrict__ pk, float4 *__restrict__ part, int *__restrict__ flags,
                     ForceLaunch L, float eps2, EwaldArgs A) {
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
                            const float2 s = ewald_pair2(dx, dy, dz, mj, A, e2);
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
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            dst[tid + k * NT] = make_float4(hx[k], hy[k], hz[k], 0.f);
            if (COMP) dst[K::ITILE + tid + k * NT] = make_float4(lx[k], ly[k], lz[k], 0.f);
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

// Body position component as FP64 from either layout.
__device__ __forceinline__ double3 body_pos(const float *pk, const double4 *pos, long long i) {
    if (pos) {
        const double4 p = pos[i];
        return make_double3(p.x, p.y, p.z);
    }
    const float *p = pk + (i >> 1) * 8 + (i & 1);
    return make_double3((double)p[0], (double)p[2], (double)p[4]);
}

__device__ __forceinline__ double body_mass(const float *pk, const double4 *pos, long long i) {
    if (pos) return pos[i].w;
    return (double)pk[(i >> 1) * 8 + (i & 1) + 6];
}

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// Phase tables of every body, once per force evaluation:
//   ph[(3 i + c) (nk + 1) + n] = exp(2 pi i n x_c / L),  n = 0..nk,
// with n x_c / L reduced exactly (FP64: exact for |n| < 2^20, minus its
// nearest integer) before sincospi.  One thread per (body, axis).
template <typename T>
__global__ void ewald_phase_kernel(const float *__restrict__ pk, const double4 *__restrict__ pos,
                                   long long N, EwaldArgs A, typename Vec2<T>::type *__restrict__ ph) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= 3 * N) return;
    const long long i = q / 3;
    const int c = (int)(q - 3 * i);
    const double3 p = body_pos(pk, pos, i);
    const double u = (c == 0 ? p.x : (c == 1 ? p.y : p.z)) / A.L;
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

constexpr int kEwBodies = 32;     // bodies per shared-memory table batch
constexpr int kEwKThreads = 128;  // k-vectors per block of the structure-factor kernel

// exp(i k.x) of one body from its three axis tables (tab: [3][nt]); negative
// ny, nz take the conjugate.
template <typename T, typename T2>
__device__ __forceinline__ void phase_of(const T2 *tab, int nt, const KVec &k, T &re, T &im) {
    const T2 x = tab[k.nx];
    T2 y = tab[nt + abs(k.ny)];
    T2 z = tab[2 * nt + abs(k.nz)];
    if (k.ny < 0) y.y = -y.y;
    if (k.nz < 0) z.y = -z.y;
    const T er = x.x * y.x - x.y * y.y, ei = x.x * y.y + x.y * y.x;
    re = er * z.x - ei * z.y;
    im = er * z.y + ei * z.x;
}

// rho[k] += sum over this block's bodies of m_j exp(i k.x_j); grid (k chunks,
// body splits), block kEwKThreads; the bodies' tables are staged through
// shared memory kEwBodies at a time.
template <typename T>
__global__ void __launch_bounds__(kEwKThreads)
    ewald_rho_kernel(const float *__restrict__ pk, const double4 *__restrict__ pos, long long N,
                     const typename Vec2<T>::type *__restrict__ ph, const KVec *__restrict__ kv,
                     int nkv, EwaldArgs A, double2 *__restrict__ rho) {
    using T2 = typename Vec2<T>::type;
    extern __shared__ __align__(16) unsigned char sm[];
    const int nt = A.nk + 1;
    T2 *tab = reinterpret_cast<T2 *>(sm);                       // [kEwBodies][3][nt]
    T *tm = reinterpret_cast<T *>(tab + kEwBodies * 3 * nt);    // [kEwBodies]
    const int kidx = blockIdx.x * kEwKThreads + threadIdx.x;
    KVec k = {0, 0, 0, 0};
    if (kidx < nkv) k = kv[kidx];
    const long long per = (N + gridDim.y - 1) / gridDim.y;
    const long long b0 = (long long)blockIdx.y * per, b1 = min(N, b0 + per);
    double cr = 0.0, ci = 0.0;
    for (long long j0 = b0; j0 < b1; j0 += kEwBodies) {
        const int nb = (int)min((long long)kEwBodies, b1 - j0);
        __syncthreads();
        const T2 *src = ph + j0 * 3 * nt;
        for (int q = threadIdx.x; q < nb * 3 * nt; q += kEwKThreads) tab[q] = src[q];
        for (int b = threadIdx.x; b < nb; b += kEwKThreads) tm[b] = (T)body_mass(pk, pos, j0 + b);
        __syncthreads();
        if (kidx < nkv) {
            T pr = 0, pi = 0;
            for (int b = 0; b < nb; ++b) {
                T fr, fi;
                phase_of<T, T2>(tab + b * 3 * nt, nt, k, fr, fi);
                pr += tm[b] * fr;
                pi += tm[b] * fi;
            }
            cr += (double)pr;
            ci += (double)pi;
        }
    }
    if (kidx < nkv) {
        atomicAdd(&rho[kidx].x, cr);
        atomicAdd(&rho[kidx].y, ci);
    }
}

// Long-range acceleration (G-less) at every body:
//   lr_i = -sum_k w_k k [sin(k.x_i) C(k) - cos(k.x_i) S(k)]
// One thread per body.  The k-vectors are staged through shared memory
// kEwKChunk at a time, already in the form the loop uses (the three table
// offsets, the conjugation signs, n as floating point, w C and w S), so the
// loop body is table reads and FMAs only; two accumulator chains.  The
// block's body tables sit in shared memory as [3 nt][kEwFThreads]: every
// thread evaluates the same k at a time, so a warp reads consecutive entries.
constexpr int kEwFThreads = 64;
constexpr int kEwKChunk = 256;

template <typename T>
struct __align__(16) KStage {   // 48 B (float) / 80 B (double): whole 16-byte loads
    int ox, oy, oz, pad;   // table rows of |nx|, |ny|, |nz| (x 64 threads)
    T sy, sz;              // signs of ny, nz (conjugation)
    T kx, ky, kz;          // n as floating point
    T wc, ws;              // w_k C(k), w_k S(k)
    T pad2;
};

template <typename T, typename T4>
__global__ void __launch_bounds__(kEwFThreads)
    ewald_kforce_kernel(long long N, const typename Vec2<T>::type *__restrict__ ph,
                        const KVec *__restrict__ kv, const double *__restrict__ w,
                        const double2 *__restrict__ rho, int nkv, EwaldArgs A, T4 *__restrict__ lr) {
    using T2 = typename Vec2<T>::type;
    extern __shared__ __align__(16) unsigned char sm[];
    const int nt = A.nk + 1;
    KStage<T> *sk = reinterpret_cast<KStage<T> *>(sm);
    T2 *tab = reinterpret_cast<T2 *>(sk + kEwKChunk);
    const long long i0 = (long long)blockIdx.x * kEwFThreads;
    const int nb = (int)min((long long)kEwFThreads, N - i0);
    for (int q = threadIdx.x; q < nb * 3 * nt; q += kEwFThreads) {
        const int b = q / (3 * nt), r = q - b * 3 * nt;
        tab[r * kEwFThreads + b] = ph[i0 * 3 * nt + q];
    }
    const long long i = i0 + threadIdx.x;
    const T2 *mine = tab + threadIdx.x;
    const double tpl = 2.0 * acos(-1.0) / A.L;
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int k0 = 0; k0 < nkv; k0 += kEwKChunk) {
        const int nc = min(kEwKChunk, nkv - k0);
        __syncthreads();
        for (int q = threadIdx.x; q < nc; q += kEwFThreads) {
            const KVec k = kv[k0 + q];
            const double2 r = rho[k0 + q];
            KStage<T> e;
            e.ox = k.nx * kEwFThreads;
            e.oy = (nt + abs(k.ny)) * kEwFThreads;
            e.oz = (2 * nt + abs(k.nz)) * kEwFThreads;
            e.pad = 0;
            e.sy = k.ny < 0 ? (T)-1 : (T)1;
            e.sz = k.nz < 0 ? (T)-1 : (T)1;
            e.kx = (T)k.nx;
            e.ky = (T)k.ny;
            e.kz = (T)k.nz;
            e.wc = (T)(w[k0 + q] * r.x);
            e.ws = (T)(w[k0 + q] * r.y);
            e.pad2 = (T)0;
            sk[q] = e;
        }
        __syncthreads();
        if (i < N) {
            T px[2] = {0, 0}, py[2] = {0, 0}, pz[2] = {0, 0};
#pragma unroll 2
            for (int q = 0; q < nc; ++q) {
                const KStage<T> &e = sk[q];
                const T2 x = mine[e.ox], y = mine[e.oy], z = mine[e.oz];
                const T yi = e.sy * y.y, zi = e.sz * z.y;
                const T er = x.x * y.x - x.y * yi, ei = x.x * yi + x.y * y.x;
                const T cr = er * z.x - ei * zi, si = er * zi + ei * z.x;   // cos, sin of k.x_i
                const T b = si * e.wc - cr * e.ws;
                const int c = q & 1;
                px[c] += b * e.kx;
                py[c] += b * e.ky;
                pz[c] += b * e.kz;
            }
            ax += (double)px[0] + (double)px[1];
            ay += (double)py[0] + (double)py[1];
            az += (double)pz[0] + (double)pz[1];
        }
    }
    if (i < N) {
        lr[i].x = (T)(-tpl * ax);
        lr[i].y = (T)(-tpl * ay);
        lr[i].z = (T)(-tpl * az);
        lr[i].w = (T)0;
    }
}

}  // namespace colatus
