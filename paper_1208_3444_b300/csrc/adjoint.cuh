// adjoint.cuh -- vector-Jacobian product (VJP) of the Eq. 1 force sum, and
// the element-wise updates of the discrete adjoint of the KDK leapfrog.
//
// For the raw force F_k = sum_{j != k} m_j d_kj / s_kj^3 (d_kj = x_j - x_k,
// s^2 = |d|^2 + eps^2) and a co-vector w_k, the gradients of L = sum_k w_k.F_k
// are (differentiating the Eq. 1 sum; J(d) = I/s^3 - 3 d d^T / s^5, even in d)
//     dL/dx_i = sum_{j != i} J(d_ij) (m_i w_j - m_j w_i)
//             = m_i U_i - B_i w_i - 3 V_i,
//     dL/dm_i = -sum_{j != i} (w_j . d_ij) / s_ij^3 = -Gm_i,
// with the per-pair accumulations
//     U_i = sum inv3 w_j,  B_i = sum m_j inv3,  Gm_i = sum inv3 (w_j . d),
//     V_i = sum inv5 (m_i (w_j . d) - m_j (w_i . d)) d.
// That is 26 FP32 lane-ops and one MUFU.RSQ per interaction (the force: 12).
// Scaled form: with w'_i = w_i / m_i the pair weight m_i l_j - m_j l_i is
// m_i (l_j - m_j (w'_i . d)), so V_i = m_i sum inv5 (l_j - m_j (w'_i . d)) d
// and the multiply by m_i leaves the pair loop: 25 lane-ops.  The scaled
// quantities differ from the general form's by the factor 1/m_i, so an i-tile
// takes this form when every body in it has a mass within 2^-40 .. 2^40 and a
// finite scaled co-vector, or a zero co-vector (padding).  Any other tile (a
// massless body with a co-vector, for one) takes the 26-op form.
// The self pair must be masked here: its U and B terms are each ~1/eps^3 and
// cancel only in exact arithmetic.  Masking is done only in the units whose
// j-tile overlaps the i-tile.
//
// Same decomposition and pipeline as force.cuh (stream-K over i-tile x j-tile
// units, bulk-copy j-tiles, bounded mbarrier waits).  FP32 bodies with their
// co-vectors are pair-interleaved, 16 floats per pair of bodies:
//     [x0 x1 y0 y1 | z0 z1 m0 m1 | wx0 wx1 wy0 wy1 | wz0 wz1 0 0]
// Segments are float4 (dL/dx, dL/dm) per body.
#pragma once

#include "common.cuh"
#include "force.cuh"
#include "vjp_sym.cuh"

namespace colatus {

// Range check of the scaled form for one i-body: mass m within 2^-40 .. 2^40
// and finite scaled co-vector (sx, sy, sz).
__device__ __forceinline__ bool scaled_fits(float m, float sx, float sy, float sz) {
    return m >= 0x1p-40f && m <= 0x1p40f && isfinite(sx) && isfinite(sy) && isfinite(sz);
}

template <int NT, int IPT, int JT, int STAGES>
struct VjpKernel {
    static constexpr int ITILE = NT * IPT;
    static constexpr uint32_t TILE_BYTES = JT * 32;   // 32 B per body
    static constexpr int SMEM = STAGES * TILE_BYTES + STAGES * 8;
};

// One j-tile of the VJP for the IPT i-bodies of this thread.  ibase: index of
// the tile's first j-body; MASK: the tile may contain i itself; SCALED: the
// 25-op form, with (wxi, wyi, wzi) holding w_i / m_i and mi unused (V then
// accumulates V_i / m_i); UNR: unroll depth of the j-pair loop (a tuning knob).
template <int IPT, int JT, bool MASK, bool SCALED, int UNR>
__device__ __forceinline__ void vjp_tile(const float4 *__restrict__ t, long long jbase,
                                         const long long (&ii)[IPT], const float2 (&nx)[IPT],
                                         const float2 (&ny)[IPT], const float2 (&nz)[IPT],
                                         const float2 (&mi)[IPT], const float2 (&wxi)[IPT],
                                         const float2 (&wyi)[IPT], const float2 (&wzi)[IPT],
                                         const float2 e2, float2 (&Ux)[IPT], float2 (&Uy)[IPT],
                                         float2 (&Uz)[IPT], float2 (&Bm)[IPT], float2 (&Vx)[IPT],
                                         float2 (&Vy)[IPT], float2 (&Vz)[IPT], float2 (&Gm)[IPT]) {
#pragma unroll (UNR)
    for (int q = 0; q < JT / 2; ++q) {
        const float4 A = t[4 * q];
        const float4 Bq = t[4 * q + 1];
        const float4 C = t[4 * q + 2];
        const float4 D = t[4 * q + 3];
        const float2 xj = make_float2(A.x, A.y), yj = make_float2(A.z, A.w);
        const float2 zj = make_float2(Bq.x, Bq.y), mj = make_float2(Bq.z, Bq.w);
        const float2 wxj = make_float2(C.x, C.y), wyj = make_float2(C.z, C.w);
        const float2 wzj = make_float2(D.x, D.y);
        const float2 nmj = make_float2(-mj.x, -mj.y);
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const float2 dx = __fadd2_rn(xj, nx[k]);
            const float2 dy = __fadd2_rn(yj, ny[k]);
            const float2 dz = __fadd2_rn(zj, nz[k]);
            float2 r2 = __ffma2_rn(dx, dx, e2);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            float2 inv = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
            if (MASK) {
                const long long j0 = jbase + 2 * q;
                inv.x = (j0 == ii[k]) ? 0.f : inv.x;
                inv.y = (j0 + 1 == ii[k]) ? 0.f : inv.y;
            }
            const float2 inv2 = __fmul2_rn(inv, inv);
            const float2 inv3 = __fmul2_rn(inv, inv2);
            const float2 inv5 = __fmul2_rn(inv3, inv2);
            Ux[k] = __ffma2_rn(inv3, wxj, Ux[k]);
            Uy[k] = __ffma2_rn(inv3, wyj, Uy[k]);
            Uz[k] = __ffma2_rn(inv3, wzj, Uz[k]);
            Bm[k] = __ffma2_rn(mj, inv3, Bm[k]);
            float2 lj = __fmul2_rn(wxj, dx);
            lj = __ffma2_rn(wyj, dy, lj);
            lj = __ffma2_rn(wzj, dz, lj);
            float2 li = __fmul2_rn(wxi[k], dx);
            li = __ffma2_rn(wyi[k], dy, li);
            li = __ffma2_rn(wzi[k], dz, li);
            const float2 dw = SCALED ? __ffma2_rn(nmj, li, lj)
                                     : __ffma2_rn(mi[k], lj, __fmul2_rn(nmj, li));
            const float2 g = __fmul2_rn(inv5, dw);
            Vx[k] = __ffma2_rn(g, dx, Vx[k]);
            Vy[k] = __ffma2_rn(g, dy, Vy[k]);
            Vz[k] = __ffma2_rn(g, dz, Vz[k]);
            Gm[k] = __ffma2_rn(inv3, lj, Gm[k]);
        }
    }
}

template <int NT, int IPT, int JT, int STAGES, int MINB, int UNR = 1>
__global__ void __launch_bounds__(NT, MINB)
    vjp_f32_kernel(const float *__restrict__ pkw, float4 *__restrict__ part, int *__restrict__ flags,
                   ForceLaunch L, float eps2) {
    using K = VjpKernel<NT, IPT, JT, STAGES>;
    extern __shared__ __align__(128) unsigned char smem[];
    float4 *tiles = reinterpret_cast<float4 *>(smem);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * K::TILE_BYTES);
    constexpr int TILE_F4 = JT * 2;   // float4 per tile

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
            bulk_load(tiles + s * TILE_F4, pkw + jt * (long long)JT * 8, K::TILE_BYTES, &full[s]);
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
        long long ii[IPT];
        float2 nx[IPT], ny[IPT], nz[IPT], mi[IPT], wxi[IPT], wyi[IPT], wzi[IPT];
        float2 Ux[IPT], Uy[IPT], Uz[IPT], Bm[IPT], Vx[IPT], Vy[IPT], Vz[IPT], Gm[IPT];
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const long long i = it * K::ITILE + tid + k * NT;
            ii[k] = i;
            const float *p = pkw + (i >> 1) * 16 + (i & 1);
            const float x = __ldg(p), y = __ldg(p + 2), z = __ldg(p + 4), m = __ldg(p + 6);
            const float wx = __ldg(p + 8), wy = __ldg(p + 10), wz = __ldg(p + 12);
            nx[k] = make_float2(-x, -x);
            ny[k] = make_float2(-y, -y);
            nz[k] = make_float2(-z, -z);
            mi[k] = make_float2(m, m);
            wxi[k] = make_float2(wx, wx);
            wyi[k] = make_float2(wy, wy);
            wzi[k] = make_float2(wz, wz);
            Ux[k] = Uy[k] = Uz[k] = Bm[k] = make_float2(0.f, 0.f);
            Vx[k] = Vy[k] = Vz[k] = Gm[k] = make_float2(0.f, 0.f);
        }
        // the scaled form for this i-tile?  (block-uniform: every thread
        // reaches this point once per i-tile)
        bool fits = true;
        float sxi[IPT], syi[IPT], szi[IPT];
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const float m = mi[k].x, r = 1.f / m;
            sxi[k] = wxi[k].x * r;
            syi[k] = wyi[k].x * r;
            szi[k] = wzi[k].x * r;
            if (wxi[k].x == 0.f && wyi[k].x == 0.f && wzi[k].x == 0.f)
                sxi[k] = syi[k] = szi[k] = 0.f;
            else
                fits = fits && scaled_fits(m, sxi[k], syi[k], szi[k]);
        }
        const bool scaled = __syncthreads_and(fits);
        if (scaled) {
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                wxi[k] = make_float2(sxi[k], sxi[k]);
                wyi[k] = make_float2(syi[k], syi[k]);
                wzi[k] = make_float2(szi[k], szi[k]);
            }
        }
        const long long ilo = it * K::ITILE, ihi = ilo + K::ITILE;
        for (; u < uend; ++u) {
            const bool ok = mbar_wait_bounded(&full[stage], parity);
            if (ok) {
                const long long jt = u % n_jt;
                const long long jlo = jt * JT;
                const float4 *t = tiles + stage * TILE_F4;
                const bool diag = jlo < ihi && jlo + JT > ilo;
                if (scaled) {
                    if (diag)
                        vjp_tile<IPT, JT, true, true, UNR>(t, jlo, ii, nx, ny, nz, mi, wxi, wyi, wzi, e2,
                                                          Ux, Uy, Uz, Bm, Vx, Vy, Vz, Gm);
                    else
                        vjp_tile<IPT, JT, false, true, UNR>(t, jlo, ii, nx, ny, nz, mi, wxi, wyi, wzi,
                                                           e2, Ux, Uy, Uz, Bm, Vx, Vy, Vz, Gm);
                } else {
                    if (diag)
                        vjp_tile<IPT, JT, true, false, UNR>(t, jlo, ii, nx, ny, nz, mi, wxi, wyi, wzi,
                                                           e2, Ux, Uy, Uz, Bm, Vx, Vy, Vz, Gm);
                    else
                        vjp_tile<IPT, JT, false, false, UNR>(t, jlo, ii, nx, ny, nz, mi, wxi, wyi,
                                                            wzi, e2, Ux, Uy, Uz, Bm, Vx, Vy, Vz, Gm);
                }
            }
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
            if (tid == 0 && u + STAGES < u1) {
                const long long jt = (u + STAGES) % n_jt;
                mbar_arrive_expect_tx(&full[stage], K::TILE_BYTES);
                bulk_load(tiles + stage * TILE_F4, pkw + jt * (long long)JT * 8, K::TILE_BYTES,
                          &full[stage]);
            }
            if (++stage == STAGES) {
                stage = 0;
                parity ^= 1u;
            }
        }
        if (bad) break;
        const long long sidx = g - sk_owner(it * n_jt, W, G);
        float4 *dst = part + (it * L.S_max + sidx) * (long long)K::ITILE;
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const float *p = pkw + (ii[k] >> 1) * 16 + (ii[k] & 1);
            const float m = mi[k].x;
            const float wx = __ldg(p + 8), wy = __ldg(p + 10), wz = __ldg(p + 12);
            const float bm = Bm[k].x + Bm[k].y;
            const float v3 = scaled ? 3.f * m : 3.f;
            const float gx = m * (Ux[k].x + Ux[k].y) - bm * wx - v3 * (Vx[k].x + Vx[k].y);
            const float gy = m * (Uy[k].x + Uy[k].y) - bm * wy - v3 * (Vy[k].x + Vy[k].y);
            const float gz = m * (Uz[k].x + Uz[k].y) - bm * wz - v3 * (Vz[k].x + Vz[k].y);
            dst[tid + k * NT] = make_float4(gx, gy, gz, -(Gm[k].x + Gm[k].y));
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

// Equal-mass VJP (every body has mass m, no zero-mass padding enters).  With
// u = w_j - w_i the pair weight m_i w_j - m_j w_i is m u, so
//     dL/dx_i = m sum_j J(d) u = m (U' - 3 V'),
//     U' = sum inv3 u,  V' = sum inv5 (u . d) d,
// and, with w_j . d = u . d + w_i . d,
//     dL/dm_i = -sum inv3 (w_j . d) = -(Gm' + w_i . P_i),  Gm' = sum inv3 (u . d),
// P_i = sum_j d inv3 = F_i / m the (G-less) force the forward pass already
// computed at the same positions.  The kernel writes (m (U' - 3 V'), -Gm')
// per segment and the consumers add -w_i . F_i / m (add_eqm_vjp): 23 FP32
// lane-ops per interaction instead of 25, and no self-pair mask (u = 0).
template <int JT, int UNR>
__device__ __forceinline__ void vjp_eqm_tile(const float4 *__restrict__ t, const float2 (&nx)[4],
                                             const float2 (&ny)[4], const float2 (&nz)[4],
                                             const float2 (&nwx)[4], const float2 (&nwy)[4],
                                             const float2 (&nwz)[4], const float2 e2,
                                             float2 (&Ux)[4], float2 (&Uy)[4], float2 (&Uz)[4],
                                             float2 (&Vx)[4], float2 (&Vy)[4], float2 (&Vz)[4],
                                             float2 (&Gm)[4]) {
#pragma unroll (UNR)
    for (int q = 0; q < JT / 2; ++q) {
        const float4 A = t[4 * q];
        const float4 Bq = t[4 * q + 1];
        const float4 C = t[4 * q + 2];
        const float4 D = t[4 * q + 3];
        const float2 xj = make_float2(A.x, A.y), yj = make_float2(A.z, A.w);
        const float2 zj = make_float2(Bq.x, Bq.y);
        const float2 wxj = make_float2(C.x, C.y), wyj = make_float2(C.z, C.w);
        const float2 wzj = make_float2(D.x, D.y);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 dx = __fadd2_rn(xj, nx[k]);
            const float2 dy = __fadd2_rn(yj, ny[k]);
            const float2 dz = __fadd2_rn(zj, nz[k]);
            float2 r2 = __ffma2_rn(dx, dx, e2);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            const float2 inv = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
            const float2 inv2 = __fmul2_rn(inv, inv);
            const float2 inv3 = __fmul2_rn(inv, inv2);
            const float2 inv5 = __fmul2_rn(inv3, inv2);
            const float2 ux = __fadd2_rn(wxj, nwx[k]);
            const float2 uy = __fadd2_rn(wyj, nwy[k]);
            const float2 uz = __fadd2_rn(wzj, nwz[k]);
            Ux[k] = __ffma2_rn(inv3, ux, Ux[k]);
            Uy[k] = __ffma2_rn(inv3, uy, Uy[k]);
            Uz[k] = __ffma2_rn(inv3, uz, Uz[k]);
            float2 du = __fmul2_rn(ux, dx);
            du = __ffma2_rn(uy, dy, du);
            du = __ffma2_rn(uz, dz, du);
            const float2 g = __fmul2_rn(inv5, du);
            Vx[k] = __ffma2_rn(g, dx, Vx[k]);
            Vy[k] = __ffma2_rn(g, dy, Vy[k]);
            Vz[k] = __ffma2_rn(g, dz, Vz[k]);
            Gm[k] = __ffma2_rn(inv3, du, Gm[k]);
        }
    }
}

// Same launch shape, pipeline and segment layout as vjp_f32_kernel with
// IPT = 4 (so the VJP's launch plan and consumers apply unchanged).
template <int NT, int JT, int STAGES, int MINB, int UNR>
__global__ void __launch_bounds__(NT, MINB)
    vjp_eqm_f32_kernel(const float *__restrict__ pkw, float4 *__restrict__ part, int *__restrict__ flags,
                       ForceLaunch L, float eps2) {
    constexpr int IPT = 4;
    using K = VjpKernel<NT, IPT, JT, STAGES>;
    extern __shared__ __align__(128) unsigned char smem[];
    float4 *tiles = reinterpret_cast<float4 *>(smem);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * K::TILE_BYTES);
    constexpr int TILE_F4 = JT * 2;
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
            bulk_load(tiles + s * TILE_F4, pkw + jt * (long long)JT * 8, K::TILE_BYTES, &full[s]);
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
        float2 nx[IPT], ny[IPT], nz[IPT], nwx[IPT], nwy[IPT], nwz[IPT];
        float2 Ux[IPT], Uy[IPT], Uz[IPT], Vx[IPT], Vy[IPT], Vz[IPT], Gm[IPT];
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const long long i = it * K::ITILE + tid + k * NT;
            const float *p = pkw + (i >> 1) * 16 + (i & 1);
            const float x = __ldg(p), y = __ldg(p + 2), z = __ldg(p + 4);
            const float wx = __ldg(p + 8), wy = __ldg(p + 10), wz = __ldg(p + 12);
            nx[k] = make_float2(-x, -x);
            ny[k] = make_float2(-y, -y);
            nz[k] = make_float2(-z, -z);
            nwx[k] = make_float2(-wx, -wx);
            nwy[k] = make_float2(-wy, -wy);
            nwz[k] = make_float2(-wz, -wz);
            Ux[k] = Uy[k] = Uz[k] = make_float2(0.f, 0.f);
            Vx[k] = Vy[k] = Vz[k] = Gm[k] = make_float2(0.f, 0.f);
        }
        for (; u < uend; ++u) {
            const bool ok = mbar_wait_bounded(&full[stage], parity);
            if (ok)
                vjp_eqm_tile<JT, UNR>(tiles + stage * TILE_F4, nx, ny, nz, nwx, nwy, nwz, e2, Ux, Uy, Uz,
                                      Vx, Vy, Vz, Gm);
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
            if (tid == 0 && u + STAGES < u1) {
                const long long jt = (u + STAGES) % n_jt;
                mbar_arrive_expect_tx(&full[stage], K::TILE_BYTES);
                bulk_load(tiles + stage * TILE_F4, pkw + jt * (long long)JT * 8, K::TILE_BYTES,
                          &full[stage]);
            }
            if (++stage == STAGES) {
                stage = 0;
                parity ^= 1u;
            }
        }
        if (bad) break;
        const long long sidx = g - sk_owner(it * n_jt, W, G);
        float4 *dst = part + (it * L.S_max + sidx) * (long long)K::ITILE;
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const long long i = it * K::ITILE + tid + k * NT;
            const float m = __ldg(pkw + (i >> 1) * 16 + (i & 1) + 6);
            const float gx = m * ((Ux[k].x + Ux[k].y) - 3.f * (Vx[k].x + Vx[k].y));
            const float gy = m * ((Uy[k].x + Uy[k].y) - 3.f * (Vy[k].x + Vy[k].y));
            const float gz = m * ((Uz[k].x + Uz[k].y) - 3.f * (Vz[k].x + Vz[k].y));
            dst[tid + k * NT] = make_float4(gx, gy, gz, -(Gm[k].x + Gm[k].y));
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

// FP64 VJP: bodies as two double4 per body, (x, y, z, m) and (wx, wy, wz, 0).
template <int NT, int JT, int STAGES>
struct Vjp64Kernel {
    static constexpr int ITILE = NT;
    static constexpr uint32_t TILE_BYTES = JT * 64;
    static constexpr int SMEM = STAGES * TILE_BYTES + STAGES * 8;
};

template <int NT, int JT, int STAGES>
__global__ void __launch_bounds__(NT)
    vjp_f64_kernel(const double4 *__restrict__ bw, double4 *__restrict__ part,
                   int *__restrict__ flags, ForceLaunch L, double eps2) {
    using K = Vjp64Kernel<NT, JT, STAGES>;
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
            bulk_load(tiles + s * 2 * JT, bw + jt * 2LL * JT, K::TILE_BYTES, &full[s]);
        }
    }
    long long u = u0;
    bool bad = false;
    int stage = 0;
    uint32_t parity = 0;
    while (u < u1) {
        const long long it = u / n_jt;
        const long long uend = min(u1, (it + 1) * (long long)n_jt);
        const long long i = it * K::ITILE + tid;
        const double4 pi = bw[2 * i], wi = bw[2 * i + 1];
        double ux = 0, uy = 0, uz = 0, bm = 0, vx = 0, vy = 0, vz = 0, gm = 0;
        for (; u < uend; ++u) {
            const bool ok = mbar_wait_bounded(&full[stage], parity);
            if (ok) {
                const double4 *t = tiles + stage * 2 * JT;
                const long long jlo = (u % n_jt) * JT;
#pragma unroll 2
                for (int j = 0; j < JT; ++j) {
                    if (jlo + j == i) continue;
                    const double4 b = t[2 * j], w = t[2 * j + 1];
                    const double dx = b.x - pi.x, dy = b.y - pi.y, dz = b.z - pi.z;
                    const double r2 = dx * dx + dy * dy + dz * dz + eps2;
                    const double inv = rsqrt(r2);
                    const double inv2 = inv * inv, inv3 = inv * inv2, inv5 = inv3 * inv2;
                    ux += inv3 * w.x;
                    uy += inv3 * w.y;
                    uz += inv3 * w.z;
                    bm += b.w * inv3;
                    const double lj = w.x * dx + w.y * dy + w.z * dz;
                    const double li = wi.x * dx + wi.y * dy + wi.z * dz;
                    const double gg = inv5 * (pi.w * lj - b.w * li);
                    vx += gg * dx;
                    vy += gg * dy;
                    vz += gg * dz;
                    gm += inv3 * lj;
                }
            }
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
            if (tid == 0 && u + STAGES < u1) {
                const long long jt = (u + STAGES) % n_jt;
                mbar_arrive_expect_tx(&full[stage], K::TILE_BYTES);
                bulk_load(tiles + stage * 2 * JT, bw + jt * 2LL * JT, K::TILE_BYTES, &full[stage]);
            }
            if (++stage == STAGES) {
                stage = 0;
                parity ^= 1u;
            }
        }
        if (bad) break;
        const long long sidx = g - sk_owner(it * n_jt, W, G);
        part[(it * L.S_max + sidx) * (long long)K::ITILE + tid] =
            make_double4(pi.w * ux - bm * wi.x - 3.0 * vx, pi.w * uy - bm * wi.y - 3.0 * vy,
                         pi.w * uz - bm * wi.z - 3.0 * vz, -gm);
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

// ------------------------------------------------------------------ packing
// (x, y, z, m) and co-vector w into the FP32 VJP layout; w = scale * wsrc.
__device__ __forceinline__ void pkw_store(float *pkw, long long i, float4 b, float wx, float wy,
                                          float wz) {
    float *p = pkw + (i >> 1) * 16 + (i & 1);
    p[0] = b.x;
    p[2] = b.y;
    p[4] = b.z;
    p[6] = b.w;
    p[8] = wx;
    p[10] = wy;
    p[12] = wz;
    p[14] = 0.f;
}

// Segment sums (fixed order) of a VJP launch: float4 (dL/dx, dL/dm).
__device__ __forceinline__ float4 reduce_vjp_f32(const float4 *__restrict__ part,
                                                 const ForceLaunch &L, int itile, long long i) {
    if (L.sym) return reduce_vjp_sym_f32(part, L, itile, i);   // each pair evaluated once
    const long long it = i / itile, il = i - it * itile;
    const long long g0 = sk_owner(it * L.n_jt, L.W, L.G);
    const long long g1 = sk_owner((it + 1) * L.n_jt - 1, L.W, L.G);
    const float4 *p = part + it * L.S_max * (long long)itile + il;
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    for (long long s = 0; s <= g1 - g0; ++s) {
        const float4 v = __ldg(p + s * itile);
        r.x += v.x;
        r.y += v.y;
        r.z += v.z;
        r.w += v.w;
    }
    return r;
}

__device__ __forceinline__ double4 reduce_vjp_f64(const double4 *__restrict__ part,
                                                  const ForceLaunch &L, int itile, long long i) {
    const long long it = i / itile, il = i - it * itile;
    const long long g0 = sk_owner(it * L.n_jt, L.W, L.G);
    const long long g1 = sk_owner((it + 1) * L.n_jt - 1, L.W, L.G);
    const double4 *p = part + it * L.S_max * (long long)itile + il;
    double4 r = make_double4(0.0, 0.0, 0.0, 0.0);
    for (long long s = 0; s <= g1 - g0; ++s) {
        const double4 v = p[s * itile];
        r.x += v.x;
        r.y += v.y;
        r.z += v.z;
        r.w += v.w;
    }
    return r;
}

}  // namespace colatus

namespace colatus {

// --------------------------------------------- element-wise adjoint updates
// Pack bodies with co-vector scale * w (FP32 VJP layout); padding bodies get
// zero mass and zero co-vector.
__global__ void vjp_pack_f32_kernel(const float4 *__restrict__ xs, const float4 *__restrict__ w,
                                    const DevClock *__restrict__ clk, double G, int use_clock,
                                    float *__restrict__ pkw, long long N, long long N_pad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    if (i >= N) {
        pkw_store(pkw, i, make_float4(0.f, 0.f, 0.f, 0.f), 0.f, 0.f, 0.f);
        return;
    }
    float s = 1.f;
    if (use_clock) {
        const double a = clk->a;
        s = (float)(G / (a * a * a));
    }
    const float4 v = w[i];
    pkw_store(pkw, i, xs[i], s * v.x, s * v.y, s * v.z);
}

__global__ void vjp_pack_f64_kernel(const double4 *__restrict__ xs, const double4 *__restrict__ w,
                                    const DevClock *__restrict__ clk, double G, int use_clock,
                                    double4 *__restrict__ bw, long long N, long long N_pad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    if (i >= N) {
        bw[2 * i] = make_double4(0.0, 0.0, 0.0, 0.0);
        bw[2 * i + 1] = make_double4(0.0, 0.0, 0.0, 0.0);
        return;
    }
    double s = 1.0;
    if (use_clock) {
        const double a = clk->a;
        s = G / (a * a * a);
    }
    const double4 v = w[i];
    bw[2 * i] = xs[i];
    bw[2 * i + 1] = make_double4(s * v.x, s * v.y, s * v.z, 0.0);
}

// gx (N x 3) and gm (N) of one VJP launch, in the caller's dtype.
template <typename T4, typename T>
__device__ __forceinline__ void store_grad(void *gx, void *gm, int out_f64, long long i, T gxx, T gxy,
                                           T gxz, T gmm) {
    if (out_f64) {
        if (gx) {
            double *o = static_cast<double *>(gx) + 3 * i;
            o[0] = gxx;
            o[1] = gxy;
            o[2] = gxz;
        }
        if (gm) static_cast<double *>(gm)[i] = gmm;
    } else {
        if (gx) {
            float *o = static_cast<float *>(gx) + 3 * i;
            o[0] = (float)gxx;
            o[1] = (float)gxy;
            o[2] = (float)gxz;
        }
        if (gm) static_cast<float *>(gm)[i] = (float)gmm;
    }
}

// Bodies and co-vector of entry i of the packed VJP input.
__device__ __forceinline__ void pkw_load(const float *pkw, long long i, float &x, float &y, float &z,
                                         float &wx, float &wy, float &wz) {
    const float *p = pkw + (i >> 1) * 16 + (i & 1);
    x = p[0];
    y = p[2];
    z = p[4];
    wx = p[8];
    wy = p[10];
    wz = p[12];
}

__global__ void vjp_out_f32_kernel(const float4 *__restrict__ part, ForceLaunch L, int itile,
                                   long long N, void *gx, void *gm, int out_f64,
                                   const float *__restrict__ pkw, Extra D) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    float4 g = reduce_vjp_f32(part, L, itile, i);
    add_kspace_vjp(D, i, g);
    if (D.on) {
        float x, y, z, wx, wy, wz;
        pkw_load(pkw, i, x, y, z, wx, wy, wz);
        defo_jacobian<float>(D, x, y, z, wx, wy, wz, g.x, g.y, g.z);
    }
    store_grad<float4, float>(gx, gm, out_f64, i, g.x, g.y, g.z, g.w);
}

__global__ void vjp_out_f64_kernel(const double4 *__restrict__ part, ForceLaunch L, int itile,
                                   long long N, void *gx, void *gm, int out_f64,
                                   const double4 *__restrict__ bw, Extra D) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double4 g = reduce_vjp_f64(part, L, itile, i);
    add_kspace_vjp(D, i, g);
    if (D.on) {
        const double4 p = bw[2 * i], w = bw[2 * i + 1];
        defo_jacobian<double>(D, p.x, p.y, p.z, w.x, w.y, w.z, g.x, g.y, g.z);
    }
    store_grad<double4, double>(gx, gm, out_f64, i, g.x, g.y, g.z, g.w);
}

// Discrete adjoint of the KDK step (Eqs. 3-5 with the KDK reading):
//   vh_n = c1_n v_n + d1_n F(x_n);  x_{n+1} = x_n + tau vh_n;
//   v_{n+1} = c2_n vh_n + d2_n F(x_{n+1}).
// F(x_n) enters step n (through d1_n) and step n-1 (through d2_{n-1}), so
// one VJP per position carries the co-vector
//   W_n = d2_{n-1} lv_n + d1_n lvh_n     (W_N = d2_{N-1} lv_N,  W_0 = d1_0 lvh_0).
// After the VJP at x_{n+1} with W_{n+1} (gradient g):
//   lx += g_x;  lm += g_m;  lvh_n = c2_n lv_{n+1} + tau lx;  lv_n = c1_n lvh_n,
// and the bodies at x_n are packed with W_n for the next VJP.

// Start: lambdas from the loss gradient; pack x_N with W_N.
template <typename T4, typename T>
__device__ __forceinline__ T4 load3(const void *p, int f64, long long i) {
    T4 r;
    if (!p) {
        r.x = r.y = r.z = 0;
    } else if (f64) {
        const double *q = static_cast<const double *>(p) + 3 * i;
        r.x = (T)q[0];
        r.y = (T)q[1];
        r.z = (T)q[2];
    } else {
        const float *q = static_cast<const float *>(p) + 3 * i;
        r.x = (T)q[0];
        r.y = (T)q[1];
        r.z = (T)q[2];
    }
    r.w = 0;
    return r;
}

__global__ void adj_init_f32_kernel(const void *gxT, const void *gvT, const void *gmT, int in_f64,
                                    const float4 *__restrict__ xN, float4 *lx, float4 *lv,
                                    float *lm, const StepCoef *__restrict__ table, long long last,
                                    float *pkw, long long N, long long N_pad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    if (i >= N) {
        pkw_store(pkw, i, make_float4(0.f, 0.f, 0.f, 0.f), 0.f, 0.f, 0.f);
        return;
    }
    const float4 ax = load3<float4, float>(gxT, in_f64, i);
    const float4 av = load3<float4, float>(gvT, in_f64, i);
    lx[i] = ax;
    lv[i] = av;
    lm[i] = gmT ? (in_f64 ? (float)static_cast<const double *>(gmT)[i] : static_cast<const float *>(gmT)[i])
                : 0.f;
    const float d2 = (float)table[last].d2;
    pkw_store(pkw, i, xN[i], d2 * av.x, d2 * av.y, d2 * av.z);
}

__global__ void adj_step_f32_kernel(const float4 *__restrict__ part, ForceLaunch L, int itile,
                                    const float4 *__restrict__ xn, float4 *lx, float4 *lv,
                                    float4 *lvh, float *lm, const StepCoef *__restrict__ table,
                                    long long n, double tau, float *pkw, long long N,
                                    long long N_pad, Extra D) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    if (i >= N) {
        pkw_store(pkw, i, make_float4(0.f, 0.f, 0.f, 0.f), 0.f, 0.f, 0.f);
        return;
    }
    float4 g = reduce_vjp_f32(part, L, itile, i);
    add_kspace_vjp(D, i, g);
    if (D.eqf) {   // the equal-mass VJP's -W_{n+1} . F(x_{n+1}) / m (W still in pkw)
        float x, y, z, wx, wy, wz;
        pkw_load(pkw, i, x, y, z, wx, wy, wz);
        add_eqm_vjp(D, i, wx, wy, wz, g);
    }
    if (D.on) {   // deformation term at x_{n+1} with W_{n+1} (still in pkw)
        float x, y, z, wx, wy, wz;
        pkw_load(pkw, i, x, y, z, wx, wy, wz);
        defo_jacobian<float>(D, x, y, z, wx, wy, wz, g.x, g.y, g.z);
    }
    float4 ax = lx[i];
    ax.x += g.x;
    ax.y += g.y;
    ax.z += g.z;
    lx[i] = ax;
    lm[i] += g.w;
    const StepCoef &e = table[n];
    const float c1 = (float)e.c1, d1 = (float)e.d1, c2 = (float)e.c2, t = (float)tau;
    const float4 av = lv[i];
    const float hx = c2 * av.x + t * ax.x, hy = c2 * av.y + t * ax.y, hz = c2 * av.z + t * ax.z;
    const float vx = c1 * hx, vy = c1 * hy, vz = c1 * hz;
    lvh[i] = make_float4(hx, hy, hz, 0.f);
    lv[i] = make_float4(vx, vy, vz, 0.f);
    const float dp = n > 0 ? (float)table[n - 1].d2 : 0.f;
    pkw_store(pkw, i, xn[i], dp * vx + d1 * hx, dp * vy + d1 * hy, dp * vz + d1 * hz);
}

__global__ void adj_final_f32_kernel(const float4 *__restrict__ part, ForceLaunch L, int itile,
                                     float4 *lx, float *lm, long long N,
                                     const float *__restrict__ pkw, Extra D) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    float4 g = reduce_vjp_f32(part, L, itile, i);
    add_kspace_vjp(D, i, g);
    if (D.eqf) {
        float x, y, z, wx, wy, wz;
        pkw_load(pkw, i, x, y, z, wx, wy, wz);
        add_eqm_vjp(D, i, wx, wy, wz, g);
    }
    if (D.on) {
        float x, y, z, wx, wy, wz;
        pkw_load(pkw, i, x, y, z, wx, wy, wz);
        defo_jacobian<float>(D, x, y, z, wx, wy, wz, g.x, g.y, g.z);
    }
    float4 ax = lx[i];
    ax.x += g.x;
    ax.y += g.y;
    ax.z += g.z;
    lx[i] = ax;
    lm[i] += g.w;
}

__global__ void adj_init_f64_kernel(const void *gxT, const void *gvT, const void *gmT, int in_f64,
                                    const double4 *__restrict__ xN, double4 *lx, double4 *lv,
                                    double *lm, const StepCoef *__restrict__ table, long long last,
                                    double4 *bw, long long N, long long N_pad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    if (i >= N) {
        bw[2 * i] = make_double4(0.0, 0.0, 0.0, 0.0);
        bw[2 * i + 1] = make_double4(0.0, 0.0, 0.0, 0.0);
        return;
    }
    const double4 ax = load3<double4, double>(gxT, in_f64, i);
    const double4 av = load3<double4, double>(gvT, in_f64, i);
    lx[i] = ax;
    lv[i] = av;
    lm[i] = gmT ? (in_f64 ? static_cast<const double *>(gmT)[i] : (double)static_cast<const float *>(gmT)[i])
                : 0.0;
    const double d2 = table[last].d2;
    bw[2 * i] = xN[i];
    bw[2 * i + 1] = make_double4(d2 * av.x, d2 * av.y, d2 * av.z, 0.0);
}

__global__ void adj_step_f64_kernel(const double4 *__restrict__ part, ForceLaunch L, int itile,
                                    const double4 *__restrict__ xn, double4 *lx, double4 *lv,
                                    double4 *lvh, double *lm, const StepCoef *__restrict__ table,
                                    long long n, double tau, double4 *bw, long long N,
                                    long long N_pad, Extra D) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    if (i >= N) {
        bw[2 * i] = make_double4(0.0, 0.0, 0.0, 0.0);
        bw[2 * i + 1] = make_double4(0.0, 0.0, 0.0, 0.0);
        return;
    }
    double4 g = reduce_vjp_f64(part, L, itile, i);
    add_kspace_vjp(D, i, g);
    if (D.on) {
        const double4 p = bw[2 * i], w = bw[2 * i + 1];
        defo_jacobian<double>(D, p.x, p.y, p.z, w.x, w.y, w.z, g.x, g.y, g.z);
    }
    double4 ax = lx[i];
    ax.x += g.x;
    ax.y += g.y;
    ax.z += g.z;
    lx[i] = ax;
    lm[i] += g.w;
    const StepCoef &e = table[n];
    const double4 av = lv[i];
    const double hx = e.c2 * av.x + tau * ax.x, hy = e.c2 * av.y + tau * ax.y,
                 hz = e.c2 * av.z + tau * ax.z;
    const double vx = e.c1 * hx, vy = e.c1 * hy, vz = e.c1 * hz;
    lvh[i] = make_double4(hx, hy, hz, 0.0);
    lv[i] = make_double4(vx, vy, vz, 0.0);
    const double dp = n > 0 ? table[n - 1].d2 : 0.0;
    bw[2 * i] = xn[i];
    bw[2 * i + 1] = make_double4(dp * vx + e.d1 * hx, dp * vy + e.d1 * hy, dp * vz + e.d1 * hz, 0.0);
}

__global__ void adj_final_f64_kernel(const double4 *__restrict__ part, ForceLaunch L, int itile,
                                     double4 *lx, double *lm, long long N,
                                     const double4 *__restrict__ bw, Extra D) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double4 g = reduce_vjp_f64(part, L, itile, i);
    add_kspace_vjp(D, i, g);
    if (D.on) {
        const double4 p = bw[2 * i], w = bw[2 * i + 1];
        defo_jacobian<double>(D, p.x, p.y, p.z, w.x, w.y, w.z, g.x, g.y, g.z);
    }
    double4 ax = lx[i];
    ax.x += g.x;
    ax.y += g.y;
    ax.z += g.z;
    lx[i] = ax;
    lm[i] += g.w;
}

// ------------------------------------------------ adjoint of the DKD leapfrog
// Forward step n (Eqs. 3-5; c_n, d_n at t^{n+1/2}):
//   xh_n = x_n + (tau/2) v_n;  v_{n+1} = c_n v_n + d_n F(xh_n);
//   x_{n+1} = xh_n + (tau/2) v_{n+1}.
// Its transpose, from the adjoints (lx, lv) of step n+1:
//   lvt = lv + (tau/2) lx;  W_n = d_n lvt;  (g_x, g_m) = VJP at xh_n with W_n;
//   lx_n = lx + g_x;  lm += g_m;  lv_n = c_n lvt + (tau/2) lx_n.
// Two element-wise kernels per step bracket the VJP: the pack of (xh_n, W_n),
// with xh_n formed by the forward's own half drift (bitwise the position the
// forward evaluated F at), and the update.
__global__ void dkd_adj_pack_f32_kernel(const float4 *__restrict__ xn, const float4 *__restrict__ vn,
                                        const float4 *__restrict__ lx, const float4 *__restrict__ lv,
                                        const StepCoef *__restrict__ table, long long n, double tau,
                                        float *pkw, long long N, long long N_pad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    if (i >= N) {
        pkw_store(pkw, i, make_float4(0.f, 0.f, 0.f, 0.f), 0.f, 0.f, 0.f);
        return;
    }
    const float h = (float)(0.5 * tau), d = (float)table[n].d;
    const float4 x = xn[i], v = vn[i], ax = lx[i], av = lv[i];
    const float4 xh = make_float4(drift1(x.x, h, v.x), drift1(x.y, h, v.y), drift1(x.z, h, v.z), x.w);
    pkw_store(pkw, i, xh, d * drift1(av.x, h, ax.x), d * drift1(av.y, h, ax.y), d * drift1(av.z, h, ax.z));
}

__global__ void dkd_adj_update_f32_kernel(const float4 *__restrict__ part, ForceLaunch L, int itile,
                                          float4 *lx, float4 *lv, float *lm,
                                          const StepCoef *__restrict__ table, long long n, double tau,
                                          const float *__restrict__ pkw, long long N, Extra D) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    float4 g = reduce_vjp_f32(part, L, itile, i);
    add_kspace_vjp(D, i, g);
    if (D.on) {   // deformation term at xh_n with W_n (in pkw)
        float x, y, z, wx, wy, wz;
        pkw_load(pkw, i, x, y, z, wx, wy, wz);
        defo_jacobian<float>(D, x, y, z, wx, wy, wz, g.x, g.y, g.z);
    }
    const float h = (float)(0.5 * tau), c = (float)table[n].c;
    const float4 ax = lx[i], av = lv[i];
    const float tx = drift1(av.x, h, ax.x), ty = drift1(av.y, h, ax.y), tz = drift1(av.z, h, ax.z);
    const float nx = ax.x + g.x, ny = ax.y + g.y, nz = ax.z + g.z;
    lx[i] = make_float4(nx, ny, nz, 0.f);
    lv[i] = make_float4(kick2(c, tx, h, nx), kick2(c, ty, h, ny), kick2(c, tz, h, nz), 0.f);
    lm[i] += g.w;
}

__global__ void dkd_adj_pack_f64_kernel(const double4 *__restrict__ xn, const double4 *__restrict__ vn,
                                        const double4 *__restrict__ lx, const double4 *__restrict__ lv,
                                        const StepCoef *__restrict__ table, long long n, double tau,
                                        double4 *bw, long long N, long long N_pad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    if (i >= N) {
        bw[2 * i] = make_double4(0.0, 0.0, 0.0, 0.0);
        bw[2 * i + 1] = make_double4(0.0, 0.0, 0.0, 0.0);
        return;
    }
    const double h = 0.5 * tau, d = table[n].d;
    const double4 x = xn[i], v = vn[i], ax = lx[i], av = lv[i];
    bw[2 * i] = make_double4(drift1(x.x, h, v.x), drift1(x.y, h, v.y), drift1(x.z, h, v.z), x.w);
    bw[2 * i + 1] = make_double4(d * drift1(av.x, h, ax.x), d * drift1(av.y, h, ax.y),
                                 d * drift1(av.z, h, ax.z), 0.0);
}

__global__ void dkd_adj_update_f64_kernel(const double4 *__restrict__ part, ForceLaunch L, int itile,
                                          double4 *lx, double4 *lv, double *lm,
                                          const StepCoef *__restrict__ table, long long n, double tau,
                                          const double4 *__restrict__ bw, long long N, Extra D) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double4 g = reduce_vjp_f64(part, L, itile, i);
    add_kspace_vjp(D, i, g);
    if (D.on) {
        const double4 p = bw[2 * i], w = bw[2 * i + 1];
        defo_jacobian<double>(D, p.x, p.y, p.z, w.x, w.y, w.z, g.x, g.y, g.z);
    }
    const double h = 0.5 * tau, c = table[n].c;
    const double4 ax = lx[i], av = lv[i];
    const double tx = drift1(av.x, h, ax.x), ty = drift1(av.y, h, ax.y), tz = drift1(av.z, h, ax.z);
    const double nx = ax.x + g.x, ny = ax.y + g.y, nz = ax.z + g.z;
    lx[i] = make_double4(nx, ny, nz, 0.0);
    lv[i] = make_double4(kick2(c, tx, h, nx), kick2(c, ty, h, ny), kick2(c, tz, h, nz), 0.0);
    lm[i] += g.w;
}

// Adjoint results in the caller's dtype: gx (N x 3), gv (N x 3), gm (N).
template <typename T4, typename T>
__global__ void adj_store_kernel(const T4 *__restrict__ lx, const T4 *__restrict__ lv,
                                 const T *__restrict__ lm, long long N, void *gx, void *gv,
                                 void *gm, int out_f64) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const T4 a = lx[i], b = lv[i];
    store_grad<T4, T>(gx, gm, out_f64, i, a.x, a.y, a.z, lm[i]);
    store_grad<T4, T>(gv, nullptr, out_f64, i, b.x, b.y, b.z, (T)0);
}

}  // namespace colatus
