// vjp_sym.cuh -- the equal-mass VJP of the all-pairs force with every pair
// evaluated once.
//
// With every mass m, the VJP of Eq. 1 (see adjoint.cuh) at body i is
//   dL/dx_i = m sum_j [ inv^3 u - 3 inv^5 (u . d) d ],
//   dL/dm_i = -sum_j inv^3 (u . d) - w_i . P_i,
// with d = x_j - x_i, u = w_j - w_i, inv = (|d|^2 + eps^2)^{-1/2} and P_i the
// (G-less) force per unit mass that the forward pass computed.  Swapping i and
// j flips both d and u, so the position term of the pair (i, j) is minus the
// one of (j, i) and the mass term is the same for both: one evaluation of
//   s = u - 3 inv^2 (u . d) d,   t = inv^3 s,   g = inv^3 (u . d)
// adds (m t, -g) to body i and (-m t, -g) to body j.  That is 27 FP32 lane-ops
// per pair and one MUFU.RSQ, against 2 x 23 when each ordered pair is taken
// on its own (vjp_eqm_f32_kernel), and the self pair is exactly 0 (u = 0).
//
// Decomposition, tables and pipeline are those of force_sym.cuh (tile pairs
// it <= jt, NW phases per unit, j-pairs rotating through the lanes with their
// sums, column slots added by the consumers in fixed order); the bodies come
// in the VJP's layout, 32 bytes per body, pair-interleaved
// [x0 x1 y0 y1 z0 z1 m0 m1 wx0 wx1 wy0 wy1 wz0 wz1 0 0], and a j-tile is
// split into (x0 x1 y0 y1), (z0 z1 wx0 wx1), (wy0 wy1 wz0 wz1), each 32-pair
// block stored twice.  Segments hold float4 (dL/dx, dL/dm without the force
// term), one plane, summed in FP32 like the other FP32 VJP kernels.
#pragma once

#include "force_sym.cuh"

namespace colatus {

template <int NT>
struct VjpSymKernel {
    static constexpr int IPT = 4;
    static constexpr int NW = NT / 32;
    static constexpr int T = NT * IPT;        // bodies per tile
    static constexpr int TP = T / 2;          // j-pairs per tile
    static constexpr int SLICE = TP / NW;     // j-pairs per warp slice
    static constexpr int ROT = SLICE / 32;    // 32-round rotations per phase
    static constexpr uint32_t TILE_BYTES = T * 32;
    // staging tile, three doubled split arrays, the column accumulators
    // [t_x t_y t_z g][TP] float2, one mbarrier
    static constexpr int SMEM = TILE_BYTES + 3 * 2 * TP * 16 + 4 * TP * 8 + 16;
    static_assert(SLICE % 32 == 0, "a warp slice is whole rotations");
};

// One 32-round rotation over a doubled block (see sym_rotation): every lane's
// 4 i-bodies against every j-pair.  SYM: the j-side sums travel with their
// j-pairs and end, in lane l, as those of j-pair base + l.
template <bool SYM, int UNR>
__device__ __forceinline__ void vjp_sym_rotation(const float4 *__restrict__ sA, const float4 *__restrict__ sB,
                                                 const float4 *__restrict__ sC, int lane,
                                                 const float2 (&nx)[4], const float2 (&ny)[4],
                                                 const float2 (&nz)[4], const float2 (&nwx)[4],
                                                 const float2 (&nwy)[4], const float2 (&nwz)[4],
                                                 const float2 e2, float2 (&tx)[4], float2 (&ty)[4],
                                                 float2 (&tz)[4], float2 (&tg)[4], float2 &jx, float2 &jy,
                                                 float2 &jz, float2 &jg) {
    const int src = (lane + 1) & 31;
    const float2 n3 = make_float2(-3.f, -3.f);
    const float4 *a = sA + lane, *b = sB + lane, *c = sC + lane;
#pragma unroll(UNR)
    for (int r = 0; r < 32; ++r) {
        const float4 A = a[r];   // x0 x1 y0 y1
        const float4 Bq = b[r];  // z0 z1 wx0 wx1
        const float4 C = c[r];   // wy0 wy1 wz0 wz1
        const float2 xj = make_float2(A.x, A.y), yj = make_float2(A.z, A.w);
        const float2 zj = make_float2(Bq.x, Bq.y), wxj = make_float2(Bq.z, Bq.w);
        const float2 wyj = make_float2(C.x, C.y), wzj = make_float2(C.z, C.w);
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
            const float2 ux = __fadd2_rn(wxj, nwx[k]);
            const float2 uy = __fadd2_rn(wyj, nwy[k]);
            const float2 uz = __fadd2_rn(wzj, nwz[k]);
            float2 du = __fmul2_rn(ux, dx);
            du = __ffma2_rn(uy, dy, du);
            du = __ffma2_rn(uz, dz, du);
            const float2 q = __fmul2_rn(__fmul2_rn(inv2, du), n3);
            const float2 sx = __ffma2_rn(q, dx, ux);
            const float2 sy = __ffma2_rn(q, dy, uy);
            const float2 sz = __ffma2_rn(q, dz, uz);
            tx[k] = __ffma2_rn(inv3, sx, tx[k]);
            ty[k] = __ffma2_rn(inv3, sy, ty[k]);
            tz[k] = __ffma2_rn(inv3, sz, tz[k]);
            tg[k] = __ffma2_rn(inv3, du, tg[k]);
            if (SYM) {
                jx = __ffma2_rn(inv3, sx, jx);
                jy = __ffma2_rn(inv3, sy, jy);
                jz = __ffma2_rn(inv3, sz, jz);
                jg = __ffma2_rn(inv3, du, jg);
            }
        }
        if (SYM) {
            jx = shfl_float2(jx, src);
            jy = shfl_float2(jy, src);
            jz = shfl_float2(jz, src);
            jg = shfl_float2(jg, src);
        }
    }
}

// Persistent pair-once equal-mass VJP kernel, FP32.  pkw: bodies and
// co-vectors in the VJP layout (N_pad a multiple of T, and no zero-mass
// padding: N_pad = N).  part: row segments [n][S_max][T] float4, then from
// float4 offset L.col_off the column slots [slot][T] float4, each float4
// (m sum t, -sum g) of the bodies it indexes (the column's position part
// negated when written).  mass: the common mass m.
template <int NT, int UNR>
__global__ void __launch_bounds__(NT, 1)
    vjp_sym_eqm_f32_kernel(const float *__restrict__ pkw, float4 *__restrict__ part, int *__restrict__ flags,
                           ForceLaunch L, float eps2, float mass) {
    using K = VjpSymKernel<NT>;
    constexpr int NW = K::NW, T = K::T, TP = K::TP;
    extern __shared__ __align__(128) unsigned char smem[];
    float4 *raw = reinterpret_cast<float4 *>(smem);   // staging: 2 T float4 (VJP layout)
    float4 *sA = raw + 2 * T;                         // 2 TP float4 each, blocks doubled
    float4 *sB = sA + 2 * TP;
    float4 *sC = sB + 2 * TP;
    float2 *acc = reinterpret_cast<float2 *>(sC + 2 * TP);   // [4][TP]
    uint64_t *bar = reinterpret_cast<uint64_t *>(acc + 4 * TP);

    const SymTab S(L.sym);
    const int n = S.n;
    const int *row_g0 = S.row_g0, *unit_g0 = S.unit_g0, *unit_ko = S.unit_ko, *cta_pu = S.cta_pu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = blockIdx.x;
    int pu = cta_pu[g];
    const int pu_end = cta_pu[g + 1];
    if (pu >= pu_end) return;
    long long u = pu / NW;
    int it, jt;
    sym_decode(u, n, it, jt);

    for (int q = tid; q < 4 * TP; q += NT) acc[q] = make_float2(0.f, 0.f);
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(bar, K::TILE_BYTES);
        bulk_load(raw, pkw + (long long)jt * T * 8, K::TILE_BYTES, bar);
    }
    bool inflight = true;

    const float2 e2 = make_float2(eps2, eps2);
    float2 nx[4], ny[4], nz[4], nwx[4], nwy[4], nwz[4];
    float hx[4], hy[4], hz[4], hg[4];
    auto load_i = [&](int row) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long long i = (long long)row * T + tid + k * NT;
            const float *p = pkw + (i >> 1) * 16 + (i & 1);
            const float x = __ldg(p), y = __ldg(p + 2), z = __ldg(p + 4);
            const float wx = __ldg(p + 8), wy = __ldg(p + 10), wz = __ldg(p + 12);
            nx[k] = make_float2(-x, -x);
            ny[k] = make_float2(-y, -y);
            nz[k] = make_float2(-z, -z);
            nwx[k] = make_float2(-wx, -wx);
            nwy[k] = make_float2(-wy, -wy);
            nwz[k] = make_float2(-wz, -wz);
            hx[k] = hy[k] = hz[k] = hg[k] = 0.f;
        }
    };
    load_i(it);

    uint32_t parity = 0;
    bool bad = false;
    while (pu < pu_end) {
        const int uend = (int)min((long long)pu_end, (u + 1) * NW);
        const int p0 = pu - (int)(u * NW), p1 = uend - (int)(u * NW);
        const bool ok = mbar_wait_bounded(bar, parity);
        if (__syncthreads_or(!ok)) {
            bad = true;
            break;
        }
        inflight = false;
        parity ^= 1u;
        for (int q = tid; q < TP; q += NT) {
            const int e = 2 * q - (q & 31);   // entry of pair q in its doubled block
            const float4 r0 = raw[4 * q], r1 = raw[4 * q + 1], r2 = raw[4 * q + 2], r3 = raw[4 * q + 3];
            const float4 Bq = make_float4(r1.x, r1.y, r2.x, r2.y);
            const float4 C = make_float4(r2.z, r2.w, r3.x, r3.y);
            sA[e] = r0;
            sA[e + 32] = r0;
            sB[e] = Bq;
            sB[e + 32] = Bq;
            sC[e] = C;
            sC[e + 32] = C;
        }
        __syncthreads();
        int it_n = it, jt_n = jt + 1;
        if (jt_n == n) {
            ++it_n;
            jt_n = it_n;
        }
        if (uend < pu_end) {
            if (tid == 0) {
                mbar_arrive_expect_tx(bar, K::TILE_BYTES);
                bulk_load(raw, pkw + (long long)jt_n * T * 8, K::TILE_BYTES, bar);
            }
            inflight = true;
        }
        const bool sym = jt != it;
        for (int p = p0; p < p1; ++p) {
            const int slice = (warp + p) % NW;
            float2 tx[4], ty[4], tz[4], tg[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) tx[k] = ty[k] = tz[k] = tg[k] = make_float2(0.f, 0.f);
#pragma unroll 1
            for (int s = 0; s < K::ROT; ++s) {
                const int base = slice * K::SLICE + s * 32;
                const float4 *bA = sA + 2 * base, *bB = sB + 2 * base, *bC = sC + 2 * base;
                float2 jx = make_float2(0.f, 0.f), jy = jx, jz = jx, jg = jx;
                if (sym) {
                    vjp_sym_rotation<true, UNR>(bA, bB, bC, lane, nx, ny, nz, nwx, nwy, nwz, e2, tx, ty, tz,
                                                tg, jx, jy, jz, jg);
                    const int q = base + lane;
                    acc[q] = __fadd2_rn(acc[q], jx);
                    acc[TP + q] = __fadd2_rn(acc[TP + q], jy);
                    acc[2 * TP + q] = __fadd2_rn(acc[2 * TP + q], jz);
                    acc[3 * TP + q] = __fadd2_rn(acc[3 * TP + q], jg);
                } else {
                    vjp_sym_rotation<false, UNR>(bA, bB, bC, lane, nx, ny, nz, nwx, nwy, nwz, e2, tx, ty, tz,
                                                 tg, jx, jy, jz, jg);
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                hx[k] += tx[k].x + tx[k].y;
                hy[k] += ty[k].x + ty[k].y;
                hz[k] += tz[k].x + tz[k].y;
                hg[k] += tg[k].x + tg[k].y;
            }
            __syncthreads();   // the slices change hands
        }
        if (sym) {
            const int slot = unit_ko[u] + (g - unit_g0[u]);
            float4 *dst = part + L.col_off + (long long)slot * T;
            for (int q = tid; q < TP; q += NT) {
                const float2 a = acc[q], b = acc[TP + q], c = acc[2 * TP + q], d = acc[3 * TP + q];
                dst[2 * q] = make_float4(-mass * a.x, -mass * b.x, -mass * c.x, -d.x);
                dst[2 * q + 1] = make_float4(-mass * a.y, -mass * b.y, -mass * c.y, -d.y);
                acc[q] = acc[TP + q] = acc[2 * TP + q] = acc[3 * TP + q] = make_float2(0.f, 0.f);
            }
            __syncthreads();
        }
        pu = uend;
        ++u;
        if (it_n != it || pu == pu_end) {
            const int sidx = g - row_g0[it];
            float4 *dst = part + ((long long)it * L.S_max + sidx) * T;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                dst[tid + k * NT] = make_float4(mass * hx[k], mass * hy[k], mass * hz[k], -hg[k]);
            if (it_n != it && pu < pu_end) load_i(it_n);
        }
        it = it_n;
        jt = jt_n;
    }
    if (bad && tid == 0) {
        atomicOr(&flags[FLAG_TIMEOUT], 1);
        if (inflight) mbar_wait_bounded(bar, parity);   // drain the copy in flight, bounded
    }
}

// ---- general masses
// The VJP of Eq. 1 at body i with any masses (adjoint.cuh):
//   dL/dx_i = sum_j J(d) u',  u' = m_i w_j - m_j w_i,  J(d) = inv^3 (I - 3 inv^2 d d^T),
//   dL/dm_i = -sum_j inv^3 (w_j . d),
// d = x_j - x_i.  Swapping i and j flips d and u', so the position term is
// antisymmetric; the mass terms of the pair are -inv^3 (w_j . d) on i and
// +inv^3 (w_i . d) on j.  One evaluation of
//   s = u' - 3 inv^2 (u' . d) d
// adds (inv^3 s, -inv^3 (w_j . d)) to body i and (-inv^3 s, inv^3 (w_i . d))
// to body j: 40 FP32 lane-ops per pair and one MUFU.RSQ, against 2 x 25 for
// the per-ordered-pair kernel's scaled form.  u' is formed as
//   u' = m_j (w_j - w_i) + (m_i - m_j) w_j:
// the difference of the co-vectors first, so that with equal masses u' is
// that difference times m (the second term exactly 0), its rounding as
// well conditioned as in the equal-mass form; a body's own pair and a
// padding body j (zero mass and co-vector) give exactly 0.  The product form
// m_i w_j - m_j w_i would leave the rounding of m_j w_i, an error that
// depends on i alone and so adds up coherently over every j (measured: 50x
// the per-ordered-pair kernel's error in a DKD adjoint).
// EQM (every mass m, no padding): u' = m (w_j - w_i), the factor m applied to
// the position sums when they are written, and w_j . d taken as
// (w_j - w_i) . d + w_i . d: 31 lane-ops per pair.
// The pair term is a policy P (J = b I + c d d^T): PlummerVjpPair here (Eq. 1),
// EwaldVjpPair (ewald_adjoint.cuh) for the real-space term of the periodic
// force, whose separations take the minimum image.

template <int NT>
struct VjpSymGenKernel {
    static constexpr int IPT = 4;
    static constexpr int NW = NT / 32;
    static constexpr int T = NT * IPT;
    static constexpr int TP = T / 2;
    static constexpr int SLICE = TP / NW;
    static constexpr int ROT = SLICE / 32;
    static constexpr uint32_t TILE_BYTES = T * 32;
    // staging tile; (x0 x1 y0 y1), (z0 z1 m0 m1), (wx0 wx1 wy0 wy1) doubled,
    // float4 each; (wz0 wz1) doubled, float2; the column sums [t_x t_y t_z g][TP]
    // float2; one mbarrier
    static constexpr int SMEM = TILE_BYTES + 3 * 2 * TP * 16 + 2 * TP * 8 + 4 * TP * 8 + 16;
    static_assert(SLICE % 32 == 0, "a warp slice is whole rotations");
};

// Pair policy of Eq. 1: J(d) = inv^3 (I - 3 inv^2 d d^T), inv = (r^2+eps^2)^-1/2.
// factors() fills the pair's factors (d unchanged); bw() is b, the weight of
// the mass terms; position() adds J u' to the row sums t and, SYM, to the
// column sums j, as inv^3 s with s = u' - 3 inv^2 (u'.d) d.
struct PlummerVjpPair {
    struct Args {};
    struct F {
        float2 inv2, inv3;
    };
    __device__ __forceinline__ static F factors(float2 &dx, float2 &dy, float2 &dz, const float2 e2, const Args &) {
        float2 r2 = __ffma2_rn(dx, dx, e2);
        r2 = __ffma2_rn(dy, dy, r2);
        r2 = __ffma2_rn(dz, dz, r2);
        const float2 inv = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
        F f;
        f.inv2 = __fmul2_rn(inv, inv);
        f.inv3 = __fmul2_rn(inv, f.inv2);
        return f;
    }
    __device__ __forceinline__ static float2 bw(const F &f) { return f.inv3; }
    template <bool SYM>
    __device__ __forceinline__ static void position(const F &f, const float2 dx, const float2 dy, const float2 dz,
                                                    const float2 ux, const float2 uy, const float2 uz,
                                                    const float2 du, float2 &tx, float2 &ty, float2 &tz, float2 &jx,
                                                    float2 &jy, float2 &jz) {
        const float2 q = __fmul2_rn(__fmul2_rn(f.inv2, du), make_float2(-3.f, -3.f));
        const float2 sx = __ffma2_rn(q, dx, ux);
        const float2 sy = __ffma2_rn(q, dy, uy);
        const float2 sz = __ffma2_rn(q, dz, uz);
        tx = __ffma2_rn(f.inv3, sx, tx);
        ty = __ffma2_rn(f.inv3, sy, ty);
        tz = __ffma2_rn(f.inv3, sz, tz);
        if (SYM) {
            jx = __ffma2_rn(f.inv3, sx, jx);
            jy = __ffma2_rn(f.inv3, sy, jy);
            jz = __ffma2_rn(f.inv3, sz, jz);
        }
    }
};

template <typename P, bool SYM, bool EQM, int UNR>
__device__ __forceinline__ void vjp_gen_rotation(const float4 *__restrict__ sA, const float4 *__restrict__ sB,
                                                 const float4 *__restrict__ sC, const float2 *__restrict__ sD,
                                                 int lane, const float2 (&nx)[4], const float2 (&ny)[4],
                                                 const float2 (&nz)[4], const float2 (&mi)[4],
                                                 const float2 (&wix)[4], const float2 (&wiy)[4],
                                                 const float2 (&wiz)[4], const float2 e2, const typename P::Args &pa,
                                                 float2 (&tx)[4], float2 (&ty)[4], float2 (&tz)[4], float2 (&tg)[4],
                                                 float2 &jx, float2 &jy, float2 &jz, float2 &jg) {
    const int src = (lane + 1) & 31;
    const float4 *a = sA + lane, *b = sB + lane, *c = sC + lane;
    const float2 *dd = sD + lane;
#pragma unroll(UNR)
    for (int r = 0; r < 32; ++r) {
        const float4 A = a[r];   // x0 x1 y0 y1
        const float4 Bq = b[r];  // z0 z1 m0 m1
        const float4 C = c[r];   // wx0 wx1 wy0 wy1
        const float2 wzj = dd[r];
        const float2 xj = make_float2(A.x, A.y), yj = make_float2(A.z, A.w);
        const float2 zj = make_float2(Bq.x, Bq.y), mj = make_float2(Bq.z, Bq.w);
        const float2 wxj = make_float2(C.x, C.y), wyj = make_float2(C.z, C.w);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 dx = __fadd2_rn(xj, nx[k]);
            float2 dy = __fadd2_rn(yj, ny[k]);
            float2 dz = __fadd2_rn(zj, nz[k]);
            const typename P::F f = P::factors(dx, dy, dz, e2, pa);
            const float2 bw = P::bw(f);
            float2 wid = __fmul2_rn(wix[k], dx);
            wid = __ffma2_rn(wiy[k], dy, wid);
            wid = __ffma2_rn(wiz[k], dz, wid);
            float2 ux, uy, uz, du, wjd;
            if (EQM) {
                // u' / m = w_j - w_i;  w_j . d = (w_j - w_i) . d + w_i . d
                ux = __fadd2_rn(wxj, make_float2(-wix[k].x, -wix[k].y));
                uy = __fadd2_rn(wyj, make_float2(-wiy[k].x, -wiy[k].y));
                uz = __fadd2_rn(wzj, make_float2(-wiz[k].x, -wiz[k].y));
                du = __fmul2_rn(ux, dx);
                du = __ffma2_rn(uy, dy, du);
                du = __ffma2_rn(uz, dz, du);
                wjd = __fadd2_rn(du, wid);
            } else {
                wjd = __fmul2_rn(wxj, dx);
                wjd = __ffma2_rn(wyj, dy, wjd);
                wjd = __ffma2_rn(wzj, dz, wjd);
                // u' = m_j (w_j - w_i) + (m_i - m_j) w_j
                const float2 dm = __fadd2_rn(mi[k], make_float2(-mj.x, -mj.y));
                ux = __ffma2_rn(mj, __fadd2_rn(wxj, make_float2(-wix[k].x, -wix[k].y)), __fmul2_rn(dm, wxj));
                uy = __ffma2_rn(mj, __fadd2_rn(wyj, make_float2(-wiy[k].x, -wiy[k].y)), __fmul2_rn(dm, wyj));
                uz = __ffma2_rn(mj, __fadd2_rn(wzj, make_float2(-wiz[k].x, -wiz[k].y)), __fmul2_rn(dm, wzj));
                du = __fmul2_rn(ux, dx);
                du = __ffma2_rn(uy, dy, du);
                du = __ffma2_rn(uz, dz, du);
            }
            P::template position<SYM>(f, dx, dy, dz, ux, uy, uz, du, tx[k], ty[k], tz[k], jx, jy, jz);
            tg[k] = __ffma2_rn(bw, wjd, tg[k]);
            if (SYM) jg = __ffma2_rn(bw, wid, jg);
        }
        if (SYM) {
            jx = shfl_float2(jx, src);
            jy = shfl_float2(jy, src);
            jz = shfl_float2(jz, src);
            jg = shfl_float2(jg, src);
        }
    }
}

// Persistent pair-once VJP kernel for any masses, FP32.  pkw: bodies and
// co-vectors in the VJP layout (N_pad a multiple of T; padding bodies have
// zero mass and co-vector, so they add nothing).  part: row segments
// [n][S_max][T] float4, then from float4 offset L.col_off the column slots
// [slot][T] float4, each float4 (dL/dx, dL/dm) of the bodies it indexes.
// EQM: every body has mass `mass` and no padding enters (N_pad = N).
// P: the pair term (PlummerVjpPair, EwaldVjpPair) and its arguments pa.
template <int NT, int UNR, bool EQM, typename P = PlummerVjpPair>
__global__ void __launch_bounds__(NT, 1)
    vjp_sym_f32_kernel(const float *__restrict__ pkw, float4 *__restrict__ part, int *__restrict__ flags,
                       ForceLaunch L, float eps2, float mass, typename P::Args pa) {
    using K = VjpSymGenKernel<NT>;
    constexpr int NW = K::NW, T = K::T, TP = K::TP;
    extern __shared__ __align__(128) unsigned char smem[];
    float4 *raw = reinterpret_cast<float4 *>(smem);   // staging: 2 T float4 (VJP layout)
    float4 *sA = raw + 2 * T;                         // 2 TP float4 each, blocks doubled
    float4 *sB = sA + 2 * TP;
    float4 *sC = sB + 2 * TP;
    float2 *sD = reinterpret_cast<float2 *>(sC + 2 * TP);   // 2 TP float2
    float2 *acc = sD + 2 * TP;                              // [4][TP]
    uint64_t *bar = reinterpret_cast<uint64_t *>(acc + 4 * TP);

    const SymTab S(L.sym);
    const int n = S.n;
    const int *row_g0 = S.row_g0, *unit_g0 = S.unit_g0, *unit_ko = S.unit_ko, *cta_pu = S.cta_pu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = blockIdx.x;
    int pu = cta_pu[g];
    const int pu_end = cta_pu[g + 1];
    if (pu >= pu_end) return;
    long long u = pu / NW;
    int it, jt;
    sym_decode(u, n, it, jt);

    for (int q = tid; q < 4 * TP; q += NT) acc[q] = make_float2(0.f, 0.f);
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(bar, K::TILE_BYTES);
        bulk_load(raw, pkw + (long long)jt * T * 8, K::TILE_BYTES, bar);
    }
    bool inflight = true;

    const float2 e2 = make_float2(eps2, eps2);
    float2 nx[4], ny[4], nz[4], mi[4], wix[4], wiy[4], wiz[4];
    float hx[4], hy[4], hz[4], hg[4];
    auto load_i = [&](int row) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long long i = (long long)row * T + tid + k * NT;
            const float *p = pkw + (i >> 1) * 16 + (i & 1);
            const float x = __ldg(p), y = __ldg(p + 2), z = __ldg(p + 4), m = __ldg(p + 6);
            const float wx = __ldg(p + 8), wy = __ldg(p + 10), wz = __ldg(p + 12);
            nx[k] = make_float2(-x, -x);
            ny[k] = make_float2(-y, -y);
            nz[k] = make_float2(-z, -z);
            mi[k] = make_float2(m, m);
            wix[k] = make_float2(wx, wx);
            wiy[k] = make_float2(wy, wy);
            wiz[k] = make_float2(wz, wz);
            hx[k] = hy[k] = hz[k] = hg[k] = 0.f;
        }
    };
    load_i(it);

    uint32_t parity = 0;
    bool bad = false;
    while (pu < pu_end) {
        const int uend = (int)min((long long)pu_end, (u + 1) * NW);
        const int p0 = pu - (int)(u * NW), p1 = uend - (int)(u * NW);
        const bool ok = mbar_wait_bounded(bar, parity);
        if (__syncthreads_or(!ok)) {
            bad = true;
            break;
        }
        inflight = false;
        parity ^= 1u;
        for (int q = tid; q < TP; q += NT) {
            const int e = 2 * q - (q & 31);   // entry of pair q in its doubled block
            const float4 r0 = raw[4 * q], r1 = raw[4 * q + 1], r2 = raw[4 * q + 2], r3 = raw[4 * q + 3];
            const float2 D = make_float2(r3.x, r3.y);
            sA[e] = r0;
            sA[e + 32] = r0;
            sB[e] = r1;
            sB[e + 32] = r1;
            sC[e] = r2;
            sC[e + 32] = r2;
            sD[e] = D;
            sD[e + 32] = D;
        }
        __syncthreads();
        int it_n = it, jt_n = jt + 1;
        if (jt_n == n) {
            ++it_n;
            jt_n = it_n;
        }
        if (uend < pu_end) {
            if (tid == 0) {
                mbar_arrive_expect_tx(bar, K::TILE_BYTES);
                bulk_load(raw, pkw + (long long)jt_n * T * 8, K::TILE_BYTES, bar);
            }
            inflight = true;
        }
        const bool sym = jt != it;
        for (int p = p0; p < p1; ++p) {
            const int slice = (warp + p) % NW;
            float2 tx[4], ty[4], tz[4], tg[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) tx[k] = ty[k] = tz[k] = tg[k] = make_float2(0.f, 0.f);
#pragma unroll 1
            for (int s = 0; s < K::ROT; ++s) {
                const int base = slice * K::SLICE + s * 32;
                const float4 *bA = sA + 2 * base, *bB = sB + 2 * base, *bC = sC + 2 * base;
                const float2 *bD = sD + 2 * base;
                float2 jx = make_float2(0.f, 0.f), jy = jx, jz = jx, jg = jx;
                if (sym) {
                    vjp_gen_rotation<P, true, EQM, UNR>(bA, bB, bC, bD, lane, nx, ny, nz, mi, wix, wiy, wiz, e2,
                                                        pa, tx, ty, tz, tg, jx, jy, jz, jg);
                    const int q = base + lane;
                    acc[q] = __fadd2_rn(acc[q], jx);
                    acc[TP + q] = __fadd2_rn(acc[TP + q], jy);
                    acc[2 * TP + q] = __fadd2_rn(acc[2 * TP + q], jz);
                    acc[3 * TP + q] = __fadd2_rn(acc[3 * TP + q], jg);
                } else {
                    vjp_gen_rotation<P, false, EQM, UNR>(bA, bB, bC, bD, lane, nx, ny, nz, mi, wix, wiy, wiz, e2,
                                                         pa, tx, ty, tz, tg, jx, jy, jz, jg);
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                hx[k] += tx[k].x + tx[k].y;
                hy[k] += ty[k].x + ty[k].y;
                hz[k] += tz[k].x + tz[k].y;
                hg[k] += tg[k].x + tg[k].y;
            }
            __syncthreads();   // the slices change hands
        }
        if (sym) {
            const int slot = unit_ko[u] + (g - unit_g0[u]);
            float4 *dst = part + L.col_off + (long long)slot * T;
            const float ms = EQM ? mass : 1.f;
            for (int q = tid; q < TP; q += NT) {
                const float2 a = acc[q], b = acc[TP + q], c = acc[2 * TP + q], d = acc[3 * TP + q];
                dst[2 * q] = make_float4(-ms * a.x, -ms * b.x, -ms * c.x, d.x);
                dst[2 * q + 1] = make_float4(-ms * a.y, -ms * b.y, -ms * c.y, d.y);
                acc[q] = acc[TP + q] = acc[2 * TP + q] = acc[3 * TP + q] = make_float2(0.f, 0.f);
            }
            __syncthreads();
        }
        pu = uend;
        ++u;
        if (it_n != it || pu == pu_end) {
            const int sidx = g - row_g0[it];
            float4 *dst = part + ((long long)it * L.S_max + sidx) * T;
            const float ms = EQM ? mass : 1.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) dst[tid + k * NT] = make_float4(ms * hx[k], ms * hy[k], ms * hz[k], -hg[k]);
            if (it_n != it && pu < pu_end) load_i(it_n);
        }
        it = it_n;
        jt = jt_n;
    }
    if (bad && tid == 0) {
        atomicOr(&flags[FLAG_TIMEOUT], 1);
        if (inflight) mbar_wait_bounded(bar, parity);   // drain the copy in flight, bounded
    }
}

// Consumer side: the VJP of body i (float4 dL/dx, dL/dm) of a pair-once plan,
// its row segments then the column slots on its tile, in that fixed order.
__device__ __forceinline__ float4 reduce_vjp_sym_f32(const float4 *__restrict__ part, const ForceLaunch &L,
                                                     int T, long long i) {
    const SymTab S(L.sym);
    const long long t = i / T, il = i - t * T;
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    auto run = [&](const float4 *p, int cnt) {
        // four loads at a time, the last batch predicated; the sum keeps its order
        for (int s = 0; s < cnt; s += 4) {
            float4 v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (s + k < cnt) v[k] = __ldg(p + (long long)(s + k) * T);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (s + k < cnt) {
                    r.x += v[k].x;
                    r.y += v[k].y;
                    r.z += v[k].z;
                    r.w += v[k].w;
                }
            }
        }
    };
    run(part + t * L.S_max * (long long)T + il, S.row_ns[t]);
    const int k0 = S.col_start[t];
    run(part + L.col_off + (long long)k0 * T + il, S.col_start[t + 1] - k0);
    return r;
}

}  // namespace colatus
