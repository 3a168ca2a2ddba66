// ewald_adjoint.cuh -- derivatives of the periodic (Ewald-summed) force of
// ewald.cuh: its vector-Jacobian product for the adjoint and its
// Jacobian-vector product for the tangent model.
//
// The periodic force is F_k = sum_j m_j Phi(x_j - x_k) with Phi odd (the
// real-space pair term over minimum images plus the reciprocal sum), so, for
// a co-vector w and L = sum_k w_k . F_k (J = dPhi/dd, symmetric and even),
//     dL/dx_i = sum_j J(d_ij) (m_i w_j - m_j w_i),
//     dL/dm_i = -sum_j w_j . Phi(d_ij).
//
// Real space.  Phi_R(d) = d b(r) with b = (r^2+eps^2)^{-3/2} + f(r),
// f = -erf(alpha r)/r^3 + cg exp(-alpha^2 r^2)/r^2, so
//     J_R = b I + c d d^T,  c = b'(r)/r = -3 (r^2+eps^2)^{-5/2} + f'(r)/r,
//     f'(r)/r = -(3 f + 2 alpha^2 cg exp(-alpha^2 r^2)) / r^2,
// taken below alpha r = 0.05 from its series (2 alpha^5/sqrt(pi))
// sum_{k>=1} (-1)^{k+1} 4k (alpha r)^{2k-2} / (k! (2k+3)): two terms in FP32
// (the next is 2e-6 of it), four in FP64.  The pair then contributes
//     U += b w_j, B += m_j b, V += c (m_i (w_j.d) - m_j (w_i.d)) d,
//     Gm += b (w_j.d),   dL/dx_i = m_i U - B w_i + V,  dL/dm_i = -Gm,
// the isolated VJP's sums with 1/s^3 -> b and -3/s^5 -> c.  The self pair is
// masked (its b w terms cancel only in exact arithmetic).  Same persistent
// stream-K pipeline as the force and VJP kernels, on the VJP's packed input.
//
// Reciprocal space (half space, weights w_k = 2 (4 pi/L^3) A(k) as in the
// force): with rho(k) = sum_j m_j e^{i k.x_j} and
// Lambda(k) = sum_j (k.w_j) e^{i k.x_j} = k . W(k), W = sum_j w_j e^{i k.x_j},
//     dL/dx_i += sum_k w_k k Re[e^{-i k.x_i} (m_i Lambda - (k.w_i) rho)],
//     dL/dm_i += -sum_k w_k Im[e^{-i k.x_i} Lambda],
// from four structure-factor passes (weights m, w_x, w_y, w_z) of
// ewald_rho_kernel and one pass over (body, k) pairs.
//
// Tangent (JVP) along dx: dF_k = sum_j m_j J(d_kj) (dx_j - dx_k).  Real space
// as the isolated JVP with a = m_j b and beta = m_j c; reciprocal space
//     dF_k += sum_k w_k k Re[e^{-i k.x_k} (D(k) - (k.dx_k) rho(k))],
//     D(k) = sum_j m_j (k.dx_j) e^{i k.x_j},
// the VJP's reciprocal pass with m_i -> 1, w_i -> dx_k and Lambda -> D, one
// tangent at a time (structure factors weighted by m_j dx_j).
#pragma once

#include "adjoint.cuh"
#include "common.cuh"
#include "ewald.cuh"
#include "force.cuh"
#include "tangent.cuh"

namespace colatus {

// b and -c of the real-space pair term for two separations at once (packed
// f32x2); A&S 7.1.26 erfc as in the force, the series below alpha r = 0.05.
__device__ __forceinline__ void ewald_pair_bc2(const float2 dx, const float2 dy, const float2 dz,
                                               const EwaldArgs &A, const float2 e2, float2 &b,
                                               float2 &nc) {
    float2 r2 = __fmul2_rn(dx, dx);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dz, dz, r2);
    const float2 s2 = __fadd2_rn(r2, e2);
    const float2 ip = make_float2(rsqrt_approx(s2.x), rsqrt_approx(s2.y));
    const float2 ip2 = __fmul2_rn(ip, ip);
    const float2 ip3 = __fmul2_rn(ip2, ip);
    const float2 ip5 = __fmul2_rn(ip3, ip2);
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
    const float2 ir2 = __fmul2_rn(ir, ir);
    float2 f = __fmul2_rn(h, ir2);                                           // -erf/r^3 + cg e/r^2
    // -f'(r)/r = (3 f + 2 alpha^2 cg e) / r^2
    const float2 k1 = __ffma2_rn(f, make_float2(3.f, 3.f), __fmul2_rn(ex, make_float2(A.c2ag, A.c2ag)));
    float2 ce = __fmul2_rn(k1, ir2);
    const float2 fs = __ffma2_rn(make_float2(A.s1, A.s1), r2, make_float2(A.s0, A.s0));
    const float2 cs = __ffma2_rn(make_float2(A.ncs1, A.ncs1), r2, make_float2(A.ncs0, A.ncs0));
    const bool sx = r2.x < A.x2_series, sy = r2.y < A.x2_series;
    f.x = sx ? fs.x : f.x;
    f.y = sy ? fs.y : f.y;
    ce.x = sx ? cs.x : ce.x;
    ce.y = sy ? cs.y : ce.y;
    b = __fadd2_rn(ip3, f);
    nc = __ffma2_rn(ip5, make_float2(3.f, 3.f), ce);
}

// Pair policy of the pair-once VJP (vjp_sym.cuh) for the real-space term:
// the separation to its minimum image, then b and -c of ewald_pair_bc2
// (finite at d = 0, where the series holds, so a body's own pair adds
// exactly 0 with u' = 0); J u' = b u' + c (u'.d) d is formed once and added
// to the row sums and, SYM, to the column sums.
struct EwaldVjpPair {
    using Args = EwaldArgs;
    struct F {
        float2 b, nc;
    };
    __device__ __forceinline__ static F factors(float2 &dx, float2 &dy, float2 &dz, const float2 e2,
                                                const EwaldArgs &A) {
        const float2 Lm = make_float2(-A.Lf, -A.Lf), iL = make_float2(A.invLf, A.invLf);
        dx = min_image2(dx, iL, Lm);
        dy = min_image2(dy, iL, Lm);
        dz = min_image2(dz, iL, Lm);
        F f;
        ewald_pair_bc2(dx, dy, dz, A, e2, f.b, f.nc);
        return f;
    }
    __device__ __forceinline__ static float2 bw(const F &f) { return f.b; }
    template <bool SYM>
    __device__ __forceinline__ static void position(const F &f, const float2 dx, const float2 dy, const float2 dz,
                                                    const float2 ux, const float2 uy, const float2 uz,
                                                    const float2 du, float2 &tx, float2 &ty, float2 &tz, float2 &jx,
                                                    float2 &jy, float2 &jz) {
        const float2 cdu = __fmul2_rn(make_float2(-f.nc.x, -f.nc.y), du);   // c (u'.d)
        const float2 sx = __ffma2_rn(cdu, dx, __fmul2_rn(f.b, ux));
        const float2 sy = __ffma2_rn(cdu, dy, __fmul2_rn(f.b, uy));
        const float2 sz = __ffma2_rn(cdu, dz, __fmul2_rn(f.b, uz));
        tx = __fadd2_rn(tx, sx);
        ty = __fadd2_rn(ty, sy);
        tz = __fadd2_rn(tz, sz);
        if (SYM) {
            jx = __fadd2_rn(jx, sx);
            jy = __fadd2_rn(jy, sy);
            jz = __fadd2_rn(jz, sz);
        }
    }
};

template <int NT, int IPT, int JT, int STAGES>
struct EwaldVjpKernel {
    static constexpr int ITILE = NT * IPT;
    static constexpr uint32_t TILE_BYTES = JT * 32;   // 32 B per body (VJP layout)
    static constexpr int SMEM = STAGES * TILE_BYTES + STAGES * 8;
};

// One j-tile of the periodic VJP for the IPT i-bodies of this thread
// (duplicated into both lanes); MASK: the tile may contain i itself.
template <int IPT, int JT, bool MASK>
__device__ __forceinline__ void ewald_vjp_tile(
    const float4 *__restrict__ t, long long jbase, const long long (&ii)[IPT], const float2 (&nx)[IPT],
    const float2 (&ny)[IPT], const float2 (&nz)[IPT], const float2 (&mi)[IPT], const float2 (&wxi)[IPT],
    const float2 (&wyi)[IPT], const float2 (&wzi)[IPT], const EwaldArgs &A, const float2 e2,
    const float2 iL, const float2 Lm, float2 (&Ux)[IPT], float2 (&Uy)[IPT], float2 (&Uz)[IPT],
    float2 (&Bm)[IPT], float2 (&Vx)[IPT], float2 (&Vy)[IPT], float2 (&Vz)[IPT], float2 (&Gm)[IPT]) {
#pragma unroll 1
    for (int q = 0; q < JT / 2; ++q) {
        const float4 Aq = t[4 * q];
        const float4 Bq = t[4 * q + 1];
        const float4 Cq = t[4 * q + 2];
        const float4 Dq = t[4 * q + 3];
        const float2 xj = make_float2(Aq.x, Aq.y), yj = make_float2(Aq.z, Aq.w);
        const float2 zj = make_float2(Bq.x, Bq.y), mj = make_float2(Bq.z, Bq.w);
        const float2 wxj = make_float2(Cq.x, Cq.y), wyj = make_float2(Cq.z, Cq.w);
        const float2 wzj = make_float2(Dq.x, Dq.y);
        const float2 nmj = make_float2(-mj.x, -mj.y);
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            float2 dx = __fadd2_rn(xj, nx[k]);
            float2 dy = __fadd2_rn(yj, ny[k]);
            float2 dz = __fadd2_rn(zj, nz[k]);
            dx = min_image2(dx, iL, Lm);
            dy = min_image2(dy, iL, Lm);
            dz = min_image2(dz, iL, Lm);
            float2 b, nc;
            ewald_pair_bc2(dx, dy, dz, A, e2, b, nc);
            if (MASK) {
                const long long j0 = jbase + 2 * q;
                if (j0 == ii[k]) b.x = nc.x = 0.f;
                if (j0 + 1 == ii[k]) b.y = nc.y = 0.f;
            }
            Ux[k] = __ffma2_rn(b, wxj, Ux[k]);
            Uy[k] = __ffma2_rn(b, wyj, Uy[k]);
            Uz[k] = __ffma2_rn(b, wzj, Uz[k]);
            Bm[k] = __ffma2_rn(mj, b, Bm[k]);
            float2 lj = __fmul2_rn(wxj, dx);
            lj = __ffma2_rn(wyj, dy, lj);
            lj = __ffma2_rn(wzj, dz, lj);
            float2 li = __fmul2_rn(wxi[k], dx);
            li = __ffma2_rn(wyi[k], dy, li);
            li = __ffma2_rn(wzi[k], dz, li);
            const float2 dw = __ffma2_rn(mi[k], lj, __fmul2_rn(nmj, li));
            const float2 g = __fmul2_rn(nc, dw);
            Vx[k] = __ffma2_rn(g, dx, Vx[k]);
            Vy[k] = __ffma2_rn(g, dy, Vy[k]);
            Vz[k] = __ffma2_rn(g, dz, Vz[k]);
            Gm[k] = __ffma2_rn(b, lj, Gm[k]);
        }
    }
}

// Real-space periodic VJP: segments float4 (dL/dx, dL/dm) per body, in the
// same [i-tile][segment][ITILE] layout as the VJP kernel (Vx.. hold -V).
template <int NT, int IPT, int JT, int STAGES, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    ewald_vjp_f32_kernel(const float *__restrict__ pkw, float4 *__restrict__ part,
                         int *__restrict__ flags, ForceLaunch L, float eps2, EwaldArgs A) {
    using K = EwaldVjpKernel<NT, IPT, JT, STAGES>;
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
    const float2 Lm = make_float2(-A.Lf, -A.Lf), iL = make_float2(A.invLf, A.invLf);
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
        const long long ilo = it * K::ITILE, ihi = ilo + K::ITILE;
        for (; u < uend; ++u) {
            const bool ok = mbar_wait_bounded(&full[stage], parity);
            if (ok) {
                const long long jt = u % n_jt;
                const long long jlo = jt * JT;
                const float4 *t = tiles + stage * TILE_F4;
                if (jlo < ihi && jlo + JT > ilo)
                    ewald_vjp_tile<IPT, JT, true>(t, jlo, ii, nx, ny, nz, mi, wxi, wyi, wzi, A, e2, iL,
                                                  Lm, Ux, Uy, Uz, Bm, Vx, Vy, Vz, Gm);
                else
                    ewald_vjp_tile<IPT, JT, false>(t, jlo, ii, nx, ny, nz, mi, wxi, wyi, wzi, A, e2,
                                                   iL, Lm, Ux, Uy, Uz, Bm, Vx, Vy, Vz, Gm);
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
            const float m = mi[k].x;
            const float bm = Bm[k].x + Bm[k].y;
            const float gx = m * (Ux[k].x + Ux[k].y) - bm * wxi[k].x - (Vx[k].x + Vx[k].y);
            const float gy = m * (Uy[k].x + Uy[k].y) - bm * wyi[k].x - (Vy[k].x + Vy[k].y);
            const float gz = m * (Uz[k].x + Uz[k].y) - bm * wzi[k].x - (Vz[k].x + Vz[k].y);
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

// FP64 b and c of the real-space pair term (library erf/exp; series below
// alpha r = 0.05 to (alpha r)^6, relative error below 1e-12 there).
__device__ __forceinline__ void ewald_pair_bc64(double r2, double eps2, const EwaldArgs &A, double &b,
                                                double &c) {
    const double al = A.alpha, al2 = al * al;
    const double rsp = rsqrt(acos(-1.0));                 // 1/sqrt(pi)
    const double ip = rsqrt(r2 + eps2), ip2 = ip * ip, ip3 = ip2 * ip, ip5 = ip3 * ip2;
    const double x2s = (0.05 / al) * (0.05 / al);
    double f, fc;
    if (r2 < x2s) {
        const double x2 = al2 * r2;
        f = 2.0 * al * al2 * rsp * (-2.0 / 3.0 + x2 * (0.4 + x2 * (-1.0 / 7.0 + x2 * (1.0 / 27.0))));
        fc = 2.0 * al2 * al2 * al * rsp *
             (0.8 + x2 * (-4.0 / 7.0 + x2 * (2.0 / 9.0 + x2 * (-2.0 / 33.0))));
    } else {
        const double ir = rsqrt(r2), r = r2 * ir, ir2 = ir * ir;
        const double e = exp(-al2 * r2), cg = 2.0 * al * rsp;
        f = -erf(al * r) * ir2 * ir + cg * e * ir2;
        fc = -(3.0 * f + 2.0 * al2 * cg * e) * ir2;
    }
    b = ip3 + f;
    c = -3.0 * ip5 + fc;
}

template <int NT, int JT, int STAGES>
struct EwaldVjp64Kernel {
    static constexpr int ITILE = NT;
    static constexpr uint32_t TILE_BYTES = JT * 64;
    static constexpr int SMEM = STAGES * TILE_BYTES + STAGES * 8;
};

// FP64 real-space periodic VJP on bodies as two double4 per body
// ((x, y, z, m), (wx, wy, wz, 0)); one i-body per thread.
template <int NT, int JT, int STAGES>
__global__ void __launch_bounds__(NT)
    ewald_vjp_f64_kernel(const double4 *__restrict__ bw, double4 *__restrict__ part,
                         int *__restrict__ flags, ForceLaunch L, double eps2, EwaldArgs A) {
    using K = EwaldVjp64Kernel<NT, JT, STAGES>;
    extern __shared__ __align__(128) unsigned char smem[];
    double4 *tiles = reinterpret_cast<double4 *>(smem);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * K::TILE_BYTES);
    const int tid = threadIdx.x;
    const long long G = gridDim.x, g = blockIdx.x;
    const long long W = L.W;
    const long long u0 = sk_begin(g, W, G), u1 = sk_begin(g + 1, W, G);
    const int n_jt = L.n_jt;
    const double Lb = A.L, invL = 1.0 / A.L;
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
#pragma unroll 1
                for (int j = 0; j < JT; ++j) {
                    if (jlo + j == i) continue;
                    const double4 p = t[2 * j], w = t[2 * j + 1];
                    double dx = p.x - pi.x, dy = p.y - pi.y, dz = p.z - pi.z;
                    dx -= Lb * rint(dx * invL);
                    dy -= Lb * rint(dy * invL);
                    dz -= Lb * rint(dz * invL);
                    double b, c;
                    ewald_pair_bc64(dx * dx + dy * dy + dz * dz, eps2, A, b, c);
                    ux += b * w.x;
                    uy += b * w.y;
                    uz += b * w.z;
                    bm += p.w * b;
                    const double lj = w.x * dx + w.y * dy + w.z * dz;
                    const double li = wi.x * dx + wi.y * dy + wi.z * dz;
                    const double gg = c * (pi.w * lj - p.w * li);
                    vx += gg * dx;
                    vy += gg * dy;
                    vz += gg * dz;
                    gm += b * lj;
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
            make_double4(pi.w * ux - bm * wi.x + vx, pi.w * uy - bm * wi.y + vy,
                         pi.w * uz - bm * wi.z + vz, -gm);
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

// ------------------------------------------------------------------ k space
// Weights of the reciprocal VJP (or of one tangent's JVP) from partial
// structure factors: rho_m[split][k] weighted by m, and three planes
// rho_w[c][split][k] weighted by w_c (or m dx_c), one thread per k (its
// pencil found by bisection on the pencils' first k):
//   wr[k] = w_k rho(k),  wl[k] = w_k Lambda(k),  Lambda = (2 pi/L) n . W(k).
template <typename T>
__global__ void ewald_vjp_weights_kernel(const double2 *__restrict__ rho_m,
                                         const double2 *__restrict__ rho_w, int splits, int nkv,
                                         const double *__restrict__ kw,
                                         const KPencil *__restrict__ pen, int npen, double tpl,
                                         typename Vec2<T>::type *__restrict__ wr,
                                         typename Vec2<T>::type *__restrict__ wl) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nkv) return;
    int lo = 0, hi = npen - 1;   // the last pencil with koff <= k
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pen[mid].koff <= k) lo = mid;
        else hi = mid - 1;
    }
    const KPencil P = pen[lo];
    const int nz = P.nz0 + (k - P.koff);
    double s[4][2];
    for (int c = 0; c < 4; ++c) {
        const double2 *src = c == 0 ? rho_m : rho_w + (long long)(c - 1) * splits * nkv;
        double r = 0.0, i = 0.0;
        for (int sp = 0; sp < splits; ++sp) {
            const double2 v = src[(long long)sp * nkv + k];
            r += v.x;
            i += v.y;
        }
        s[c][0] = r;
        s[c][1] = i;
    }
    const double lr = tpl * (P.nx * s[1][0] + P.ny * s[2][0] + nz * s[3][0]);
    const double li = tpl * (P.nx * s[1][1] + P.ny * s[2][1] + nz * s[3][1]);
    wr[k].x = (T)(kw[k] * s[0][0]);
    wr[k].y = (T)(kw[k] * s[0][1]);
    wl[k].x = (T)(kw[k] * lr);
    wl[k].y = (T)(kw[k] * li);
}

// Channel weights of a multi-channel structure-factor pass: mode 0, entries
// widx[c] of each body's packed record (the VJP's m, w_x, w_y, w_z); mode 1,
// m_j dx_b[j] of the tangents b = b0 + c / 3 (component c % 3; 0 past B).
struct ChanSrc {
    BodySrc src;
    int mode;
    int widx[4];
    const float4 *tdx;   // [B][n_pad] tangent positions (mode 1)
    long long n_pad;
    int b0, B;
};

__device__ __forceinline__ double chan_weight(const ChanSrc &C, long long j, int c) {
    if (C.mode == 0) {
        const int w = c == 0 ? C.widx[0] : (c == 1 ? C.widx[1] : (c == 2 ? C.widx[2] : C.widx[3]));
        return body_entry(C.src, j, w);
    }
    const int b = C.b0 + c / 3;
    if (b >= C.B) return 0.0;
    const float4 d = C.tdx[(long long)b * C.n_pad + j];
    const int q = c % 3;
    return body_entry(C.src, j, 6) * (double)(q == 0 ? d.x : (q == 1 ? d.y : d.z));
}

// NCH structure factors in one pass: rho_part[c][split][k] = sum over the
// split's bodies of w_c(j) exp(i k.x_j).  ewald_rho_kernel's decomposition
// (k chunks x body splits, one k per thread, batches of bodies staged with
// their tables); the per-(body, pencil) base holds the bare x-y phase, so a
// (k, body) pair costs one complex product and two FMAs per channel.
template <typename T, int NCH>
__global__ void __launch_bounds__(kEwKThreads)
    ewald_rho_multi_kernel(ChanSrc C, long long N, const typename Vec2<T>::type *__restrict__ ph,
                           const KPencil *__restrict__ pen, const int *__restrict__ rchunk,
                           int np_max, int nkv, EwaldArgs A, double2 *__restrict__ rho_part) {
    using T2 = typename Vec2<T>::type;
    constexpr int NB = ew_bodies<T>();
    extern __shared__ __align__(16) unsigned char sm[];
    const int nt = A.nk + 1;
    T2 *tab = reinterpret_cast<T2 *>(sm);                  // [NB][3][nt]
    T2 *base = tab + NB * 3 * nt;                          // [NB][np_max]
    T *tw = reinterpret_cast<T *>(base + NB * np_max);     // [NB][NCH]
    int2 *sp = reinterpret_cast<int2 *>(tw + NB * NCH);    // [np_max]
    const int p0 = rchunk[blockIdx.x], np = rchunk[blockIdx.x + 1] - p0;
    const int k0 = pen[p0].koff;
    const int nkc = pen[p0 + np - 1].koff + pen[p0 + np - 1].len - k0;
    const int t = threadIdx.x;
    for (int l = t; l < np; l += kEwKThreads) sp[l] = make_int2(pen[p0 + l].nx, pen[p0 + l].ny);
    int lp = 0;
    while (lp + 1 < np && pen[p0 + lp + 1].koff <= k0 + t) ++lp;
    const int nz = pen[p0 + lp].nz0 + (k0 + t - pen[p0 + lp].koff);
    const int zrow = 2 * nt + (nz < 0 ? -nz : nz);
    const T zs = nz < 0 ? (T)-1 : (T)1;
    const long long per = (N + gridDim.y - 1) / gridDim.y;
    const long long b0 = (long long)blockIdx.y * per, b1 = min(N, b0 + per);
    double cr[NCH], ci[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) cr[c] = ci[c] = 0.0;
    for (long long j0 = b0; j0 < b1; j0 += NB) {
        const int nb = (int)min((long long)NB, b1 - j0);
        __syncthreads();
        const T2 *tsrc = ph + j0 * 3 * nt;
        for (int q = t; q < nb * 3 * nt; q += kEwKThreads) tab[q] = tsrc[q];
        for (int q = t; q < nb * NCH; q += kEwKThreads)
            tw[q] = (T)chan_weight(C, j0 + q / NCH, q % NCH);
        __syncthreads();
        for (int q = t; q < nb * np; q += kEwKThreads) {
            const int b = q / np, l = q - b * np;
            const int2 P = sp[l];
            const T2 *tb = tab + b * 3 * nt;
            const T2 x = tb[P.x];
            const T2 y = axis_phase<T, T2>(tb + nt, P.y, 1);
            T2 v;
            v.x = x.x * y.x - x.y * y.y;
            v.y = x.x * y.y + x.y * y.x;
            base[q] = v;
        }
        __syncthreads();
        if (t < nkc) {
            T pr[NCH], pi[NCH];
#pragma unroll
            for (int c = 0; c < NCH; ++c) pr[c] = pi[c] = 0;
#pragma unroll 2
            for (int b = 0; b < nb; ++b) {
                const T2 z = tab[b * 3 * nt + zrow];
                const T2 w = base[b * np + lp];
                const T zi = zs * z.y;
                const T er = w.x * z.x - w.y * zi, ei = w.x * zi + w.y * z.x;
                const T *wb = tw + b * NCH;
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    pr[c] += wb[c] * er;
                    pi[c] += wb[c] * ei;
                }
            }
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                cr[c] += (double)pr[c];
                ci[c] += (double)pi[c];
            }
        }
    }
    if (t < nkc) {
        const long long plane = (long long)gridDim.y * nkv;
#pragma unroll
        for (int c = 0; c < NCH; ++c)
            rho_part[c * plane + (long long)blockIdx.y * nkv + k0 + t] = make_double2(cr[c], ci[c]);
    }
}

// Shared memory of ewald_rho_multi_kernel.
template <typename T, int NCH>
__host__ inline size_t ew_rho_multi_smem(int nk, int np_max) {
    using T2 = typename Vec2<T>::type;
    constexpr int nb = ew_bodies<T>();
    return ((size_t)nb * 3 * (nk + 1) + (size_t)nb * np_max) * sizeof(T2) + (size_t)nb * NCH * sizeof(T) +
           (size_t)np_max * sizeof(int2);
}

// Reciprocal-space VJP at every body, or (NTAN tangents) the JVP of up to
// NTAN tangents at once.  VJP (wv null, NTAN = 1): m_i and w_i from the
// packed record,
//   out_i = ( (2 pi/L) sum_k n Re[e^{-ik.x_i} (m_i wl - (k.w_i) wr)],
//             -sum_k Im[e^{-ik.x_i} wl] ).
// JVP: m_i -> 1, w_i -> dx_t[i] = wv[t wstride + i], wl -> the tangent's own
// plane wl + t nkv, out[t ostride + i] (x, y, z; w unused); the phase and
// the wr part are shared by the tangents.  Blocks of kEwFThreads bodies with
// kEwFSlices threads per body, each taking every kEwFSlices-th pencil, the
// bodies' phase tables staged in shared memory as in ewald_kforce_kernel;
// the slices are added in order (deterministic).
template <typename T, typename T4, int NTAN>
__global__ void __launch_bounds__(kEwFThreads * kEwFSlices)
    ewald_kvjp_kernel(long long N, const typename Vec2<T>::type *__restrict__ ph,
                      const KPencil *__restrict__ pen, int npen, int nkv,
                      const typename Vec2<T>::type *__restrict__ wr,
                      const typename Vec2<T>::type *__restrict__ wl, BodySrc src,
                      const float4 *__restrict__ wv, long long wstride, int ntan, EwaldArgs A,
                      T4 *__restrict__ out, long long ostride) {
    using T2 = typename Vec2<T>::type;
    constexpr int NT = kEwFThreads * kEwFSlices;
    constexpr int NQ = NTAN == 1 ? 4 : 3 * NTAN;   // reduced quantities per body
    extern __shared__ __align__(16) unsigned char sm[];
    const int nt = A.nk + 1;
    T2 *tab = reinterpret_cast<T2 *>(sm);   // [3 nt][kEwFThreads]
    const long long i0 = (long long)blockIdx.x * kEwFThreads;
    const int nb = (int)min((long long)kEwFThreads, N - i0);
    for (int q = threadIdx.x; q < nb * 3 * nt; q += NT) {
        const int b = q / (3 * nt), r = q - b * 3 * nt;
        tab[r * kEwFThreads + b] = ph[i0 * 3 * nt + q];
    }
    __syncthreads();
    const int bi = threadIdx.x % kEwFThreads, sl = threadIdx.x / kEwFThreads;
    const long long i = i0 + bi;
    const T2 *mine = tab + bi;
    const T2 *zt = mine + 2 * nt * kEwFThreads;
    const double tpl = 2.0 * acos(-1.0) / A.L;
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    if (i < N) {
        T m = (T)1, wx[NTAN], wy[NTAN], wz[NTAN];
        if (!wv) {
            m = (T)body_entry(src, i, src.pos ? 3 : 6);
            wx[0] = (T)body_entry(src, i, src.pos ? 4 : 8);
            wy[0] = (T)body_entry(src, i, src.pos ? 5 : 10);
            wz[0] = (T)body_entry(src, i, src.pos ? 6 : 12);
        } else {
#pragma unroll
            for (int t = 0; t < NTAN; ++t) {
                const float4 d = t < ntan ? wv[t * wstride + i] : make_float4(0.f, 0.f, 0.f, 0.f);
                wx[t] = (T)d.x;
                wy[t] = (T)d.y;
                wz[t] = (T)d.z;
            }
        }
        for (int p = sl; p < npen; p += kEwFSlices) {
            const KPencil P = pen[p];
            const T2 x = mine[P.nx * kEwFThreads];
            const T2 y = axis_phase<T, T2>(mine + nt * kEwFThreads, P.ny, kEwFThreads);
            const T er = x.x * y.x - x.y * y.y, ei = x.x * y.y + x.y * y.x;
            T c0[NTAN], c1[NTAN], B[NTAN], Bz[NTAN];
#pragma unroll
            for (int t = 0; t < NTAN; ++t) {
                c0[t] = (T)tpl * ((T)P.nx * wx[t] + (T)P.ny * wy[t]);
                c1[t] = (T)tpl * wz[t];
                B[t] = Bz[t] = 0;
            }
            T M = 0;
            const long long koff = P.koff - P.nz0;   // wr[koff + nz] is this pencil's k
            for (int nz = P.nz0; nz < P.nz0 + P.len; ++nz) {
                T2 z = zt[(nz < 0 ? -nz : nz) * kEwFThreads];
                if (nz < 0) z.y = -z.y;
                const T Er = er * z.x - ei * z.y, Ei = er * z.y + ei * z.x;   // e^{i k.x_i}
                const T2 R = wr[koff + nz];
                const T rr = Er * R.x + Ei * R.y;                             // Re[conj(E) wr]
#pragma unroll
                for (int t = 0; t < NTAN; ++t) {
                    const T2 W = wl[t * (long long)nkv + koff + nz];
                    const T lr = Er * W.x + Ei * W.y;                         // Re[conj(E) wl]
                    const T tt = m * lr - (c0[t] + (T)nz * c1[t]) * rr;
                    B[t] += tt;
                    Bz[t] += tt * (T)nz;
                    if (NTAN == 1) M += Er * W.y - Ei * W.x;                  // Im[conj(E) wl]
                }
            }
#pragma unroll
            for (int t = 0; t < NTAN; ++t) {
                acc[3 * t] += (double)((T)P.nx * B[t]);
                acc[3 * t + 1] += (double)((T)P.ny * B[t]);
                acc[3 * t + 2] += (double)Bz[t];
            }
            if (NTAN == 1) acc[3] += (double)M;
        }
    }
    __syncthreads();
    double *red = reinterpret_cast<double *>(sm);   // [NQ][kEwFSlices][kEwFThreads]
#pragma unroll
    for (int q = 0; q < NQ; ++q) red[(q * kEwFSlices + sl) * kEwFThreads + bi] = acc[q];
    __syncthreads();
    if (sl == 0 && i < N) {
        double sum[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            sum[q] = 0.0;
            for (int u = 0; u < kEwFSlices; ++u) sum[q] += red[(q * kEwFSlices + u) * kEwFThreads + bi];
        }
        if (NTAN == 1) {
            out[i].x = (T)(tpl * sum[0]);
            out[i].y = (T)(tpl * sum[1]);
            out[i].z = (T)(tpl * sum[2]);
            out[i].w = (T)(-sum[3]);
        } else {
#pragma unroll
            for (int t = 0; t < NTAN; ++t) {
                if (t >= ntan) break;
                T4 &o = out[t * ostride + i];
                o.x = (T)(tpl * sum[3 * t]);
                o.y = (T)(tpl * sum[3 * t + 1]);
                o.z = (T)(tpl * sum[3 * t + 2]);
                o.w = (T)0;
            }
        }
    }
}

// Shared memory of ewald_kvjp_kernel: the tables, or the slice reduction.
template <typename T, int NTAN>
__host__ inline size_t ew_kvjp_smem(int nk) {
    constexpr int NQ = NTAN == 1 ? 4 : 3 * NTAN;
    const size_t tabs = (size_t)kEwFThreads * 3 * (nk + 1) * 2 * sizeof(T);
    const size_t red = (size_t)NQ * kEwFSlices * kEwFThreads * sizeof(double);
    return tabs > red ? tabs : red;
}

// Real-space periodic JVP for kTB tangents per chunk: jvp_f32x2_kernel's
// pipeline, layout and segments with the periodic pair geometry (minimum
// image, b and c of the Ewald real-space term shared by the tangents):
//     dF_k += a u + (beta (d . u)) d,  a = m_j b,  beta = m_j c,  u = dx_j - dx_k.
// The self pair contributes 0 (u = 0 exactly).
template <int NT, int IPT, int JT, int STAGES, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    ewald_jvp_f32x2_kernel(const float *__restrict__ pkt, float4 *__restrict__ part,
                           int *__restrict__ flags, ForceLaunch L, long long n_pad, float eps2,
                           EwaldArgs A) {
    using K = JvpKernel<NT, IPT, JT, STAGES>;
    static_assert(JT % 2 == 0, "pairs of j-bodies");
    constexpr int TILE_F4 = K::TILE_BYTES / 16;
    extern __shared__ __align__(128) unsigned char smem[];
    float4 *tiles = reinterpret_cast<float4 *>(smem);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * K::TILE_BYTES);
    const int tid = threadIdx.x;
    const long long G = gridDim.x, g = blockIdx.x;
    const long long W = L.W;
    const long long u0 = sk_begin(g, W, G), u1 = sk_begin(g + 1, W, G);
    const int n_jt = L.n_jt;
    const long long per_it = n_jt;
    auto tile_src = [&](long long u) -> const float * {
        const long long ct = u / per_it;
        const long long chunk = ct / L.n_it;
        const long long jt = u % per_it;
        return pkt + (chunk * n_pad + jt * JT) * kPktSlots;
    };
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < STAGES && u0 + s < u1; ++s) {
            mbar_arrive_expect_tx(&full[s], K::TILE_BYTES);
            bulk_load(tiles + s * TILE_F4, tile_src(u0 + s), K::TILE_BYTES, &full[s]);
        }
    }
    const float2 e2 = make_float2(eps2, eps2);
    const float2 Lm = make_float2(-A.Lf, -A.Lf), iL = make_float2(A.invLf, A.invLf);
    long long u = u0;
    bool bad = false;
    int stage = 0;
    uint32_t parity = 0;
    while (u < u1) {
        const long long ct = u / per_it;
        const long long chunk = ct / L.n_it, it = ct % L.n_it;
        const long long uend = min(u1, (ct + 1) * per_it);
        float2 nx[IPT], ny[IPT], nz[IPT], ti[IPT][3 * kTB], ac[IPT][3 * kTB];
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const long long i = it * K::ITILE + tid + k * NT;
            const float *p = pkt_body(pkt, chunk, n_pad, i);
            const float x = __ldg(p), y = __ldg(p + 2), z = __ldg(p + 4);
            nx[k] = make_float2(-x, -x);
            ny[k] = make_float2(-y, -y);
            nz[k] = make_float2(-z, -z);
#pragma unroll
            for (int c = 0; c < 3 * kTB; ++c) {
                const float t = -__ldg(p + 2 * (4 + c));
                ti[k][c] = make_float2(t, t);
                ac[k][c] = make_float2(0.f, 0.f);
            }
        }
        for (; u < uend; ++u) {
            const bool ok = mbar_wait_bounded(&full[stage], parity);
            if (ok) {
                const float4 *tl = tiles + stage * TILE_F4;
#pragma unroll 1
                for (int q = 0; q < JT / 2; ++q) {
                    float2 v[kPktSlots];
#pragma unroll
                    for (int f = 0; f < kPktSlots / 2; ++f) {
                        const float4 F = tl[(kPktSlots / 2) * q + f];
                        v[2 * f] = make_float2(F.x, F.y);
                        v[2 * f + 1] = make_float2(F.z, F.w);
                    }
                    const float2 mj = v[3];
                    const float2 nmj = make_float2(-mj.x, -mj.y);
#pragma unroll
                    for (int k = 0; k < IPT; ++k) {
                        float2 dx = __fadd2_rn(v[0], nx[k]);
                        float2 dy = __fadd2_rn(v[1], ny[k]);
                        float2 dz = __fadd2_rn(v[2], nz[k]);
                        dx = min_image2(dx, iL, Lm);
                        dy = min_image2(dy, iL, Lm);
                        dz = min_image2(dz, iL, Lm);
                        float2 b, nc;
                        ewald_pair_bc2(dx, dy, dz, A, e2, b, nc);
                        const float2 al = __fmul2_rn(mj, b);
                        const float2 be = __fmul2_rn(nmj, nc);
#pragma unroll
                        for (int t = 0; t < kTB; ++t) {
                            const float2 ux = __fadd2_rn(v[4 + 3 * t], ti[k][3 * t]);
                            const float2 uy = __fadd2_rn(v[5 + 3 * t], ti[k][3 * t + 1]);
                            const float2 uz = __fadd2_rn(v[6 + 3 * t], ti[k][3 * t + 2]);
                            const float2 s =
                                __fmul2_rn(be, __ffma2_rn(dz, uz, __ffma2_rn(dy, uy, __fmul2_rn(dx, ux))));
                            ac[k][3 * t] = __ffma2_rn(s, dx, __ffma2_rn(al, ux, ac[k][3 * t]));
                            ac[k][3 * t + 1] = __ffma2_rn(s, dy, __ffma2_rn(al, uy, ac[k][3 * t + 1]));
                            ac[k][3 * t + 2] = __ffma2_rn(s, dz, __ffma2_rn(al, uz, ac[k][3 * t + 2]));
                        }
                    }
                }
            }
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
            if (tid == 0 && u + STAGES < u1) {
                mbar_arrive_expect_tx(&full[stage], K::TILE_BYTES);
                bulk_load(tiles + stage * TILE_F4, tile_src(u + STAGES), K::TILE_BYTES, &full[stage]);
            }
            if (++stage == STAGES) {
                stage = 0;
                parity ^= 1u;
            }
        }
        if (bad) break;
        const long long sidx = g - sk_owner(ct * per_it, W, G);
        float4 *dst = part + (ct * L.S_max + sidx) * (long long)kTPlanes * K::ITILE;
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const int il = tid + k * NT;
            float a[kTC];
#pragma unroll
            for (int c = 0; c < kTC; ++c) a[c] = ac[k][c].x + ac[k][c].y;
#pragma unroll
            for (int pl = 0; pl < kTPlanes; ++pl)
                dst[pl * K::ITILE + il] = make_float4(a[4 * pl], a[4 * pl + 1], a[4 * pl + 2], a[4 * pl + 3]);
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

}  // namespace colatus
