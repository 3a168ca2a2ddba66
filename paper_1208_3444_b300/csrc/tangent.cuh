// tangent.cuh -- tangent-linear (JVP) model of the Eq. 1 force and of the
// KDK and DKD leapfrogs, for finite-time Lyapunov growth of single tracers.
//
// For a perturbation dx of all positions, the force perturbation is
//     dF_k = sum_{j != k} m_j J(d_kj) (dx_j - dx_k),
//     J(d) = I/s^3 - 3 d d^T / s^5      (d_kj = x_j - x_k, s^2 = |d|^2 + eps^2),
// the derivative of the Eq. 1 pair term.  The pair geometry (d, 1/s^3, 1/s^5)
// is computed once and applied to TB tangents at a time:
//     dF_k += a u + (b (d . u)) d,   u = dx_j - dx_k,  a = m_j/s^3,  b = -3 m_j/s^5,
// 11 + 13 TB FP32 ops and one MUFU.RSQ per pair.  The self pair needs no mask
// (u = 0 exactly).
//
// Same stream-K decomposition and bulk-copy pipeline as force.cuh, over
// (tangent chunk, i-tile, j-tile) units.  Per body and chunk the packed tile
// holds (x, y, z, m) and TB tangent positions: 16 + 12 TB bytes (112 B for TB = 8).
#pragma once

#include "common.cuh"
#include "force.cuh"
#include "integrate.cuh"

namespace colatus {

constexpr int kTB = 8;              // tangents per chunk
constexpr int kTC = 3 * kTB;        // tangent components per body and chunk
constexpr int kTPlanes = kTC / 4;   // float4 planes per body in the segments
static_assert(kTC % 4 == 0, "segments hold whole float4 planes");

template <int NT, int IPT, int JT, int STAGES>
struct JvpKernel {
    static constexpr int ITILE = NT * IPT;
    static constexpr uint32_t TILE_BYTES = JT * (4 + kTC) * 4;   // (x, y, z, m) + tangents
    static constexpr int SMEM = STAGES * TILE_BYTES + STAGES * 8;
};

// Two j-bodies per f32x2 lane pair: every FP32 operation of the pair term is
// one f32x2 instruction for two interactions (half the issue slots of scalar
// code at the same FMA-pipe work).  Bodies are pair-interleaved: per pair of
// bodies (2p, 2p + 1) and chunk, 32 floats
//     [x0 x1 y0 y1 | z0 z1 m0 m1 | t0x0 t0x1 t0y0 t0y1 | t0z0 t0z1 t1x0 t1x1 | ...]
// i.e. slot s of body i at float 2 s + (i & 1), slots x, y, z, m, then the TB
// tangent positions (x, y, z) in order; a j-tile of JT bodies is JT * (16 + 12 TB) B.
// Units: chunk-major, then i-tile, then j-tile (W = nchunk * n_it * n_jt);
// part: [nchunk * n_it][S_max][3][ITILE] float4.
constexpr int kPktSlots = 4 + 3 * kTB;   // 28 for TB = 8

__device__ __forceinline__ float *pkt_body(float *pkt, long long chunk, long long n_pad, long long i) {
    return pkt + (chunk * n_pad + (i & ~1LL)) * kPktSlots + (i & 1);
}
__device__ __forceinline__ const float *pkt_body(const float *pkt, long long chunk, long long n_pad,
                                                 long long i) {
    return pkt + (chunk * n_pad + (i & ~1LL)) * kPktSlots + (i & 1);
}

template <int NT, int IPT, int JT, int STAGES, int MINB, int UNR = 1>
__global__ void __launch_bounds__(NT, MINB)
    jvp_f32x2_kernel(const float *__restrict__ pkt, float4 *__restrict__ part, int *__restrict__ flags,
                     ForceLaunch L, long long n_pad, float eps2) {
    using K = JvpKernel<NT, IPT, JT, STAGES>;
    static_assert(JT % 2 == 0, "pairs of j-bodies");
    constexpr int TILE_F4 = K::TILE_BYTES / 16;   // float4 per tile
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
    long long u = u0;
    bool bad = false;
    int stage = 0;
    uint32_t parity = 0;
    while (u < u1) {
        const long long ct = u / per_it;
        const long long chunk = ct / L.n_it, it = ct % L.n_it;
        const long long uend = min(u1, (ct + 1) * per_it);
        // i-side values broadcast to both lanes, negated
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
#pragma unroll (UNR)
                for (int q = 0; q < JT / 2; ++q) {
                    float2 v[kPktSlots];
#pragma unroll
                    for (int f = 0; f < kPktSlots / 2; ++f) {
                        const float4 F = tl[(kPktSlots / 2) * q + f];
                        v[2 * f] = make_float2(F.x, F.y);
                        v[2 * f + 1] = make_float2(F.z, F.w);
                    }
                    const float2 mj = v[3];
                    const float2 m3 = __fmul2_rn(make_float2(-3.f, -3.f), mj);
#pragma unroll
                    for (int k = 0; k < IPT; ++k) {
                        const float2 dx = __fadd2_rn(v[0], nx[k]);
                        const float2 dy = __fadd2_rn(v[1], ny[k]);
                        const float2 dz = __fadd2_rn(v[2], nz[k]);
                        float2 r2 = __ffma2_rn(dx, dx, e2);
                        r2 = __ffma2_rn(dy, dy, r2);
                        r2 = __ffma2_rn(dz, dz, r2);
                        const float2 inv = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                        const float2 inv2 = __fmul2_rn(inv, inv);
                        const float2 inv3 = __fmul2_rn(inv, inv2);
                        const float2 al = __fmul2_rn(mj, inv3);
                        const float2 be = __fmul2_rn(m3, __fmul2_rn(inv3, inv2));
#pragma unroll
                        for (int b = 0; b < kTB; ++b) {
                            const float2 ux = __fadd2_rn(v[4 + 3 * b], ti[k][3 * b]);
                            const float2 uy = __fadd2_rn(v[5 + 3 * b], ti[k][3 * b + 1]);
                            const float2 uz = __fadd2_rn(v[6 + 3 * b], ti[k][3 * b + 2]);
                            const float2 s =
                                __fmul2_rn(be, __ffma2_rn(dz, uz, __ffma2_rn(dy, uy, __fmul2_rn(dx, ux))));
                            ac[k][3 * b] = __ffma2_rn(s, dx, __ffma2_rn(al, ux, ac[k][3 * b]));
                            ac[k][3 * b + 1] = __ffma2_rn(s, dy, __ffma2_rn(al, uy, ac[k][3 * b + 1]));
                            ac[k][3 * b + 2] = __ffma2_rn(s, dz, __ffma2_rn(al, uz, ac[k][3 * b + 2]));
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

// Sum the segments of (chunk, body i): the TB force perturbations.
__device__ __forceinline__ void jvp_reduce(const float4 *__restrict__ part, const ForceLaunch &L,
                                           int itile, long long chunk, long long i, float (&f)[kTC]) {
    const long long it = i / itile, il = i - it * itile;
    const long long ct = chunk * L.n_it + it;
    const long long g0 = sk_owner(ct * L.n_jt, L.W, L.G);
    const long long g1 = sk_owner((ct + 1) * L.n_jt - 1, L.W, L.G);
    const float4 *p = part + ct * L.S_max * (long long)kTPlanes * itile + il;
#pragma unroll
    for (int c = 0; c < kTC; ++c) f[c] = 0.f;
    for (long long s = 0; s <= g1 - g0; ++s) {
#pragma unroll
        for (int pl = 0; pl < kTPlanes; ++pl) {
            const float4 a = __ldg(p + (kTPlanes * s + pl) * itile);
            f[4 * pl] += a.x;
            f[4 * pl + 1] += a.y;
            f[4 * pl + 2] += a.z;
            f[4 * pl + 3] += a.w;
        }
    }
}

// Tangent state per (tangent b, body i): dx, dv, dvh as float4 in
// [B][N_pad] arrays; seeds[b] is the body whose own growth is recorded.
// dx and dv are the tangent at the state's step; dvh (KDK) the half-kicked
// velocity tangent of the step about to be taken.  The tangent position at
// which a step's JVP is evaluated is formed when it is packed (TanDrift).
struct TangentState {
    float4 *dx, *dv, *dvh;
    float4 *dxp;              // [B][N_pad] the packed tangent positions as float4, or null
    float *pkt;               // [nchunk][N_pad / 2][32], pair-interleaved (jvp_f32x2_kernel)
    const long long *seeds;   // [B]
    float *growth;            // [cap][B]
    long long cap, base;      // records kept, absolute step at which recording started
    int B, nchunk;
};

// Tangent position packed for a JVP: the state's own (TAN_AT_STATE), the
// KDK drift dx + tau dvh to x^{n+1} (TAN_KDK_DRIFT), or the DKD half drift
// dx + (tau/2) dv to x^{n+1/2} (TAN_DKD_HALF), with the rounding of the
// state's drift (drift1), so the tangent epilogues recompute it bit for bit.
enum TanDrift { TAN_AT_STATE = 0, TAN_KDK_DRIFT = 1, TAN_DKD_HALF = 2 };

__device__ __forceinline__ float4 tan_drifted(const TangentState &T, long long k, int mode, float t) {
    const float4 d = T.dx[k];
    if (mode == TAN_AT_STATE) return d;
    const float4 w = mode == TAN_KDK_DRIFT ? T.dvh[k] : T.dv[k];
    return make_float4(drift1(d.x, t, w.x), drift1(d.y, t, w.y), drift1(d.z, t, w.z), 0.f);
}

// Pack positions (pair-interleaved pk, padded) and tangent positions.
__global__ void tan_pack_kernel(const float *__restrict__ pk, TangentState T, long long N,
                                long long n_pad, int mode, float t_drift) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int chunk = blockIdx.y;
    if (i >= n_pad) return;
    const float4 x = pk_load(pk, i);
    float t[kTC];
#pragma unroll
    for (int q = 0; q < kTB; ++q) {
        const long long b = (long long)chunk * kTB + q;
        float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < N && b < T.B) d = tan_drifted(T, b * n_pad + i, mode, t_drift);
        if (T.dxp && b < T.B) T.dxp[b * n_pad + i] = d;
        t[3 * q] = d.x;
        t[3 * q + 1] = d.y;
        t[3 * q + 2] = d.z;
    }
    float *o = pkt_body(T.pkt, chunk, n_pad, i);
    o[0] = x.x;
    o[2] = x.y;
    o[4] = x.z;
    o[6] = x.w;
#pragma unroll
    for (int c = 0; c < 3 * kTB; ++c) o[2 * (4 + c)] = t[c];
}

// Deformation term's tangent at the packed position and tangent position
// of (chunk, i).
__device__ __forceinline__ void tan_defo(const TangentState &T, const Extra &D, int chunk,
                                         long long i, long long n_pad, float (&f)[kTC]) {
    if (!D.on) return;
    const float *x = pkt_body(T.pkt, chunk, n_pad, i);
#pragma unroll
    for (int q = 0; q < kTB; ++q) {
        const long long b = (long long)chunk * kTB + q;
        if (b >= T.B) break;
        const float *d = x + 2 * (4 + 3 * q);
        defo_jacobian<float>(D, x[0], x[2], x[4], d[0], d[2], d[4], f[3 * q], f[3 * q + 1], f[3 * q + 2]);
    }
}

// Reciprocal-space JVP of every tangent of the chunk at body i (periodic
// boundaries: lr32 holds [B][n_pad] float4, one plane per tangent).
__device__ __forceinline__ void tan_kspace(const TangentState &T, const Extra &D, int chunk,
                                           long long i, long long n_pad, float (&f)[kTC]) {
    if (!D.lr32) return;
#pragma unroll
    for (int q = 0; q < kTB; ++q) {
        const long long b = (long long)chunk * kTB + q;
        if (b >= T.B) break;
        const float4 l = D.lr32[b * n_pad + i];
        f[3 * q] += l.x;
        f[3 * q + 1] += l.y;
        f[3 * q + 2] += l.z;
    }
}

// KDK opening of the tangent after the JVP at x^n: dvh = c1 dv + d1 dF(x^n).
__global__ void tan_open_kernel(const float4 *__restrict__ part, ForceLaunch L, int itile,
                                TangentState T, const StepCoef *__restrict__ table, int tcap,
                                long long step, long long N, long long n_pad, Extra D) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int chunk = blockIdx.y;
    if (i >= N) return;
    float f[kTC];
    jvp_reduce(part, L, itile, chunk, i, f);
    tan_kspace(T, D, chunk, i, n_pad, f);
    tan_defo(T, D, chunk, i, n_pad, f);
    const StepCoef &e = table[step % tcap];
    const float c1 = (float)e.c1, d1 = (float)e.d1;
#pragma unroll
    for (int q = 0; q < kTB; ++q) {
        const long long b = (long long)chunk * kTB + q;
        if (b >= T.B) break;
        const long long k = b * n_pad + i;
        const float4 v = T.dv[k];
        const float hx = kick2(c1, v.x, d1, f[3 * q]), hy = kick2(c1, v.y, d1, f[3 * q + 1]),
                    hz = kick2(c1, v.z, d1, f[3 * q + 2]);
        T.dvh[k] = make_float4(hx, hy, hz, 0.f);
    }
}

// KDK step of the tangent after the JVP at x^{n+1} (packed as
// TAN_KDK_DRIFT): dx' = dx + tau dvh, dv' = c2 dvh + d2 dF; record the seed
// body's |(dx', dv')|; the next step's half kick with the next entry's
// coefficients: dvh = c1' dv' + d1' dF.
__global__ void tan_step_kernel(const float4 *__restrict__ part, ForceLaunch L, int itile,
                                TangentState T, const StepCoef *__restrict__ table, int tcap,
                                long long step, double tau, long long N, long long n_pad, Extra D) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int chunk = blockIdx.y;
    if (i >= N) return;
    float f[kTC];
    jvp_reduce(part, L, itile, chunk, i, f);
    tan_kspace(T, D, chunk, i, n_pad, f);
    tan_defo(T, D, chunk, i, n_pad, f);
    const StepCoef &e = table[step % tcap];
    const StepCoef &en = table[(step + 1) % tcap];
    const float c2 = (float)e.c2, d2 = (float)e.d2, t = (float)tau;
    const float c1n = (float)en.c1, d1n = (float)en.d1;
#pragma unroll
    for (int q = 0; q < kTB; ++q) {
        const long long b = (long long)chunk * kTB + q;
        if (b >= T.B) break;
        const long long k = b * n_pad + i;
        const float4 h = T.dvh[k];
        const float vx = kick2(c2, h.x, d2, f[3 * q]), vy = kick2(c2, h.y, d2, f[3 * q + 1]),
                    vz = kick2(c2, h.z, d2, f[3 * q + 2]);
        const float4 x = tan_drifted(T, k, TAN_KDK_DRIFT, t);
        T.dv[k] = make_float4(vx, vy, vz, 0.f);
        if (T.seeds[b] == i && T.cap > 0) {
            const long long r = (step - T.base) % T.cap;
            T.growth[r * T.B + b] =
                sqrtf(x.x * x.x + x.y * x.y + x.z * x.z + vx * vx + vy * vy + vz * vz);
        }
        const float nx = kick2(c1n, vx, d1n, f[3 * q]), ny = kick2(c1n, vy, d1n, f[3 * q + 1]),
                    nz = kick2(c1n, vz, d1n, f[3 * q + 2]);
        T.dvh[k] = make_float4(nx, ny, nz, 0.f);
        T.dx[k] = x;
    }
}

// DKD step of the tangent (Eqs. 3-5 linearised; c, d at t^{n+1/2}) after the
// JVP at x^{n+1/2} (packed as TAN_DKD_HALF):
//   dxh = dx + (tau/2) dv;  dv' = c dv + d dF;  dx' = dxh + (tau/2) dv';
// record the seed body's |(dx', dv')|.
__global__ void tan_dkd_step_kernel(const float4 *__restrict__ part, ForceLaunch L, int itile,
                                    TangentState T, const StepCoef *__restrict__ table, int tcap,
                                    long long step, double tau, long long N, long long n_pad, Extra D) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int chunk = blockIdx.y;
    if (i >= N) return;
    float f[kTC];
    jvp_reduce(part, L, itile, chunk, i, f);
    tan_kspace(T, D, chunk, i, n_pad, f);
    tan_defo(T, D, chunk, i, n_pad, f);
    const StepCoef &e = table[step % tcap];
    const float c = (float)e.c, d = (float)e.d, h = (float)(0.5 * tau);
#pragma unroll
    for (int q = 0; q < kTB; ++q) {
        const long long b = (long long)chunk * kTB + q;
        if (b >= T.B) break;
        const long long k = b * n_pad + i;
        const float4 xh = tan_drifted(T, k, TAN_DKD_HALF, h);
        const float4 v0 = T.dv[k];
        const float vx = kick2(c, v0.x, d, f[3 * q]), vy = kick2(c, v0.y, d, f[3 * q + 1]),
                    vz = kick2(c, v0.z, d, f[3 * q + 2]);
        const float x1 = drift1(xh.x, h, vx), y1 = drift1(xh.y, h, vy), z1 = drift1(xh.z, h, vz);
        T.dv[k] = make_float4(vx, vy, vz, 0.f);
        T.dx[k] = make_float4(x1, y1, z1, 0.f);
        if (T.seeds[b] == i && T.cap > 0) {
            const long long r = (step - T.base) % T.cap;
            T.growth[r * T.B + b] = sqrtf(x1 * x1 + y1 * y1 + z1 * z1 + vx * vx + vy * vy + vz * vz);
        }
    }
}

}  // namespace colatus
