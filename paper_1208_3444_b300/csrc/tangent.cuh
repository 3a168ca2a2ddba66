// tangent.cuh -- tangent-linear (JVP) model of the Eq. 1 force and of the
// KDK leapfrog, for finite-time Lyapunov growth of single tracers.
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
// holds (x, y, z, m) and TB tangent positions: 4 float4 = 64 B for TB = 4.
#pragma once

#include "common.cuh"
#include "force.cuh"
#include "integrate.cuh"

namespace colatus {

constexpr int kTB = 4;   // tangents per chunk

template <int NT, int IPT, int JT, int STAGES>
struct JvpKernel {
    static constexpr int ITILE = NT * IPT;
    static constexpr uint32_t TILE_BYTES = JT * 64;
    static constexpr int SMEM = STAGES * TILE_BYTES + STAGES * 8;
};

// units: chunk-major, then i-tile, then j-tile (W = nchunk * n_it * n_jt).
// pkt: [nchunk][N_pad][4] float4; part: [nchunk * n_it][S_max][3][ITILE] float4
template <int NT, int IPT, int JT, int STAGES, int MINB, int UNR = 1>
__global__ void __launch_bounds__(NT, MINB)
    jvp_f32_kernel(const float4 *__restrict__ pkt, float4 *__restrict__ part, int *__restrict__ flags,
                   ForceLaunch L, long long n_pad, float eps2) {
    using K = JvpKernel<NT, IPT, JT, STAGES>;
    extern __shared__ __align__(128) unsigned char smem[];
    float4 *tiles = reinterpret_cast<float4 *>(smem);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * K::TILE_BYTES);
    const int tid = threadIdx.x;
    const long long G = gridDim.x, g = blockIdx.x;
    const long long W = L.W;
    const long long u0 = sk_begin(g, W, G), u1 = sk_begin(g + 1, W, G);
    const int n_jt = L.n_jt;
    const long long per_it = n_jt;                           // units per (chunk, i-tile)
    auto tile_src = [&](long long u) -> const float4 * {
        const long long ct = u / per_it;                     // (chunk, i-tile) index
        const long long chunk = ct / L.n_it;
        const long long jt = u % per_it;
        return pkt + (chunk * n_pad + jt * JT) * 4;
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
            bulk_load(tiles + s * JT * 4, tile_src(u0 + s), K::TILE_BYTES, &full[s]);
        }
    }
    const float e2 = eps2;
    long long u = u0;
    bool bad = false;
    int stage = 0;
    uint32_t parity = 0;
    while (u < u1) {
        const long long ct = u / per_it;
        const long long chunk = ct / L.n_it, it = ct % L.n_it;
        const long long uend = min(u1, (ct + 1) * per_it);
        float xi[IPT], yi[IPT], zi[IPT], tx[IPT][kTB], ty[IPT][kTB], tz[IPT][kTB];
        float ax[IPT][kTB], ay[IPT][kTB], az[IPT][kTB];
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const long long i = it * K::ITILE + tid + k * NT;
            const float4 *p = pkt + (chunk * n_pad + i) * 4;
            const float4 P = p[0], A = p[1], Bv = p[2], C = p[3];
            xi[k] = P.x;
            yi[k] = P.y;
            zi[k] = P.z;
            const float t[12] = {A.x, A.y, A.z, A.w, Bv.x, Bv.y, Bv.z, Bv.w, C.x, C.y, C.z, C.w};
#pragma unroll
            for (int b = 0; b < kTB; ++b) {
                tx[k][b] = t[3 * b];
                ty[k][b] = t[3 * b + 1];
                tz[k][b] = t[3 * b + 2];
                ax[k][b] = ay[k][b] = az[k][b] = 0.f;
            }
        }
        for (; u < uend; ++u) {
            const bool ok = mbar_wait_bounded(&full[stage], parity);
            if (ok) {
                const float4 *tl = tiles + stage * JT * 4;
#pragma unroll (UNR)
                for (int j = 0; j < JT; ++j) {
                    const float4 P = tl[4 * j], A = tl[4 * j + 1], Bv = tl[4 * j + 2], C = tl[4 * j + 3];
                    const float t[12] = {A.x, A.y, A.z, A.w, Bv.x, Bv.y, Bv.z, Bv.w, C.x, C.y, C.z, C.w};
                    const float m3 = -3.f * P.w;
#pragma unroll
                    for (int k = 0; k < IPT; ++k) {
                        const float dx = P.x - xi[k], dy = P.y - yi[k], dz = P.z - zi[k];
                        const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, e2)));
                        const float inv = rsqrt_approx(r2);
                        const float inv2 = inv * inv;
                        const float inv3 = inv * inv2;
                        const float al = P.w * inv3;
                        const float be = m3 * (inv3 * inv2);
#pragma unroll
                        for (int b = 0; b < kTB; ++b) {
                            const float ux = t[3 * b] - tx[k][b];
                            const float uy = t[3 * b + 1] - ty[k][b];
                            const float uz = t[3 * b + 2] - tz[k][b];
                            const float s = be * fmaf(dz, uz, fmaf(dy, uy, dx * ux));
                            ax[k][b] = fmaf(s, dx, fmaf(al, ux, ax[k][b]));
                            ay[k][b] = fmaf(s, dy, fmaf(al, uy, ay[k][b]));
                            az[k][b] = fmaf(s, dz, fmaf(al, uz, az[k][b]));
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
                bulk_load(tiles + stage * JT * 4, tile_src(u + STAGES), K::TILE_BYTES, &full[stage]);
            }
            if (++stage == STAGES) {
                stage = 0;
                parity ^= 1u;
            }
        }
        if (bad) break;
        const long long sidx = g - sk_owner(ct * per_it, W, G);
        float4 *dst = part + (ct * L.S_max + sidx) * 3LL * K::ITILE;
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const int il = tid + k * NT;
            dst[il] = make_float4(ax[k][0], ay[k][0], az[k][0], ax[k][1]);
            dst[K::ITILE + il] = make_float4(ay[k][1], az[k][1], ax[k][2], ay[k][2]);
            dst[2 * K::ITILE + il] = make_float4(az[k][2], ax[k][3], ay[k][3], az[k][3]);
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
                                           int itile, long long chunk, long long i, float (&f)[12]) {
    const long long it = i / itile, il = i - it * itile;
    const long long ct = chunk * L.n_it + it;
    const long long g0 = sk_owner(ct * L.n_jt, L.W, L.G);
    const long long g1 = sk_owner((ct + 1) * L.n_jt - 1, L.W, L.G);
    const float4 *p = part + ct * L.S_max * 3LL * itile + il;
#pragma unroll
    for (int c = 0; c < 12; ++c) f[c] = 0.f;
    for (long long s = 0; s <= g1 - g0; ++s) {
        const float4 a = __ldg(p + (3 * s) * itile), b = __ldg(p + (3 * s + 1) * itile),
                     c = __ldg(p + (3 * s + 2) * itile);
        const float v[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
#pragma unroll
        for (int q = 0; q < 12; ++q) f[q] += v[q];
    }
}

// Tangent state per (tangent b, body i): dx, dv, dvh as float4 in
// [B][N_pad] arrays; seeds[b] is the body whose own growth is recorded.
struct TangentState {
    float4 *dx, *dv, *dvh;
    float4 *pkt;              // [nchunk][N_pad][4]
    const long long *seeds;   // [B]
    float *growth;            // [cap][B]
    long long cap, base;      // records kept, absolute step at which recording started
    int B, nchunk;
};

// Pack positions (pair-interleaved pk, padded) and tangent positions.
__global__ void tan_pack_kernel(const float *__restrict__ pk, TangentState T, long long N,
                                long long n_pad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int chunk = blockIdx.y;
    if (i >= n_pad) return;
    const float4 x = pk_load(pk, i);
    float t[12];
#pragma unroll
    for (int q = 0; q < kTB; ++q) {
        const long long b = (long long)chunk * kTB + q;
        float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < N && b < T.B) d = T.dx[b * n_pad + i];
        t[3 * q] = d.x;
        t[3 * q + 1] = d.y;
        t[3 * q + 2] = d.z;
    }
    float4 *o = T.pkt + ((long long)chunk * n_pad + i) * 4;
    o[0] = x;
    o[1] = make_float4(t[0], t[1], t[2], t[3]);
    o[2] = make_float4(t[4], t[5], t[6], t[7]);
    o[3] = make_float4(t[8], t[9], t[10], t[11]);
}

// Opening of the tangent: dvh = c1 dv + d1 dF(x^n);  dx' = dx + tau dvh.
// Deformation term's tangent at the packed position of (chunk, i).
__device__ __forceinline__ void tan_defo(const TangentState &T, const Extra &D, int chunk,
                                         long long i, long long n_pad, float (&f)[12]) {
    if (!D.on) return;
    const float4 x = T.pkt[((long long)chunk * n_pad + i) * 4];
#pragma unroll
    for (int q = 0; q < kTB; ++q) {
        const long long b = (long long)chunk * kTB + q;
        if (b >= T.B) break;
        const float4 d = T.dx[b * n_pad + i];
        defo_jacobian<float>(D, x.x, x.y, x.z, d.x, d.y, d.z, f[3 * q], f[3 * q + 1], f[3 * q + 2]);
    }
}

__global__ void tan_open_kernel(const float4 *__restrict__ part, ForceLaunch L, int itile,
                                TangentState T, const StepCoef *__restrict__ table, int tcap,
                                long long step, double tau, long long N, long long n_pad, Extra D) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int chunk = blockIdx.y;
    if (i >= N) return;
    float f[12];
    jvp_reduce(part, L, itile, chunk, i, f);
    tan_defo(T, D, chunk, i, n_pad, f);
    const StepCoef &e = table[step % tcap];
    const float c1 = (float)e.c1, d1 = (float)e.d1, t = (float)tau;
#pragma unroll
    for (int q = 0; q < kTB; ++q) {
        const long long b = (long long)chunk * kTB + q;
        if (b >= T.B) break;
        const long long k = b * n_pad + i;
        const float4 v = T.dv[k];
        const float hx = c1 * v.x + d1 * f[3 * q], hy = c1 * v.y + d1 * f[3 * q + 1],
                    hz = c1 * v.z + d1 * f[3 * q + 2];
        T.dvh[k] = make_float4(hx, hy, hz, 0.f);
        const float4 x = T.dx[k];
        T.dx[k] = make_float4(x.x + t * hx, x.y + t * hy, x.z + t * hz, 0.f);
    }
}

// Step of the tangent after the JVP at x^{n+1}: dv = c2 dvh + d2 dF; record
// the seed body's |(dx, dv)|; open the next step with the next entry's
// coefficients: dvh = c1' dv + d1' dF, dx += tau dvh.
__global__ void tan_step_kernel(const float4 *__restrict__ part, ForceLaunch L, int itile,
                                TangentState T, const StepCoef *__restrict__ table, int tcap,
                                long long step, double tau, long long N, long long n_pad, Extra D) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int chunk = blockIdx.y;
    if (i >= N) return;
    float f[12];
    jvp_reduce(part, L, itile, chunk, i, f);
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
        const float vx = c2 * h.x + d2 * f[3 * q], vy = c2 * h.y + d2 * f[3 * q + 1],
                    vz = c2 * h.z + d2 * f[3 * q + 2];
        const float4 x = T.dx[k];
        T.dv[k] = make_float4(vx, vy, vz, 0.f);
        if (T.seeds[b] == i && T.cap > 0) {
            const long long r = (step - T.base) % T.cap;
            T.growth[r * T.B + b] =
                sqrtf(x.x * x.x + x.y * x.y + x.z * x.z + vx * vx + vy * vy + vz * vz);
        }
        const float nx = c1n * vx + d1n * f[3 * q], ny = c1n * vy + d1n * f[3 * q + 1],
                    nz = c1n * vz + d1n * f[3 * q + 2];
        T.dvh[k] = make_float4(nx, ny, nz, 0.f);
        T.dx[k] = make_float4(x.x + t * nx, x.y + t * ny, x.z + t * nz, 0.f);
    }
}

}  // namespace colatus
