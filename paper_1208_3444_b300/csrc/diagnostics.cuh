// diagnostics.cuh -- FP64 energy and moment reductions of the comoving system.
//
// With the canonical momentum p = m a^2 v of the paper's Hamiltonian section,
// the dynamics of Eq. 1 conserve P = sum m a^2 v and L = sum m a^2 x cross v,
// and K + W obeys the Layzer-Irvine equation d(K+W)/dt = -H (2K + W), with
//   K = (1/2) sum m a^2 |v|^2,   W = W_x / a,
//   W_x = -(G/2) sum_k sum_{j != k} m_k m_j / (|x_k - x_j|^2 + eps^2)^{1/2}.
// Per-block partial sums go to fixed slots and are added in block order by a
// single thread, so the results are deterministic.
#pragma once

#include "common.cuh"
#include "integrate.cuh"

namespace colatus {

constexpr int kDiagThreads = 256;
constexpr int kDiagQ = 12;            // quantities per block
constexpr int kDiagMaxBlocks = 1024;
constexpr int kDiagOut = kDiagMaxBlocks * kDiagQ;
constexpr int kDiagSlots = kDiagOut + 16;

// Sum `v` over the block into slot[0] (FP64, fixed order within the block).
__device__ __forceinline__ void block_sum_to(double v, double *slot) {
    __shared__ double red[kDiagThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < kDiagThreads / 32; ++k) s += red[k];
        *slot = s;
    }
}

// ------------------------------------------------------------- potential
// W_x needs sum_k m_k sum_{j != k} m_j / s_kj.  The pair sums are tiled like
// the force: a block takes kPotITILE target bodies (kPotIPT per thread) and
// one split of the source tiles, staged kPotJT at a time in shared memory, and
// writes its per-body sums to part[split][k]; potential_sum_kernel then adds
// the splits in order and forms sum_k m_k (...).  The self pair is masked in
// the tiles that contain it.  FP32 modes use FP32 pair terms (rsqrt refined by
// one Newton step) summed 64 sources at a time, each partial added in FP64.
constexpr int kPotIPT = 4;
constexpr int kPotJT = 256;
constexpr int kPotITILE = kDiagThreads * kPotIPT;
constexpr int kPotChunk = 64;

// One source tile, pair-interleaved in shared memory (per source pair: x0 x1
// y0 y1 | z0 z1 m0 m1), two sources per f32x2 lane pair; the 64 sources of
// each chunk are summed in FP32 and added to s in FP64.
template <bool MASK>
__device__ __forceinline__ void pot_f32_tile(const float4 *__restrict__ t, long long j0, long long i0,
                                             const float2 (&nx)[kPotIPT], const float2 (&ny)[kPotIPT],
                                             const float2 (&nz)[kPotIPT], float2 e2,
                                             double (&s)[kPotIPT]) {
    const float2 mhalf = make_float2(-0.5f, -0.5f), three_halves = make_float2(1.5f, 1.5f);
    for (int q0 = 0; q0 < kPotJT / 2; q0 += kPotChunk / 2) {
        float2 p[kPotIPT];
#pragma unroll
        for (int k = 0; k < kPotIPT; ++k) p[k] = make_float2(0.f, 0.f);
#pragma unroll 2
        for (int q = q0; q < q0 + kPotChunk / 2; ++q) {
            const float4 A = t[2 * q];      // x0 x1 y0 y1
            const float4 B = t[2 * q + 1];  // z0 z1 m0 m1
            const float2 xj = make_float2(A.x, A.y), yj = make_float2(A.z, A.w);
            const float2 zj = make_float2(B.x, B.y);
#pragma unroll
            for (int k = 0; k < kPotIPT; ++k) {
                const float2 dx = __fadd2_rn(xj, nx[k]), dy = __fadd2_rn(yj, ny[k]),
                             dz = __fadd2_rn(zj, nz[k]);
                float2 r2 = __ffma2_rn(dz, dz, e2);
                r2 = __ffma2_rn(dy, dy, r2);
                r2 = __ffma2_rn(dx, dx, r2);
                float2 y = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                // one Newton step: y (3/2 - r2 y^2 / 2)
                y = __fmul2_rn(y, __ffma2_rn(__fmul2_rn(__fmul2_rn(mhalf, r2), y), y, three_halves));
                float2 w = make_float2(B.z, B.w);
                if (MASK) {
                    const long long i = i0 + threadIdx.x + k * kDiagThreads, j = j0 + 2 * q;
                    if (j == i) w.x = 0.f;
                    if (j + 1 == i) w.y = 0.f;
                }
                p[k] = __ffma2_rn(w, y, p[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < kPotIPT; ++k) s[k] += (double)p[k].x + (double)p[k].y;
    }
}

// Grid (ceil(N / kPotITILE), splits); split y covers source tiles
// [y tps, (y + 1) tps).  Bodies past N (in the last tiles) have zero mass.
__global__ void __launch_bounds__(kDiagThreads)
    potential_f32_kernel(const float4 *__restrict__ xs, long long N, float e2, int tps,
                         double *__restrict__ part) {
    __shared__ __align__(16) float tile[kPotJT * 4];
    const long long i0 = (long long)blockIdx.x * kPotITILE;
    const long long n_jt = (N + kPotJT - 1) / kPotJT;
    const long long jt0 = (long long)blockIdx.y * tps, jt1 = min(jt0 + tps, n_jt);
    float2 nx[kPotIPT], ny[kPotIPT], nz[kPotIPT];
    double s[kPotIPT];
#pragma unroll
    for (int k = 0; k < kPotIPT; ++k) {
        const long long i = i0 + threadIdx.x + k * kDiagThreads;
        const float4 b = i < N ? xs[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        nx[k] = make_float2(-b.x, -b.x);
        ny[k] = make_float2(-b.y, -b.y);
        nz[k] = make_float2(-b.z, -b.z);
        s[k] = 0.0;
    }
    const float2 e22 = make_float2(e2, e2);
    float *slot = tile + (threadIdx.x >> 1) * 8 + (threadIdx.x & 1);
    for (long long jt = jt0; jt < jt1; ++jt) {
        const long long j0 = jt * kPotJT, j = j0 + threadIdx.x;
        const float4 c = j < N ? xs[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        slot[0] = c.x;
        slot[2] = c.y;
        slot[4] = c.z;
        slot[6] = c.w;
        __syncthreads();
        const float4 *t4 = reinterpret_cast<const float4 *>(tile);
        if (j0 < i0 + kPotITILE && j0 + kPotJT > i0)
            pot_f32_tile<true>(t4, j0, i0, nx, ny, nz, e22, s);
        else
            pot_f32_tile<false>(t4, j0, i0, nx, ny, nz, e22, s);
    }
#pragma unroll
    for (int k = 0; k < kPotIPT; ++k) {
        const long long i = i0 + threadIdx.x + k * kDiagThreads;
        if (i < N) part[(long long)blockIdx.y * N + i] = s[k];
    }
}

// The same in FP64 (library rsqrt, FP64 sums).
__global__ void __launch_bounds__(kDiagThreads)
    potential_f64_kernel(const double4 *__restrict__ xs, long long N, double e2, int tps,
                         double *__restrict__ part) {
    __shared__ double4 tile[kPotJT];
    const long long i0 = (long long)blockIdx.x * kPotITILE;
    const long long n_jt = (N + kPotJT - 1) / kPotJT;
    const long long jt0 = (long long)blockIdx.y * tps, jt1 = min(jt0 + tps, n_jt);
    double bx[kPotIPT], by[kPotIPT], bz[kPotIPT], s[kPotIPT];
#pragma unroll
    for (int k = 0; k < kPotIPT; ++k) {
        const long long i = i0 + threadIdx.x + k * kDiagThreads;
        const double4 b = i < N ? xs[i] : make_double4(0.0, 0.0, 0.0, 0.0);
        bx[k] = b.x;
        by[k] = b.y;
        bz[k] = b.z;
        s[k] = 0.0;
    }
    for (long long jt = jt0; jt < jt1; ++jt) {
        const long long j0 = jt * kPotJT, j = j0 + threadIdx.x;
        __syncthreads();
        tile[threadIdx.x] = j < N ? xs[j] : make_double4(0.0, 0.0, 0.0, 0.0);
        __syncthreads();
        const bool diag = j0 < i0 + kPotITILE && j0 + kPotJT > i0;
        for (int jj = 0; jj < kPotJT; ++jj) {
            const double4 c = tile[jj];
#pragma unroll
            for (int k = 0; k < kPotIPT; ++k) {
                const double dx = c.x - bx[k], dy = c.y - by[k], dz = c.z - bz[k];
                const double w = diag && j0 + jj == i0 + threadIdx.x + k * kDiagThreads ? 0.0 : c.w;
                s[k] = fma(w, rsqrt(fma(dx, dx, fma(dy, dy, fma(dz, dz, e2)))), s[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kPotIPT; ++k) {
        const long long i = i0 + threadIdx.x + k * kDiagThreads;
        if (i < N) part[(long long)blockIdx.y * N + i] = s[k];
    }
}

// sum_k m_k sum_split part[split][k], the splits in order, into the block's slot.
__global__ void __launch_bounds__(kDiagThreads)
    potential_sum_kernel(const double *__restrict__ part, int splits, const float4 *__restrict__ xs,
                         const double4 *__restrict__ xs64, int f64, long long N, double *diag) {
    double acc = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N;
         k += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < splits; ++q) s += part[(long long)q * N + k];
        acc += (f64 ? xs64[k].w : (double)xs[k].w) * s;
    }
    block_sum_to(acc, diag + blockIdx.x * kDiagQ + 0);
}

// sum m |v|^2, sum m v, sum m x cross v, sum m x, sum m (FP64).
__global__ void __launch_bounds__(kDiagThreads)
    moments_kernel(const float4 *__restrict__ xs, const float4 *__restrict__ vs,
                   const double4 *__restrict__ xs64, const double4 *__restrict__ vs64, int f64,
                   long long N, double *diag) {
    double q[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N;
         k += (long long)gridDim.x * blockDim.x) {
        double x, y, z, m, u, v, w;
        if (f64) {
            const double4 a = xs64[k], b = vs64[k];
            x = a.x; y = a.y; z = a.z; m = a.w; u = b.x; v = b.y; w = b.z;
        } else {
            const float4 a = xs[k], b = vs[k];
            x = a.x; y = a.y; z = a.z; m = a.w; u = b.x; v = b.y; w = b.z;
        }
        q[0] += m * (u * u + v * v + w * w);
        q[1] += m * u;
        q[2] += m * v;
        q[3] += m * w;
        q[4] += m * (y * w - z * v);
        q[5] += m * (z * u - x * w);
        q[6] += m * (x * v - y * u);
        q[7] += m * x;
        q[8] += m * y;
        q[9] += m * z;
        q[10] += m;
    }
    for (int c = 0; c < 11; ++c) block_sum_to(q[c], diag + blockIdx.x * kDiagQ + 1 + c);
}

// Combine the slots of the nb blocks used into the output record.  Warp c
// sums quantity c: lane l adds blocks l, l + 32, ... in order, then a fixed
// shuffle tree adds the lanes, so the result does not depend on timing.
// Launch with kDiagQ warps.
__global__ void __launch_bounds__(kDiagQ * 32)
    finish_diagnostics_kernel(double *diag, int nb, const DevClock *clk, Cosmo cosmo, double G) {
    __shared__ double s[kDiagQ];
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double v = 0.0;
    for (int b = lane; b < nb; b += 32) v += diag[b * kDiagQ + c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s[c] = v;
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double a = clk->a, a2 = a * a;
    bool bad = false;
    const double H = hubble_of(a, cosmo, bad);
    double *o = diag + kDiagOut;
    const double Wx = -0.5 * G * s[0];
    o[0] = 0.5 * a2 * s[1];
    o[1] = Wx / a;
    for (int q = 0; q < 3; ++q) o[2 + q] = a2 * s[2 + q];
    for (int q = 0; q < 3; ++q) o[5 + q] = a2 * s[5 + q];
    for (int q = 0; q < 3; ++q) o[8 + q] = s[8 + q] / s[11];
    o[11] = a;
    o[12] = clk->t;
    o[13] = bad ? __longlong_as_double(0x7ff8000000000000LL) : H;
    o[14] = Wx;
    o[15] = (double)clk->step;
}

}  // namespace colatus
