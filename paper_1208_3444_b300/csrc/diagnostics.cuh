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

// sum_k m_k sum_{j != k} m_j / s_kj (the self pair is masked).  FP32 modes use
// FP32 pair terms (refined rsqrt) summed in FP64 every 64 sources.
__global__ void __launch_bounds__(kDiagThreads)
    potential_energy_kernel(const float4 *__restrict__ xs, const double4 *__restrict__ xs64,
                            int f64, long long N, double eps2, double *diag) {
    double acc = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N;
         k += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        if (f64) {
            const double4 b = xs64[k];
            for (long long j = 0; j < N; ++j) {
                if (j == k) continue;
                const double4 c = xs64[j];
                const double dx = c.x - b.x, dy = c.y - b.y, dz = c.z - b.z;
                s += c.w * rsqrt(dx * dx + dy * dy + dz * dz + eps2);
            }
            acc += b.w * s;
        } else {
            const float4 b = xs[k];
            const float e2 = (float)eps2;
            for (long long j0 = 0; j0 < N; j0 += 64) {
                float p = 0.f;
                const long long j1 = j0 + 64 < N ? j0 + 64 : N;
                for (long long j = j0; j < j1; ++j) {
                    if (j == k) continue;
                    const float4 c = xs[j];
                    const float dx = c.x - b.x, dy = c.y - b.y, dz = c.z - b.z;
                    const float r2 = dx * dx + dy * dy + dz * dz + e2;
                    float y = rsqrt_approx(r2);
                    y = y * (1.5f - 0.5f * r2 * y * y);
                    p += c.w * y;
                }
                s += (double)p;
            }
            acc += (double)b.w * s;
        }
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

// Combine the block slots (in block order) into the output record.
__global__ void finish_diagnostics_kernel(double *diag, const DevClock *clk, Cosmo cosmo, double G) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s[kDiagQ];
    for (int c = 0; c < kDiagQ; ++c) s[c] = 0.0;
    for (int b = 0; b < kDiagMaxBlocks; ++b)
        for (int c = 0; c < kDiagQ; ++c) s[c] += diag[b * kDiagQ + c];
    const double a = clk->a, a2 = a * a;
    bool bad = false;
    const double H = hubble_of(a, cosmo, bad);
    double *o = diag + kDiagOut;
    const double Wx = -0.5 * G * s[0];
    o[0] = 0.5 * a2 * s[1];
    o[1] = Wx / a;
    for (int c = 0; c < 3; ++c) o[2 + c] = a2 * s[2 + c];
    for (int c = 0; c < 3; ++c) o[5 + c] = a2 * s[5 + c];
    for (int c = 0; c < 3; ++c) o[8 + c] = s[8 + c] / s[11];
    o[11] = a;
    o[12] = clk->t;
    o[13] = bad ? __longlong_as_double(0x7ff8000000000000LL) : H;
    o[14] = Wx;
    o[15] = (double)clk->step;
}

}  // namespace colatus
