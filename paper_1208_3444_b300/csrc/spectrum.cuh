// spectrum.cuh -- one-sided energy spectrum of tracer velocity records
// (Sec. I and Sec. IV: the velocity of single bodies at every step and its
// energy power spectrum, the statistic of chaotic advection).
//
// Input: T samples per tracer at uniform spacing dt; sample n of tracer k,
// component c is at base[row(n) * row_stride + k * tr_stride + c] with
// row(n) = (first + n) mod cap (the tracer ring is read oldest first, in place).
// Per tracer, u = v - mean(v) (detrend) or v, w the rectangular or periodic
// Hann window, U = (1/T) sum w^2:
//     E_k(f_j) = c_j dt / (T U) * 1/2 sum_c |sum_n w_n u_{n,k,c} exp(-2 pi i j n / T)|^2,
// j = 0 .. T/2, c_j = 2 except for j = 0 and j = T/2 (T even).
//
// One block per (tracer, chunk of 256 frequencies); the block stages the
// windowed series in shared memory, 512 samples at a time, and every thread
// accumulates one frequency in FP64.  The twiddle of (j, n) is the table entry
// (j n mod T), so the angle is reduced exactly before any rounding.
#pragma once

#include "common.cuh"

namespace colatus {

constexpr int kSpecThreads = 256;
constexpr int kSpecChunk = 512;

struct SpecSeries {
    const void *base;          // first velocity component of row 0, tracer 0
    long long T, ntr;          // samples, tracers
    long long row_stride;      // elements between consecutive rows
    long long tr_stride;       // elements between consecutive tracers
    long long first, cap;      // sample n lives in row (first + n) % cap
    int f64;                   // element type: double (1) or float (0)
};

// tw[m] = (cos, sin)(2 pi m / T)
__global__ void spectrum_twiddle_kernel(double2 *tw, long long T) {
    const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= T) return;
    double s, c;
    sincospi(2.0 * (double)m / (double)T, &s, &c);
    tw[m] = make_double2(c, s);
}

__device__ __forceinline__ double spec_load(const SpecSeries &S, long long n, long long k, int c) {
    const long long r = (S.first + n) % S.cap;
    const long long off = r * S.row_stride + k * S.tr_stride + c;
    return S.f64 ? static_cast<const double *>(S.base)[off]
                 : (double)static_cast<const float *>(S.base)[off];
}

__device__ __forceinline__ double spec_window(const double2 *tw, long long n, int window) {
    return window ? 0.5 - 0.5 * tw[n].x : 1.0;
}

// Block-wide sum of four doubles (blockDim.x == kSpecThreads).
__device__ __forceinline__ void spec_block_sum4(double (&v)[4], double *red) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) red[warp * 4 + q] = v[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        double s = 0.0;
        for (int w = 0; w < kSpecThreads / 32; ++w) s += red[w * 4 + q];
        v[q] = s;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kSpecThreads)
spectrum_kernel(SpecSeries S, const double2 *__restrict__ tw, double dt, int window, int detrend,
                double *__restrict__ E) {
    __shared__ double3 su[kSpecChunk];
    __shared__ double red[(kSpecThreads / 32) * 4];
    const long long k = blockIdx.x;
    const long long T = S.T, nf = T / 2 + 1;
    const long long j = (long long)blockIdx.y * kSpecThreads + threadIdx.x;

    // per-component means and the window's mean square U
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long n = threadIdx.x; n < T; n += kSpecThreads) {
        const double w = spec_window(tw, n, window);
        if (detrend) {
            acc[0] += spec_load(S, n, k, 0);
            acc[1] += spec_load(S, n, k, 1);
            acc[2] += spec_load(S, n, k, 2);
        }
        acc[3] += w * w;
    }
    spec_block_sum4(acc, red);
    const double inv_T = 1.0 / (double)T;
    const double mx = acc[0] * inv_T, my = acc[1] * inv_T, mz = acc[2] * inv_T;
    const double U = acc[3] * inv_T;

    double re[3] = {0.0, 0.0, 0.0}, im[3] = {0.0, 0.0, 0.0};
    for (long long n0 = 0; n0 < T; n0 += kSpecChunk) {
        const int len = (int)min((long long)kSpecChunk, T - n0);
        for (int q = threadIdx.x; q < len; q += kSpecThreads) {
            const long long n = n0 + q;
            const double w = spec_window(tw, n, window);
            su[q] = make_double3(w * (spec_load(S, n, k, 0) - mx), w * (spec_load(S, n, k, 1) - my),
                                 w * (spec_load(S, n, k, 2) - mz));
        }
        __syncthreads();
        if (j < nf) {
            long long m = (j * n0) % T;   // j < T, n0 < T: fits in 64 bits
            for (int q = 0; q < len; ++q) {
                const double2 e = __ldg(&tw[m]);
                const double3 u = su[q];
                // exp(-i theta) = cos - i sin
                re[0] = fma(u.x, e.x, re[0]);
                im[0] = fma(-u.x, e.y, im[0]);
                re[1] = fma(u.y, e.x, re[1]);
                im[1] = fma(-u.y, e.y, im[1]);
                re[2] = fma(u.z, e.x, re[2]);
                im[2] = fma(-u.z, e.y, im[2]);
                m += j;
                if (m >= T) m -= T;
            }
        }
        __syncthreads();
    }
    if (j < nf) {
        const double cj = (j == 0 || 2 * j == T) ? 1.0 : 2.0;
        const double p = re[0] * re[0] + im[0] * im[0] + re[1] * re[1] + im[1] * im[1] +
                         re[2] * re[2] + im[2] * im[2];
        E[k * nf + j] = cj * dt / ((double)T * U) * 0.5 * p;
    }
}

}  // namespace colatus
