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
// Two kernels compute the same sums, both in FP64 with every twiddle angle
// reduced exactly (table entry (e mod T) of exp(2 pi i e / T)):
//
// * spectrum_fft_kernel, for T <= kSpecFftMaxT whose prime factors are all
//   <= kSpecFftMaxP: a mixed-radix Stockham FFT in shared memory (radix-4 and
//   radix-5 butterflies written out, other radices as direct p-point sums).  A cluster of two CTAs per tracer: CTA 0 transforms the
//   complex series u_x + i u_y, CTA 1 the series u_z; the sum over components
//   of the real series' power is (|Z_j|^2 + |Z_{T-j}|^2) / 2 for either, and
//   CTA 0 reads CTA 1's transform through distributed shared memory.
// * spectrum_kernel otherwise: the direct sum, one block per (tracer, chunk
//   of 256 frequencies); the block stages the windowed series in shared
//   memory, 512 samples at a time, and every thread accumulates one frequency.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"

namespace colatus {

constexpr int kSpecThreads = 256;
constexpr int kSpecChunk = 512;
constexpr int kSpecFftMaxT = 6144;       // two complex FP64 buffers of T: 192 KB of shared memory
constexpr int kSpecFftMaxP = 64;         // largest radix taken as one stage
constexpr int kSpecFftMaxStages = 16;    // 4^6 > kSpecFftMaxT, so at most 13 factors

// Radices of the FFT stages, in order (T = p[0] p[1] ... p[nst-1]).
struct SpecPlan {
    int nst;
    int p[kSpecFftMaxStages];
};

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

// Requires 0 <= first < cap and n < T <= cap, so first + n < 2 cap.
__device__ __forceinline__ double spec_load(const SpecSeries &S, long long n, long long k, int c) {
    long long r = S.first + n;
    if (r >= S.cap) r -= S.cap;
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

// Stockham stage of radix p over N = T points: with L the length of the
// transforms done so far and m = N / (p L), the input holds the L-point
// transforms Y_r (r < p m) at [r L, r L + L), and output o = k p L + j'
// (k < m, j' < p L) is the p L-point transform
//     Z_k[j'] = sum_q exp(-2 pi i q m j' / N) Y_{k + m q}[j' mod L].
// Radix 4 and 5 take one butterfly per thread: the inputs a_q =
// Y_{k + m q}[j] exp(-2 pi i q m j / N) (q m j < N) and their p-point DFT
// written out; other radices take one output per thread, the exponent
// q m j' advanced by m j' < N and reduced by one subtraction.

// v exp(-i theta) for the table entry c = (cos theta, sin theta)
__device__ __forceinline__ double2 spec_rot(double2 v, double2 c) {
    return make_double2(fma(v.x, c.x, v.y * c.y), fma(v.y, c.x, -(v.x * c.y)));
}

__device__ __forceinline__ void spec_fft_stage(const double2 *__restrict__ src,
                                               double2 *__restrict__ dst,
                                               const double2 *__restrict__ tw, int N, int p, int L) {
    const int pL = p * L, m = N / pL, step = m * L;
    if (p == 4) {
        for (int b = threadIdx.x; b < N / 4; b += kSpecThreads) {
            const int k = b / L, j = b - k * L, e = m * j;
            const double2 *y = src + k * L + j;
            const double2 a0 = y[0], a1 = spec_rot(y[step], __ldg(&tw[e])),
                          a2 = spec_rot(y[2 * step], __ldg(&tw[2 * e])),
                          a3 = spec_rot(y[3 * step], __ldg(&tw[3 * e]));
            const double2 t0 = make_double2(a0.x + a2.x, a0.y + a2.y);
            const double2 t1 = make_double2(a0.x - a2.x, a0.y - a2.y);
            const double2 t2 = make_double2(a1.x + a3.x, a1.y + a3.y);
            const double2 t3 = make_double2(a1.y - a3.y, a3.x - a1.x);   // -i (a1 - a3)
            double2 *z = dst + k * pL + j;
            z[0] = make_double2(t0.x + t2.x, t0.y + t2.y);
            z[L] = make_double2(t1.x + t3.x, t1.y + t3.y);
            z[2 * L] = make_double2(t0.x - t2.x, t0.y - t2.y);
            z[3 * L] = make_double2(t1.x - t3.x, t1.y - t3.y);
        }
        return;
    }
    if (p == 5) {
        // cos and sin of 2 pi / 5 and 4 pi / 5 from the table (N is a multiple of 5)
        const double2 w1 = __ldg(&tw[N / 5]), w2 = __ldg(&tw[2 * (N / 5)]);
        for (int b = threadIdx.x; b < N / 5; b += kSpecThreads) {
            const int k = b / L, j = b - k * L, e = m * j;
            const double2 *y = src + k * L + j;
            const double2 a0 = y[0], a1 = spec_rot(y[step], __ldg(&tw[e])),
                          a2 = spec_rot(y[2 * step], __ldg(&tw[2 * e])),
                          a3 = spec_rot(y[3 * step], __ldg(&tw[3 * e])),
                          a4 = spec_rot(y[4 * step], __ldg(&tw[4 * e]));
            const double2 b1 = make_double2(a1.x + a4.x, a1.y + a4.y);
            const double2 b2 = make_double2(a2.x + a3.x, a2.y + a3.y);
            const double2 d1 = make_double2(a1.x - a4.x, a1.y - a4.y);
            const double2 d2 = make_double2(a2.x - a3.x, a2.y - a3.y);
            const double2 r1 = make_double2(fma(w2.x, b2.x, fma(w1.x, b1.x, a0.x)),
                                            fma(w2.x, b2.y, fma(w1.x, b1.y, a0.y)));
            const double2 r2 = make_double2(fma(w1.x, b2.x, fma(w2.x, b1.x, a0.x)),
                                            fma(w1.x, b2.y, fma(w2.x, b1.y, a0.y)));
            const double2 i1 = make_double2(fma(w2.y, d2.x, w1.y * d1.x), fma(w2.y, d2.y, w1.y * d1.y));
            const double2 i2 = make_double2(fma(-w1.y, d2.x, w2.y * d1.x), fma(-w1.y, d2.y, w2.y * d1.y));
            // Z_1 = r1 - i i1, Z_4 = r1 + i i1, Z_2 = r2 - i i2, Z_3 = r2 + i i2
            double2 *z = dst + k * pL + j;
            z[0] = make_double2(a0.x + b1.x + b2.x, a0.y + b1.y + b2.y);
            z[L] = make_double2(r1.x + i1.y, r1.y - i1.x);
            z[4 * L] = make_double2(r1.x - i1.y, r1.y + i1.x);
            z[2 * L] = make_double2(r2.x + i2.y, r2.y - i2.x);
            z[3 * L] = make_double2(r2.x - i2.y, r2.y + i2.x);
        }
        return;
    }
    for (int o = threadIdx.x; o < N; o += kSpecThreads) {
        const int kk = o / pL, jp = o - kk * pL, j = jp % L;
        const int de = m * jp;
        const double2 *y = src + kk * L + j;
        double re = 0.0, im = 0.0;
        int e = 0;
        for (int q = 0; q < p; ++q) {
            const double2 c = __ldg(&tw[e]);
            const double2 v = y[q * step];
            // v (cos - i sin)
            re = fma(v.x, c.x, re);
            re = fma(v.y, c.y, re);
            im = fma(v.y, c.x, im);
            im = fma(-v.x, c.y, im);
            e += de;
            if (e >= N) e -= N;
        }
        dst[o] = make_double2(re, im);
    }
}

// Grid (ntr, 2), clusters of (1, 2): block rank 0 transforms u_x + i u_y and
// writes E, block rank 1 transforms u_z.  Dynamic shared memory: 2 T double2.
__global__ void __cluster_dims__(1, 2, 1) __launch_bounds__(kSpecThreads)
spectrum_fft_kernel(SpecSeries S, const double2 *__restrict__ tw, SpecPlan plan, double dt,
                    int window, int detrend, double *__restrict__ E) {
    extern __shared__ double2 spec_buf[];
    __shared__ double red[(kSpecThreads / 32) * 4];
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int s = (int)cluster.block_rank();
    const long long k = blockIdx.x;
    const int N = (int)S.T;
    const long long nf = N / 2 + 1;
    const int c0 = s == 0 ? 0 : 2;

    // means of this block's components and the window's mean square U
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int n = threadIdx.x; n < N; n += kSpecThreads) {
        const double w = spec_window(tw, n, window);
        if (detrend) {
            acc[0] += spec_load(S, n, k, c0);
            if (s == 0) acc[1] += spec_load(S, n, k, 1);
        }
        acc[3] += w * w;
    }
    spec_block_sum4(acc, red);
    const double inv_T = 1.0 / (double)N;
    const double m0 = acc[0] * inv_T, m1 = acc[1] * inv_T, U = acc[3] * inv_T;

    double2 *src = spec_buf, *dst = spec_buf + N;
    for (int n = threadIdx.x; n < N; n += kSpecThreads) {
        const double w = spec_window(tw, n, window);
        src[n] = make_double2(w * (spec_load(S, n, k, c0) - m0),
                              s == 0 ? w * (spec_load(S, n, k, 1) - m1) : 0.0);
    }
    __syncthreads();
    int L = 1;
    for (int st = 0; st < plan.nst; ++st) {
        spec_fft_stage(src, dst, tw, N, plan.p[st], L);
        __syncthreads();
        double2 *t = src;
        src = dst;
        dst = t;
        L *= plan.p[st];
    }

    // both transforms complete; block 0 reads block 1's through DSMEM
    cluster.sync();
    if (s == 0) {
        const double2 *z = cluster.map_shared_rank(src, 1);
        const double scale = dt / ((double)N * U) * 0.5 * 0.5;
        for (int j = threadIdx.x; j < nf; j += kSpecThreads) {
            const int jm = j == 0 ? 0 : N - j;
            const double2 a = src[j], b = src[jm], c = z[j], d = z[jm];
            const double pxy = a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y;
            const double pz = c.x * c.x + c.y * c.y + d.x * d.x + d.y * d.y;
            const double cj = (j == 0 || 2 * j == N) ? 1.0 : 2.0;
            E[k * nf + j] = cj * scale * (pxy + pz);
        }
    }
    // block 1's shared memory stays alive until block 0 has read it
    cluster.sync();
}

}  // namespace colatus
