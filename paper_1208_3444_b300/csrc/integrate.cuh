// integrate.cuh -- everything around the force sum: the FP64 Friedmann
// schedule (Eq. 2), packing of bodies into the force kernels' layout, the
// fixed-order reduction of force segments, and the fused kick / drift /
// tracer-record epilogues of the Hubble-drag leapfrog (Eqs. 3-5 and KDK).
#pragma once

#include "common.cuh"
#include "force.cuh"
#include "sym_reduce.cuh"

namespace colatus {

// ------------------------------------------------------------ Friedmann (Eq. 2)
// da/dt = a H(a),  H = H0 sqrt(Omega_R a^-4 + Omega_M a^-3 + Omega_K a^-2 + Omega_L).
// With P(a) = a^4 (Omega_R a^-4 + ...) = Omega_R + Omega_M a + Omega_K a^2 +
// Omega_L a^4, a H = H0 sqrt(P) / a = H0 P rsqrt(P a^2): one reciprocal
// square root and no division per evaluation (FP64 is scarce on this GPU).
__device__ inline double friedmann_rhs(double a, const Cosmo &c, bool &bad) {
    const double a2 = a * a;
    const double P = c.Omega_R + a * (c.Omega_M + a * (c.Omega_K + c.Omega_L * a2));
    if (!(P > 0.0) || !(a > 0.0)) {
        bad = bad || !(P >= 0.0) || !(a > 0.0);
        return 0.0;
    }
    return c.H0 * P * rsqrt(P * a2);
}

__device__ inline double hubble_of(double a, const Cosmo &c, bool &bad) {
    return friedmann_rhs(a, c, bad) / a;
}

// Classical RK4 with nsub equal sub-steps over dt, on the system
// (a, I1, I2)' = (a H(a), 1/a, 1/a^2): I1 and I2 accumulate int dt/a and
// int dt/a^2, the kick and drift factors of the canonical leapfrog.  The
// a-chain is the same instruction sequence with or without the integrals
// (INTEG), so a(t) is bitwise the same for every scheme; the drag schemes
// skip the integrals and their four FP64 divisions per sub-step (this GPU's
// FP64 pipe takes about 16 cycles per warp instruction, even for one thread).
template <bool INTEG>
__device__ inline double friedmann_advance(double a, double dt, const Cosmo &c, int nsub,
                                           bool &bad, double &I1, double &I2) {
    const double h = dt / nsub, h6 = h / 6.0;
    for (int s = 0; s < nsub; ++s) {
        const double s2 = a;
        const double k1 = friedmann_rhs(s2, c, bad);
        const double s3 = a + 0.5 * h * k1;
        const double k2 = friedmann_rhs(s3, c, bad);
        const double s4 = a + 0.5 * h * k2;
        const double k3 = friedmann_rhs(s4, c, bad);
        const double s5 = a + h * k3;
        const double k4 = friedmann_rhs(s5, c, bad);
        if (INTEG) {
            const double r1 = 1.0 / s2, r2 = 1.0 / s3, r3 = 1.0 / s4, r4 = 1.0 / s5;
            I1 += h6 * (r1 + 2.0 * r2 + 2.0 * r3 + r4);
            I2 += h6 * (r1 * r1 + 2.0 * (r2 * r2) + 2.0 * (r3 * r3) + r4 * r4);
        }
        a = a + h6 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
    }
    return a;
}

// Kick over span h at (a, H): c = (1 - H h)/(1 + H h), d = G h / (a^3 (1 + H h)).
__device__ inline void kick_coef(double a, double H, double h, double G, double &c, double &d) {
    c = (1.0 - H * h) / (1.0 + H * h);
    d = G * h / (a * a * a * (1.0 + H * h));
}

// One thread: extend the look-ahead schedule by n steps of size tau from its
// frontier `tclk` (a, t and the absolute index of the next step), writing
// the entry of step s to table[s % tcap].  The per-step sequence (advance
// tau/2 to t^{n+1/2}, then tau/2 to t^{n+1}) is the same for every scheme,
// so a(t) does not depend on the scheme.  canonical != 0 replaces the KDK
// coefficients by those of the canonical (symplectic) leapfrog of Sec. II:
// p = a^2 v, kick p += G F int dt/a, drift x += p int dt/a^2, written in the
// velocity form vh = c1 v + d1 F, x' = x + tau vh, v' = c2 vh + d2 F with
// c1 = (D/tau) a0^2, d1 = G (D/tau) K1, c2 = tau / (D a1^2), d2 = G K2 / a1^2
// (K1, K2: int dt/a over the half steps; D: int dt/a^2 over the step).  A
// negative Eq. 2 radicand marks the entry bad; the step that consumes it
// raises FLAG_FRIEDMANN.
__global__ void friedmann_table_kernel(Cosmo cosmo, DevClock *tclk, StepCoef *table, int tcap,
                                       int n, double tau, double G, int nsub, int canonical) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double a = tclk->a, t = tclk->t;
    const long long step0 = tclk->step;
    for (int j = 0; j < n; ++j) {
        bool bad = false;
        StepCoef s;
        double K1 = 0.0, K2 = 0.0, D = 0.0;
        s.a0 = a;
        if (canonical) {
            s.ah = friedmann_advance<true>(a, 0.5 * tau, cosmo, nsub, bad, K1, D);
            s.a1 = friedmann_advance<true>(s.ah, 0.5 * tau, cosmo, nsub, bad, K2, D);
        } else {
            s.ah = friedmann_advance<false>(a, 0.5 * tau, cosmo, nsub, bad, K1, D);
            s.a1 = friedmann_advance<false>(s.ah, 0.5 * tau, cosmo, nsub, bad, K2, D);
        }
        kick_coef(s.ah, hubble_of(s.ah, cosmo, bad), tau, G, s.c, s.d);
        if (canonical) {
            const double Dt = D / tau;
            s.c1 = Dt * (s.a0 * s.a0);
            s.d1 = G * Dt * K1;
            s.c2 = tau / (D * (s.a1 * s.a1));
            s.d2 = G * K2 / (s.a1 * s.a1);
        } else {
            kick_coef(s.a0, hubble_of(s.a0, cosmo, bad), 0.5 * tau, G, s.c1, s.d1);
            kick_coef(s.a1, hubble_of(s.a1, cosmo, bad), 0.5 * tau, G, s.c2, s.d2);
        }
        t = t + tau;
        s.t1 = t;
        s.step = step0 + j;
        s.bad = bad ? 1 : 0;
        s.pad = 0;
        if (bad) {
            const double nan = __longlong_as_double(0x7ff8000000000000LL);
            s.c = s.d = s.c1 = s.d1 = s.c2 = s.d2 = nan;
        }
        table[(step0 + j) % tcap] = s;
        a = s.a1;
    }
    tclk->a = a;
    tclk->t = t;
    tclk->step = step0 + n;
}

// Copy the state clock into the schedule frontier (schedule restart).
__global__ void clock_copy_kernel(const DevClock *src, DevClock *dst) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *dst = *src;
}

// The state clock follows the step just completed; a bad schedule entry
// raises FLAG_FRIEDMANN.  Called by one thread of each step's epilogue.
__device__ __forceinline__ void advance_clock(DevClock *clk, const StepCoef &e, int *flags) {
    clk->a = e.a1;
    clk->t = e.t1;
    clk->step = e.step + 1;
    if (e.bad) atomicOr(&flags[FLAG_FRIEDMANN], 1);
}

// ---------------------------------------------------------------- packing
// FP32 force input: pair-interleaved [x0 x1 y0 y1 z0 z1 m0 m1]; bodies
// i >= N (padding up to N_pad) are zero-mass at the origin and contribute
// exactly zero.
__device__ __forceinline__ void pk_store(float *pk, long long i, float x, float y, float z, float m) {
    float *p = pk + (i >> 1) * 8 + (i & 1);
    p[0] = x;
    p[2] = y;
    p[4] = z;
    p[6] = m;
}

__device__ __forceinline__ float4 pk_load(const float *pk, long long i) {
    const float *p = pk + (i >> 1) * 8 + (i & 1);
    return make_float4(p[0], p[2], p[4], p[6]);
}

__global__ void pack_f32_kernel(const float4 *__restrict__ xs, float *__restrict__ pk, long long N,
                                long long N_pad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    if (i < N) {
        const float4 b = xs[i];
        pk_store(pk, i, b.x, b.y, b.z, b.w);
    } else {
        pk_store(pk, i, 0.f, 0.f, 0.f, 0.f);
    }
}

__global__ void pack_f64_kernel(const double4 *__restrict__ xs, double4 *__restrict__ pos,
                                long long N, long long N_pad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    pos[i] = i < N ? xs[i] : make_double4(0.0, 0.0, 0.0, 0.0);
}

// ------------------------------------------------------- segment reduction
// Loads in flight per thread in the pair-once epilogues' sums.
constexpr int kSymEpiBatch = 4;

// Sum the segments of body i's i-tile in CTA order (deterministic).  Loads
// are issued four at a time so that several are in flight per thread; the
// additions keep the fixed order.  (Plans that evaluate each pair once sum
// through reduce_sym_f32.)
template <bool COMP>
__device__ __forceinline__ float3 reduce_f32(const float4 *__restrict__ part, const ForceLaunch &L,
                                             int itile, long long i) {
    const long long it = i / itile, il = i - it * itile;
    const long long G = L.G, W = L.W;
    const long long g0 = sk_owner(it * L.n_jt, W, G);
    const long long g1 = sk_owner((it + 1) * L.n_jt - 1, W, G);
    const int ns = (int)(g1 - g0 + 1);
    const int plane = COMP ? 2 : 1;
    const float4 *p = part + it * L.S_max * plane * (long long)itile + il;
    const long long step = (long long)plane * itile;
    if (!COMP) {
        float fx = 0.f, fy = 0.f, fz = 0.f;
        int s = 0;
        for (; s + 4 <= ns; s += 4) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = __ldg(p + (s + u) * step);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                fx += v[u].x;
                fy += v[u].y;
                fz += v[u].z;
            }
        }
        for (; s < ns; ++s) {
            const float4 v = __ldg(p + s * step);
            fx += v.x;
            fy += v.y;
            fz += v.z;
        }
        return make_float3(fx, fy, fz);
    } else {
        float hx = 0.f, hy = 0.f, hz = 0.f, lx = 0.f, ly = 0.f, lz = 0.f;
        int s = 0;
        for (; s + 4 <= ns; s += 4) {
            float4 h[4], l[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                h[u] = __ldg(p + (s + u) * step);
                l[u] = __ldg(p + (s + u) * step + itile);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                acc2_add(hx, lx, h[u].x);
                acc2_add(hy, ly, h[u].y);
                acc2_add(hz, lz, h[u].z);
                lx += l[u].x;
                ly += l[u].y;
                lz += l[u].z;
            }
        }
        for (; s < ns; ++s) {
            const float4 h = __ldg(p + s * step), l = __ldg(p + s * step + itile);
            acc2_add(hx, lx, h.x);
            acc2_add(hy, ly, h.y);
            acc2_add(hz, lz, h.z);
            lx += l.x;
            ly += l.y;
            lz += l.z;
        }
        return make_float3(hx + lx, hy + ly, hz + lz);
    }
}

__device__ __forceinline__ double3 reduce_f64(const double4 *__restrict__ part, const ForceLaunch &L,
                                              int itile, long long i) {
    const long long it = i / itile, il = i - it * itile;
    const long long G = L.G, W = L.W;
    const long long g0 = sk_owner(it * L.n_jt, W, G);
    const long long g1 = sk_owner((it + 1) * L.n_jt - 1, W, G);
    const double4 *p = part + it * L.S_max * (long long)itile + il;
    double3 f = make_double3(0.0, 0.0, 0.0);
    for (long long s = 0; s <= g1 - g0; ++s) {
        const double4 v = p[s * itile];
        f.x += v.x;
        f.y += v.y;
        f.z += v.z;
    }
    return f;
}

// out (N x 3, float or double) = G a^-3 F at the device clock's a (the
// comoving acceleration of Eq. 1); optionally cache the G-less F in acc.
// SYM: the plan evaluates each pair once (reduce_sym_f32), else every ordered
// pair (reduce_f32).
template <bool COMP, bool SYM>
__global__ void forces_out_f32_kernel(const float4 *__restrict__ part, ForceLaunch L, int itile,
                                      long long N, const DevClock *__restrict__ clk, double G,
                                      void *out, int out_f64, float4 *__restrict__ acc,
                                      const float *__restrict__ pk, Extra D) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double a = clk->a;
    const float scale = (float)(G / (a * a * a));
    float3 f = SYM ? reduce_sym_f32<COMP, kSymEpiBatch>(part, L, itile, i) : reduce_f32<COMP>(part, L, itile, i);
    if (D.on) {
        const float4 x = pk_load(pk, i);
        defo_force(D, x.x, x.y, x.z, f.x, f.y, f.z);
    }
    add_long_range(D, i, f.x, f.y, f.z);
    if (acc) acc[i] = make_float4(f.x, f.y, f.z, 0.f);
    if (out) {
        if (out_f64) {
            double *o = static_cast<double *>(out) + 3 * i;
            o[0] = (double)(scale * f.x);
            o[1] = (double)(scale * f.y);
            o[2] = (double)(scale * f.z);
        } else {
            float *o = static_cast<float *>(out) + 3 * i;
            o[0] = scale * f.x;
            o[1] = scale * f.y;
            o[2] = scale * f.z;
        }
    }
}

__global__ void forces_out_f64_kernel(const double4 *__restrict__ part, ForceLaunch L, int itile,
                                      long long N, const DevClock *__restrict__ clk, double G,
                                      void *out, int out_f64, double4 *__restrict__ acc,
                                      const double4 *__restrict__ pos, Extra D) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double a = clk->a;
    const double scale = G / (a * a * a);
    double3 f = reduce_f64(part, L, itile, i);
    if (D.on) {
        const double4 x = pos[i];
        defo_force(D, x.x, x.y, x.z, f.x, f.y, f.z);
    }
    add_long_range(D, i, f.x, f.y, f.z);
    if (acc) acc[i] = make_double4(f.x, f.y, f.z, 0.0);
    if (out) {
        if (out_f64) {
            double *o = static_cast<double *>(out) + 3 * i;
            o[0] = scale * f.x;
            o[1] = scale * f.y;
            o[2] = scale * f.z;
        } else {
            float *o = static_cast<float *>(out) + 3 * i;
            o[0] = (float)(scale * f.x);
            o[1] = (float)(scale * f.y);
            o[2] = (float)(scale * f.z);
        }
    }
}

// ------------------------------------------------------------- tracer record
struct Tracers {
    const int *slot;   // [N]: -1, or the tracer's column
    float *rec;        // [cap][ntr][6]
    long long cap;     // records kept
    long long base;    // absolute step at which recording started
    int ntr;
};

template <typename T>
__device__ __forceinline__ void record(const Tracers &tr, long long i, long long step, T x, T y, T z,
                                       T vx, T vy, T vz) {
    if (tr.ntr == 0) return;
    const int s = tr.slot[i];
    if (s < 0) return;
    const long long r = (step - tr.base) % tr.cap;
    float *o = tr.rec + (r * tr.ntr + s) * 6;
    o[0] = (float)x;
    o[1] = (float)y;
    o[2] = (float)z;
    o[3] = (float)vx;
    o[4] = (float)vy;
    o[5] = (float)vz;
}

__device__ __forceinline__ bool finite3(float a, float b, float c) {
    return isfinite(a) && isfinite(b) && isfinite(c);
}
__device__ __forceinline__ bool finite3(double a, double b, double c) {
    return isfinite(a) && isfinite(b) && isfinite(c);
}

// --------------------------------------------------------------- FP32 steps
// KDK opening half kick + drift of step j from the state:
//   vh = c1 v + d1 F(x);  x' = x + tau vh  (packed into pk_out)
__global__ void kdk_open_f32_kernel(const float4 *__restrict__ xs, const float4 *__restrict__ vs,
                                    const float4 *__restrict__ acc, float4 *__restrict__ vh,
                                    float *__restrict__ pk_out, const StepCoef *__restrict__ table,
                                    int tcap, long long step, double tau, long long N, long long N_pad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    if (i >= N) {
        pk_store(pk_out, i, 0.f, 0.f, 0.f, 0.f);
        return;
    }
    const float c1 = (float)table[step % tcap].c1, d1 = (float)table[step % tcap].d1, t = (float)tau;
    const float4 x = xs[i], v = vs[i], F = acc[i];
    const float hx = kick2(c1, v.x, d1, F.x), hy = kick2(c1, v.y, d1, F.y), hz = kick2(c1, v.z, d1, F.z);
    vh[i] = make_float4(hx, hy, hz, 0.f);
    pk_store(pk_out, i, drift1(x.x, t, hx), drift1(x.y, t, hy), drift1(x.z, t, hz), x.w);
}

// KDK step j, after the force at x^{n+1} (pk_in):
//   v^{n+1} = c2 vh + d2 F;  record;  next step's opening with the next
//   entry's coefficients: vh = c1' v^{n+1} + d1' F;  x^{n+2} = x^{n+1} + tau vh.
// (For the drag scheme c1', d1' equal c2, d2 bit for bit: both are the half
// kick at t^{n+1}.)
// SYM as in forces_out_f32_kernel.
template <bool COMP, bool SYM>
__global__ void kdk_step_f32_kernel(const float4 *__restrict__ part, ForceLaunch L, int itile,
                                    const float *__restrict__ pk_in, float4 *__restrict__ xs,
                                    float4 *__restrict__ vs, float4 *__restrict__ vh,
                                    float4 *__restrict__ acc, float *__restrict__ pk_out,
                                    const StepCoef *__restrict__ table, int tcap, long long step, double tau,
                                    long long N, long long N_pad, Tracers tr, int *flags, DevClock *clk, Extra D) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    if (i >= N) {
        pk_store(pk_out, i, 0.f, 0.f, 0.f, 0.f);
        return;
    }
    const StepCoef &sc = table[step % tcap];
    const StepCoef &nc = table[(step + 1) % tcap];
    if (i == 0) advance_clock(clk, sc, flags);
    const float c2 = (float)sc.c2, d2 = (float)sc.d2, t = (float)tau;
    const float c1n = (float)nc.c1, d1n = (float)nc.d1;
    float3 F = SYM ? reduce_sym_f32<COMP, kSymEpiBatch>(part, L, itile, i) : reduce_f32<COMP>(part, L, itile, i);
    const float4 x = pk_load(pk_in, i);
    defo_force(D, x.x, x.y, x.z, F.x, F.y, F.z);
    add_long_range(D, i, F.x, F.y, F.z);
    const float4 h = vh[i];
    const float vx = kick2(c2, h.x, d2, F.x), vy = kick2(c2, h.y, d2, F.y), vz = kick2(c2, h.z, d2, F.z);
    acc[i] = make_float4(F.x, F.y, F.z, 0.f);
    xs[i] = x;
    vs[i] = make_float4(vx, vy, vz, 0.f);
    record(tr, i, sc.step, x.x, x.y, x.z, vx, vy, vz);
    const float nx = kick2(c1n, vx, d1n, F.x), ny = kick2(c1n, vy, d1n, F.y), nz = kick2(c1n, vz, d1n, F.z);
    vh[i] = make_float4(nx, ny, nz, 0.f);
    pk_store(pk_out, i, drift1(x.x, t, nx), drift1(x.y, t, ny), drift1(x.z, t, nz), x.w);
    if (!finite3(x.x, x.y, x.z) || !finite3(vx, vy, vz)) atomicOr(&flags[FLAG_NONFINITE], 1);
}

// DKD opening half drift: x^{n+1/2} = x^n + (tau/2) v^n (packed).
__global__ void dkd_open_f32_kernel(const float4 *__restrict__ xs, const float4 *__restrict__ vs,
                                    float *__restrict__ pk_out, double tau, long long N,
                                    long long N_pad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    if (i >= N) {
        pk_store(pk_out, i, 0.f, 0.f, 0.f, 0.f);
        return;
    }
    const float h = (float)(0.5 * tau);
    const float4 x = xs[i], v = vs[i];
    pk_store(pk_out, i, drift1(x.x, h, v.x), drift1(x.y, h, v.y), drift1(x.z, h, v.z), x.w);
}

// DKD step j (Eqs. 3-5), after the force at x^{n+1/2} (pk_in):
//   v^{n+1} = c v^n + d F;  x^{n+1} = x^{n+1/2} + (tau/2) v^{n+1};  record;
//   next half drift x^{n+3/2} = x^{n+1} + (tau/2) v^{n+1}.
// SYM as in forces_out_f32_kernel.
template <bool COMP, bool SYM>
__global__ void dkd_step_f32_kernel(const float4 *__restrict__ part, ForceLaunch L, int itile,
                                    const float *__restrict__ pk_in, float4 *__restrict__ xs,
                                    float4 *__restrict__ vs, float4 *__restrict__ acc,
                                    float *__restrict__ pk_out, const StepCoef *__restrict__ table,
                                    int tcap, long long step, double tau, long long N, long long N_pad, Tracers tr,
                                    int *flags, DevClock *clk, Extra D) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    if (i >= N) {
        pk_store(pk_out, i, 0.f, 0.f, 0.f, 0.f);
        return;
    }
    const StepCoef &sc = table[step % tcap];
    if (i == 0) advance_clock(clk, sc, flags);
    const float c = (float)sc.c, d = (float)sc.d, h = (float)(0.5 * tau);
    float3 F = SYM ? reduce_sym_f32<COMP, kSymEpiBatch>(part, L, itile, i) : reduce_f32<COMP>(part, L, itile, i);
    const float4 xh = pk_load(pk_in, i);
    defo_force(D, xh.x, xh.y, xh.z, F.x, F.y, F.z);
    add_long_range(D, i, F.x, F.y, F.z);
    const float4 v0 = vs[i];
    const float vx = kick2(c, v0.x, d, F.x), vy = kick2(c, v0.y, d, F.y), vz = kick2(c, v0.z, d, F.z);
    const float x1 = drift1(xh.x, h, vx), y1 = drift1(xh.y, h, vy), z1 = drift1(xh.z, h, vz);
    acc[i] = make_float4(F.x, F.y, F.z, 0.f);
    xs[i] = make_float4(x1, y1, z1, xh.w);
    vs[i] = make_float4(vx, vy, vz, 0.f);
    record(tr, i, sc.step, x1, y1, z1, vx, vy, vz);
    pk_store(pk_out, i, drift1(x1, h, vx), drift1(y1, h, vy), drift1(z1, h, vz), xh.w);
    if (!finite3(x1, y1, z1) || !finite3(vx, vy, vz)) atomicOr(&flags[FLAG_NONFINITE], 1);
}

// --------------------------------------------------------------- FP64 steps
__global__ void kdk_open_f64_kernel(const double4 *__restrict__ xs, const double4 *__restrict__ vs,
                                    const double4 *__restrict__ acc, double4 *__restrict__ vh,
                                    double4 *__restrict__ pos_out,
                                    const StepCoef *__restrict__ table, int tcap, long long step, double tau,
                                    long long N, long long N_pad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    if (i >= N) {
        pos_out[i] = make_double4(0.0, 0.0, 0.0, 0.0);
        return;
    }
    const double c1 = table[step % tcap].c1, d1 = table[step % tcap].d1;
    const double4 x = xs[i], v = vs[i], F = acc[i];
    const double hx = kick2(c1, v.x, d1, F.x), hy = kick2(c1, v.y, d1, F.y), hz = kick2(c1, v.z, d1, F.z);
    vh[i] = make_double4(hx, hy, hz, 0.0);
    pos_out[i] = make_double4(drift1(x.x, tau, hx), drift1(x.y, tau, hy), drift1(x.z, tau, hz), x.w);
}

__global__ void kdk_step_f64_kernel(const double4 *__restrict__ part, ForceLaunch L, int itile,
                                    const double4 *__restrict__ pos_in, double4 *__restrict__ xs,
                                    double4 *__restrict__ vs, double4 *__restrict__ vh,
                                    double4 *__restrict__ acc, double4 *__restrict__ pos_out,
                                    const StepCoef *__restrict__ table, int tcap, long long step, double tau,
                                    long long N, long long N_pad, Tracers tr, int *flags, DevClock *clk, Extra D) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    if (i >= N) {
        pos_out[i] = make_double4(0.0, 0.0, 0.0, 0.0);
        return;
    }
    const StepCoef &sc = table[step % tcap];
    const StepCoef &nc = table[(step + 1) % tcap];
    if (i == 0) advance_clock(clk, sc, flags);
    const double c2 = sc.c2, d2 = sc.d2, c1n = nc.c1, d1n = nc.d1;
    double3 F = reduce_f64(part, L, itile, i);
    const double4 x = pos_in[i];
    defo_force(D, x.x, x.y, x.z, F.x, F.y, F.z);
    add_long_range(D, i, F.x, F.y, F.z);
    const double4 h = vh[i];
    const double vx = kick2(c2, h.x, d2, F.x), vy = kick2(c2, h.y, d2, F.y), vz = kick2(c2, h.z, d2, F.z);
    acc[i] = make_double4(F.x, F.y, F.z, 0.0);
    xs[i] = x;
    vs[i] = make_double4(vx, vy, vz, 0.0);
    record(tr, i, sc.step, x.x, x.y, x.z, vx, vy, vz);
    const double nx = kick2(c1n, vx, d1n, F.x), ny = kick2(c1n, vy, d1n, F.y), nz = kick2(c1n, vz, d1n, F.z);
    vh[i] = make_double4(nx, ny, nz, 0.0);
    pos_out[i] = make_double4(drift1(x.x, tau, nx), drift1(x.y, tau, ny), drift1(x.z, tau, nz), x.w);
    if (!finite3(x.x, x.y, x.z) || !finite3(vx, vy, vz)) atomicOr(&flags[FLAG_NONFINITE], 1);
}

__global__ void dkd_open_f64_kernel(const double4 *__restrict__ xs, const double4 *__restrict__ vs,
                                    double4 *__restrict__ pos_out, double tau, long long N,
                                    long long N_pad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    if (i >= N) {
        pos_out[i] = make_double4(0.0, 0.0, 0.0, 0.0);
        return;
    }
    const double h = 0.5 * tau;
    const double4 x = xs[i], v = vs[i];
    pos_out[i] = make_double4(drift1(x.x, h, v.x), drift1(x.y, h, v.y), drift1(x.z, h, v.z), x.w);
}

__global__ void dkd_step_f64_kernel(const double4 *__restrict__ part, ForceLaunch L, int itile,
                                    const double4 *__restrict__ pos_in, double4 *__restrict__ xs,
                                    double4 *__restrict__ vs, double4 *__restrict__ acc,
                                    double4 *__restrict__ pos_out,
                                    const StepCoef *__restrict__ table, int tcap, long long step, double tau,
                                    long long N, long long N_pad, Tracers tr, int *flags, DevClock *clk, Extra D) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    if (i >= N) {
        pos_out[i] = make_double4(0.0, 0.0, 0.0, 0.0);
        return;
    }
    const StepCoef &sc = table[step % tcap];
    if (i == 0) advance_clock(clk, sc, flags);
    const double c = sc.c, d = sc.d, h = 0.5 * tau;
    double3 F = reduce_f64(part, L, itile, i);
    const double4 xh = pos_in[i];
    defo_force(D, xh.x, xh.y, xh.z, F.x, F.y, F.z);
    add_long_range(D, i, F.x, F.y, F.z);
    const double4 v0 = vs[i];
    const double vx = kick2(c, v0.x, d, F.x), vy = kick2(c, v0.y, d, F.y), vz = kick2(c, v0.z, d, F.z);
    const double x1 = drift1(xh.x, h, vx), y1 = drift1(xh.y, h, vy), z1 = drift1(xh.z, h, vz);
    acc[i] = make_double4(F.x, F.y, F.z, 0.0);
    xs[i] = make_double4(x1, y1, z1, xh.w);
    vs[i] = make_double4(vx, vy, vz, 0.0);
    record(tr, i, sc.step, x1, y1, z1, vx, vy, vz);
    pos_out[i] = make_double4(drift1(x1, h, vx), drift1(y1, h, vy), drift1(z1, h, vz), xh.w);
    if (!finite3(x1, y1, z1) || !finite3(vx, vy, vz)) atomicOr(&flags[FLAG_NONFINITE], 1);
}

}  // namespace colatus
