// common.cuh -- shared device helpers of the COLATUS sm_103a library:
// mbarrier / bulk-copy (TMA) wrappers with bounded waits, the approximate
// reciprocal square root, two-float summation, and the FP64 scalar records.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace colatus {

// Host-side NVTX range over one library call, for profiler timelines and for
// ncu's --nvtx filters (header-only NVTX: a no-op without a tool attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};


// Device error flags (one int each, OR-ed by kernels, read by the host).
enum DevFlag : int { FLAG_NONFINITE = 0, FLAG_FRIEDMANN = 1, FLAG_TIMEOUT = 2, NUM_FLAGS = 4 };

// Cycles a bounded wait may spin before it gives up (about 1-2 s at the
// B300's 1.1-2.0 GHz SM clocks).  A wait that gives up raises FLAG_TIMEOUT
// and the kernel returns instead of hanging.
constexpr long long kWaitCycles = 2000000000LL;

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// Make mbarrier initialisation visible to the asynchronous (bulk-copy) proxy.
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// One-dimensional bulk copy global -> shared, completing on `bar`.
// Both addresses must be 16-byte aligned and `bytes` a multiple of 16.
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                          uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of `bar` to complete, for at most `limit` cycles
// (kWaitCycles, about a second, unless a self-test asks for less).
// Returns false (and leaves the caller to raise FLAG_TIMEOUT) on give-up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  long long limit = kWaitCycles) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

// Approximate 1/sqrt(x) on the SFU (MUFU.RSQ), flushing subnormals.
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The kick a x + b y and the drift x + t v with one fixed rounding sequence.
// The _rn intrinsics are never contracted or reordered by the compiler, so
// every kernel that applies the same kick or drift (a step's epilogue and a
// later call's opening, for one) produces the same bits.
__device__ __forceinline__ float kick2(float a, float x, float b, float y) {
    return __fmaf_rn(b, y, __fmul_rn(a, x));
}
__device__ __forceinline__ double kick2(double a, double x, double b, double y) {
    return __fma_rn(b, y, __dmul_rn(a, x));
}
__device__ __forceinline__ float drift1(float x, float t, float v) { return __fmaf_rn(t, v, x); }
__device__ __forceinline__ double drift1(double x, double t, double v) { return __fma_rn(t, v, x); }

// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// Add b to the two-float (hi, lo) accumulator.
__device__ __forceinline__ void acc2_add(float &hi, float &lo, float b) {
    float s, e;
    two_sum(hi, b, s, e);
    hi = s;
    lo += e;
}

// --------------------------------------------------------- FP64 scalar records
// Per-step scale factors and kick coefficients, written by the Friedmann
// kernel (FP64) and read by the step kernels.  Kick over a span h at scale
// factor a with Hubble rate H (Eq. 4 with tau -> h):
//     v' = c v + d G F,   c = (1 - H h)/(1 + H h),  d = h / (a^3 (1 + H h)).
// The d stored below already includes G.
struct StepCoef {
    double a0, ah, a1;   // a at t^n, t^{n+1/2}, t^{n+1}
    double c, d;         // DKD kick at t^{n+1/2}, span tau
    double c1, d1;       // KDK first half kick at t^n, span tau/2
    double c2, d2;       // KDK second half kick at t^{n+1}, span tau/2
    double t1;           // t^{n+1}
    long long step;      // absolute index n of the step
    int bad;             // Eq. 2 radicand went negative (coefficients are NaN)
    int pad;
};

// Device-resident clock of a context: t, a(t) and the number of steps taken.
struct DevClock {
    double t, a;
    long long step;
    long long pad;
};

struct Cosmo {
    double Omega_R, Omega_M, Omega_K, Omega_L, H0;
};

// O(N) per-body terms the epilogues add to the pair sum (all G-less, like
// the raw force):
//  * the Eq. 6 deformation pull kappa (x_psi - x) / (|x - x_psi|^2 + eps^2)^{3/2}
//    with kappa = C psi / G (a fixed point mass C psi / G at x_psi), when on;
//  * the reciprocal-space part of the periodic (Ewald) force, lr32 / lr64[i],
//    when not null (in the VJP and tangent consumers: that part of the VJP or
//    JVP);
//  * for the equal-mass FP32 VJP (vjp_eqm_f32_kernel): the forces at the VJP's
//    positions, eqf, and 1 / m, whose term -w_i . F_i / m the VJP consumers
//    add to dL/dm_i, when eqf is not null.
struct Extra {
    double kappa, x, y, z, eps2;
    int on, pad;
    const float4 *lr32;
    const double4 *lr64;
    const float4 *eqf;
    float eqminv;
};

__device__ __forceinline__ void defo_force(const Extra &D, double px, double py, double pz, double &fx,
                                           double &fy, double &fz) {
    if (!D.on) return;
    const double dx = D.x - px, dy = D.y - py, dz = D.z - pz;
    const double r2 = dx * dx + dy * dy + dz * dz + D.eps2;
    const double inv = 1.0 / sqrt(r2);
    const double s = D.kappa * inv * inv * inv;
    fx += s * dx;
    fy += s * dy;
    fz += s * dz;
}

// FP32 paths evaluate the O(N) term in FP64 too: x_psi is not float-exact,
// and near x_psi its rounding is amplified by 1/s.
__device__ __forceinline__ void defo_force(const Extra &D, float px, float py, float pz, float &fx,
                                           float &fy, float &fz) {
    if (!D.on) return;
    double gx = 0.0, gy = 0.0, gz = 0.0;
    defo_force(D, (double)px, (double)py, (double)pz, gx, gy, gz);
    fx += (float)gx;
    fy += (float)gy;
    fz += (float)gz;
}

__device__ __forceinline__ void add_long_range(const Extra &E, long long i, float &fx, float &fy,
                                               float &fz) {
    if (!E.lr32) return;
    const float4 l = E.lr32[i];
    fx += l.x;
    fy += l.y;
    fz += l.z;
}

__device__ __forceinline__ void add_long_range(const Extra &E, long long i, double &fx, double &fy,
                                               double &fz) {
    if (!E.lr64) return;
    const double4 l = E.lr64[i];
    fx += l.x;
    fy += l.y;
    fz += l.z;
}

// The equal-mass VJP's per-body term of dL/dm_i: -w_i . F_i / m.
__device__ __forceinline__ void add_eqm_vjp(const Extra &E, long long i, float wx, float wy, float wz,
                                            float4 &g) {
    if (!E.eqf) return;
    const float4 f = E.eqf[i];
    g.w -= E.eqminv * (wx * f.x + wy * f.y + wz * f.z);
}

// Add the reciprocal-space part of a periodic VJP (x, y, z: dL/dx; w:
// dL/dm) of body i, when the VJP consumers are given one in lr32 / lr64.
__device__ __forceinline__ void add_kspace_vjp(const Extra &E, long long i, float4 &g) {
    if (!E.lr32) return;
    const float4 l = E.lr32[i];
    g.x += l.x;
    g.y += l.y;
    g.z += l.z;
    g.w += l.w;
}

__device__ __forceinline__ void add_kspace_vjp(const Extra &E, long long i, double4 &g) {
    if (!E.lr64) return;
    const double4 l = E.lr64[i];
    g.x += l.x;
    g.y += l.y;
    g.z += l.z;
    g.w += l.w;
}

// Derivative of the deformation term along w: -kappa J(d) w, d = x_psi - x,
// J(d) = I/s^3 - 3 d d^T/s^5 (symmetric, so this is also its transpose).
// Evaluated in FP64 for both element types.
template <typename T>
__device__ __forceinline__ void defo_jacobian(const Extra &D, T px, T py, T pz, T wx, T wy, T wz,
                                              T &gx, T &gy, T &gz) {
    if (!D.on) return;
    const double dx = D.x - (double)px, dy = D.y - (double)py, dz = D.z - (double)pz;
    const double r2 = dx * dx + dy * dy + dz * dz + D.eps2;
    const double inv = 1.0 / sqrt(r2);
    const double inv3 = inv * inv * inv, inv5 = inv3 / r2;
    const double dw = dx * (double)wx + dy * (double)wy + dz * (double)wz;
    const double k = D.kappa;
    gx -= (T)(k * ((double)wx * inv3 - 3.0 * dx * dw * inv5));
    gy -= (T)(k * ((double)wy * inv3 - 3.0 * dy * dw * inv5));
    gz -= (T)(k * ((double)wz * inv3 - 3.0 * dz * dw * inv5));
}

}  // namespace colatus
