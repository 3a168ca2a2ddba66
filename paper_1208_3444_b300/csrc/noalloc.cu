// noalloc.cu -- colatus_forces_noalloc: the FP32 all-pairs force for callers
// that cannot allocate device memory.
//
// Some callers must not call cudaMalloc: code that runs inside another
// framework's memory pool or under a fixed device-memory budget, where an
// extra allocation can fail or fragment the pool, and latency-bound loops
// where cudaMalloc's implicit device synchronisation is not acceptable.  This
// entry point runs the same persistent force kernel as colatus_forces but
// keeps every scratch byte it needs (the packed bodies, the force segments and
// the error flags) in one file-scope static device array of fixed size, so it
// allocates nothing.  A GPU holds that array (about 8.6 MiB) from the first
// use of the library's kernels on it until the process exits (with lazy
// module loading, the CUDA default, it is placed on a device when the module
// is first used there).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "colatus.h"
#include "common.cuh"
#include "force.cuh"

using namespace colatus;

namespace {

constexpr long long kNoAllocMaxBodies = 32768;      // largest N accepted
constexpr long long kPkFloat4 = kNoAllocMaxBodies;  // pair-interleaved bodies (16 B each)
constexpr long long kSegFloat4 = 524288;            // 8 MiB of force segments
constexpr long long kFlagFloat4 = 1;                // NUM_FLAGS ints
constexpr long long kScratchFloat4 = kPkFloat4 + kSegFloat4 + kFlagFloat4;
constexpr int kMaxDevices = 64;
// Persistent-grid caps.  A tile is touched by at most ceil(G / n_it) + 1 CTAs,
// so the segments need n_it * S_max <= G + 2 n_it slots of ITILE bodies.  At
// N <= 32768, n_it <= 32 (wide, 1024-body i-tiles) or 128 (narrow, 256), and
// kSegFloat4 holds 512 or 2048 such slots: G <= 448 and G <= 1792 fit on any
// device, whatever its SM count and occupancy.
constexpr long long kWideMaxGrid = 448;
constexpr long long kNarrowMaxGrid = 1792;

// The scratch.  Host code must not use this name as an address: on the host
// it is only a stand-in; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) float4 g_noalloc_scratch[kScratchFloat4];

constexpr int kStagesNA = 4;
// the same two FP32 shapes as colatus_forces uses for general masses
#define NA_WIDE force_f32_kernel<256, 4, 512, kStagesNA, 256, false, false, 2, 2>
#define NA_NARROW force_f32_kernel<128, 2, 64, kStagesNA, 32, false, false, 4, 2>
using WideK = F32Kernel<256, 4, 512, kStagesNA, 256, false, false>;
using NarrowK = F32Kernel<128, 2, 64, kStagesNA, 32, false, false>;

struct DeviceSetup {
    bool done = false;
    float4 *scratch = nullptr;   // device address of g_noalloc_scratch
    int num_sms = 0;
    int occ_wide = 0, occ_narrow = 0;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

// Once per device, with that device current: resolve the scratch's device
// address and the launch limits.  Allocates nothing.
colatus_status setup_device(int dev, DeviceSetup **out) {
    if (dev < 0 || dev >= kMaxDevices) return COLATUS_E_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    DeviceSetup &s = g_setup[dev];
    if (!s.done) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return COLATUS_E_CUDA;
        if (cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return COLATUS_E_CUDA;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s.occ_wide, NA_WIDE, 256, WideK::SMEM) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s.occ_narrow, NA_NARROW, 128,
                                                          NarrowK::SMEM) != cudaSuccess)
            return COLATUS_E_CUDA;
        if (s.occ_wide < 1 || s.occ_narrow < 1) return COLATUS_E_CUDA;
        s.scratch = static_cast<float4 *>(p);
        s.done = true;
    }
    *out = &s;
    return COLATUS_OK;
}

long long round_up_na(long long n, long long m) { return (n + m - 1) / m * m; }

ForceLaunch plan_na(long long n_pad, int itile, int jt, long long g_target, int *s_max) {
    ForceLaunch L{};
    L.n_it = (int)(n_pad / itile);
    L.n_jt = (int)(n_pad / jt);
    L.W = (long long)L.n_it * L.n_jt;
    L.G = (int)(g_target < L.W ? g_target : L.W);
    long long sm = 1;
    for (long long it = 0; it < L.n_it; ++it) {
        const long long a = sk_owner(it * L.n_jt, L.W, L.G);
        const long long b = sk_owner((it + 1) * L.n_jt - 1, L.W, L.G);
        if (b - a + 1 > sm) sm = b - a + 1;
    }
    L.S_max = (int)sm;
    *s_max = (int)sm;
    return L;
}

// (x, y, z, m) per body -> pair-interleaved [x0 x1 y0 y1 z0 z1 m0 m1];
// padding bodies are zero-mass at the origin.
__global__ void na_pack_kernel(const float4 *__restrict__ pos, float *__restrict__ pk, long long N,
                               long long n_pad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    const float4 b = i < N ? pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    float *p = pk + (i >> 1) * 8 + (i & 1);
    p[0] = b.x;
    p[2] = b.y;
    p[4] = b.z;
    p[6] = b.w;
}

// acc_out[3i..3i+2] = scale * (sum of body i's segments, in CTA order)
__global__ void na_out_kernel(const float4 *__restrict__ seg, ForceLaunch L, int itile, long long N,
                              float scale, float *__restrict__ acc_out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const long long it = i / itile, il = i - it * itile;
    const long long g0 = sk_owner(it * L.n_jt, L.W, L.G);
    const long long g1 = sk_owner((it + 1) * L.n_jt - 1, L.W, L.G);
    const float4 *p = seg + it * L.S_max * (long long)itile + il;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (long long s = 0; s <= g1 - g0; ++s) {
        const float4 v = p[s * itile];
        fx += v.x;
        fy += v.y;
        fz += v.z;
    }
    acc_out[3 * i + 0] = scale * fx;
    acc_out[3 * i + 1] = scale * fy;
    acc_out[3 * i + 2] = scale * fz;
}

// A device pointer that the current device can use: device or managed
// memory allocated on that device.
bool on_device(const void *p, int dev) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

long long min_ll(long long a, long long b) { return a < b ? a : b; }

}  // namespace

extern "C" colatus_status colatus_forces_noalloc(const float *pos, int64_t N, double eps, double G,
                                                 double a, float *acc_out, void *cuda_stream) {
    if (!pos || !acc_out) return COLATUS_E_ARG;
    if (N < 1 || N > kNoAllocMaxBodies) return COLATUS_E_ARG;
    if (!(eps > 0.0) || !std::isfinite(eps) || !(a > 0.0) || !std::isfinite(a) || !std::isfinite(G))
        return COLATUS_E_ARG;
    // the pack kernel reads pos as float4
    if ((reinterpret_cast<uintptr_t>(pos) & 15) || (reinterpret_cast<uintptr_t>(acc_out) & 3))
        return COLATUS_E_ARG;
    // a non-sticky error left by an earlier, unrelated call would otherwise be
    // reported as this call's launch failure
    cudaGetLastError();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return COLATUS_E_CUDA;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    // the call synchronises and reads flags back: not allowed inside a capture
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
        cudaGetLastError();
        return COLATUS_E_STATE;
    }
    if (cap != cudaStreamCaptureStatusNone) return COLATUS_E_STATE;
    // every buffer and the stream must belong to the current device
    if (stream) {
        int sdev = -1;
        if (cudaStreamGetDevice(stream, &sdev) != cudaSuccess) {
            cudaGetLastError();
            return COLATUS_E_ARG;
        }
        if (sdev != dev) return COLATUS_E_ARG;
    }
    if (!on_device(pos, dev) || !on_device(acc_out, dev)) return COLATUS_E_ARG;
    DeviceSetup *ds = nullptr;
    colatus_status st = setup_device(dev, &ds);
    if (st != COLATUS_OK) return st;

    // wide tiles when every CTA gets at least four units, narrow otherwise
    int s_max = 0;
    long long n_pad = round_up_na(N, 1024);
    int itile = WideK::ITILE;
    ForceLaunch L = plan_na(n_pad, itile, 512,
                            min_ll((long long)ds->occ_wide * ds->num_sms, kWideMaxGrid), &s_max);
    bool wide = L.W >= 4LL * L.G;
    if (!wide) {
        n_pad = round_up_na(N, 256);
        itile = NarrowK::ITILE;
        L = plan_na(n_pad, itile, 64,
                    min_ll((long long)ds->occ_narrow * ds->num_sms, kNarrowMaxGrid), &s_max);
    }
    if ((long long)L.n_it * s_max * itile > kSegFloat4) return COLATUS_E_ARG;
    if (n_pad > kPkFloat4) return COLATUS_E_ARG;

    float *pk = reinterpret_cast<float *>(ds->scratch);
    float4 *seg = ds->scratch + kPkFloat4;
    int *flags = reinterpret_cast<int *>(ds->scratch + kPkFloat4 + kSegFloat4);
    if (cudaMemsetAsync(flags, 0, NUM_FLAGS * sizeof(int), stream) != cudaSuccess) return COLATUS_E_CUDA;
    na_pack_kernel<<<(unsigned)((n_pad + 255) / 256), 256, 0, stream>>>(
        reinterpret_cast<const float4 *>(pos), pk, N, n_pad);
    if (cudaGetLastError() != cudaSuccess) return COLATUS_E_CUDA;
    const float eps2 = (float)(eps * eps);
    if (wide)
        NA_WIDE<<<L.G, 256, WideK::SMEM, stream>>>(pk, seg, flags, L, eps2, 1.f);
    else
        NA_NARROW<<<L.G, 128, NarrowK::SMEM, stream>>>(pk, seg, flags, L, eps2, 1.f);
    if (cudaGetLastError() != cudaSuccess) return COLATUS_E_CUDA;
    const float scale = (float)(G / (a * a * a));
    na_out_kernel<<<(unsigned)((N + 255) / 256), 256, 0, stream>>>(seg, L, itile, N, scale, acc_out);
    if (cudaGetLastError() != cudaSuccess) return COLATUS_E_CUDA;
    int f[NUM_FLAGS];
    if (cudaMemcpyAsync(f, flags, sizeof(f), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return COLATUS_E_CUDA;
    if (f[FLAG_TIMEOUT]) return COLATUS_E_TIMEOUT;
    return COLATUS_OK;
}
