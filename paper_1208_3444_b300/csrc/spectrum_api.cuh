// spectrum_api.cuh -- host side of the tracer velocity energy spectrum
// (colatus_velocity_spectrum, colatus_tracer_spectrum), included by colatus.cu
// after its helpers.
#pragma once

namespace {

constexpr long long kSpecMaxT = 1LL << 24;   // gridDim.y = ceil((T/2+1)/256) <= 65535

colatus_status spec_check(colatus_t ctx, long long T, long long ntr, double dt, int window) {
    if (T < 2 || T > kSpecMaxT) return fail(ctx, COLATUS_E_ARG, "T must be in [2, 2^24]");
    if (ntr < 1 || ntr > 0x7fffffffLL) return fail(ctx, COLATUS_E_ARG, "ntr must be in [1, 2^31)");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, COLATUS_E_ARG, "dt must be > 0");
    if (window != 0 && window != 1) return fail(ctx, COLATUS_E_ARG, "window must be 0 or 1");
    return COLATUS_OK;
}

// FFT stages for T: radix 4 while it divides, then 2, then the odd primes in
// increasing order.  False if T is too long for shared memory or has a prime
// factor above kSpecFftMaxP (the direct sum is taken then).
bool spec_plan(long long T, SpecPlan &plan) {
    plan.nst = 0;
    if (T > kSpecFftMaxT) return false;
    long long n = T;
    auto take = [&](int p) {
        while (n % p == 0 && plan.nst < kSpecFftMaxStages) {
            plan.p[plan.nst++] = p;
            n /= p;
        }
    };
    take(4);
    take(2);
    for (int p = 3; p <= kSpecFftMaxP && n > 1; p += 2) take(p);
    return n == 1;
}

// Twiddles into tw (T double2), then E (device, ntr x (T/2+1) doubles).
colatus_status spec_launch(colatus_t ctx, const SpecSeries &S, double2 *tw, double dt, int window,
                           int detrend, double *E, cudaStream_t stream) {
    spectrum_twiddle_kernel<<<blocks_for(S.T, 256), 256, 0, stream>>>(tw, S.T);
    CU(cudaGetLastError());
    SpecPlan plan;
    if (spec_plan(S.T, plan)) {
        const size_t smem = 2 * (size_t)S.T * sizeof(double2);
        CU(cudaFuncSetAttribute(spectrum_fft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
        const dim3 grid((unsigned)S.ntr, 2);
        spectrum_fft_kernel<<<grid, kSpecThreads, smem, stream>>>(S, tw, plan, dt, window,
                                                                  detrend ? 1 : 0, E);
    } else {
        const long long nf = S.T / 2 + 1;
        const dim3 grid((unsigned)S.ntr, blocks_for(nf, kSpecThreads));
        spectrum_kernel<<<grid, kSpecThreads, 0, stream>>>(S, tw, dt, window, detrend ? 1 : 0, E);
    }
    CU(cudaGetLastError());
    if (ctx) ctx->launches += 2;
    return COLATUS_OK;
}

}  // namespace

colatus_status colatus_velocity_spectrum(const void *v, int dtype, int on_device, int64_t T,
                                         int64_t ntr, int64_t stride, double dt, int window,
                                         int detrend, double *E_out, int out_on_device,
                                         void *cuda_stream) {
    colatus_t ctx = nullptr;   // errors go to colatus_last_error(NULL)
    if (!v || !E_out) return fail(ctx, COLATUS_E_ARG, "v and E_out must not be NULL");
    if (dtype != COLATUS_F32 && dtype != COLATUS_F64) return fail(ctx, COLATUS_E_ARG, "bad dtype");
    if (stride < 3) return fail(ctx, COLATUS_E_ARG, "stride must be >= 3");
    TRY(spec_check(ctx, T, ntr, dt, window));
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    const size_t esz = dtype == COLATUS_F64 ? 8 : 4;
    const size_t in_bytes = (size_t)T * ntr * stride * esz;
    const long long nf = T / 2 + 1;
    const size_t out_bytes = (size_t)ntr * nf * sizeof(double);
    // one scratch block: [twiddles | E (unless the caller's is on the device) | input copy]
    size_t bytes = (size_t)T * sizeof(double2);
    const size_t off_E = bytes;
    if (!out_on_device) bytes += out_bytes;
    const size_t off_in = (bytes + 255) / 256 * 256;
    if (!on_device) bytes = off_in + in_bytes;
    char *scratch = nullptr;
    CU(cudaMallocAsync(reinterpret_cast<void **>(&scratch), bytes, stream));
    double *dE = out_on_device ? E_out : reinterpret_cast<double *>(scratch + off_E);
    const void *dv = v;
    colatus_status st = COLATUS_OK;
    if (!on_device) {
        cudaError_t e = cudaMemcpyAsync(scratch + off_in, v, in_bytes, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) st = fail(ctx, COLATUS_E_CUDA, "input copy: %s", cudaGetErrorString(e));
        dv = scratch + off_in;
    }
    if (st == COLATUS_OK) {
        SpecSeries S{dv, T, ntr, ntr * stride, stride, 0, T, dtype == COLATUS_F64 ? 1 : 0};
        st = spec_launch(ctx, S, reinterpret_cast<double2 *>(scratch), dt, window, detrend, dE, stream);
    }
    if (st == COLATUS_OK && !out_on_device) {
        cudaError_t e = cudaMemcpyAsync(E_out, dE, out_bytes, cudaMemcpyDeviceToHost, stream);
        if (e != cudaSuccess) st = fail(ctx, COLATUS_E_CUDA, "output copy: %s", cudaGetErrorString(e));
    }
    cudaFreeAsync(scratch, stream);
    if (st == COLATUS_OK && (!out_on_device || !on_device)) CU(cudaStreamSynchronize(stream));
    return st;
}

colatus_status colatus_tracer_spectrum(colatus_t ctx, double dt, int window, int detrend,
                                       double *E_out, int64_t *nrec_out) {
    NvtxRange nvtx_("colatus_tracer_spectrum");
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    if (!nrec_out) return fail(ctx, COLATUS_E_ARG, "nrec_out is NULL");
    TRY(sync_and_check(ctx));
    const long long total = ctx->host_step - ctx->rec_base;
    const long long nrec = ctx->ntr > 0 ? std::min(total, ctx->rec_cap) : 0;
    *nrec_out = nrec;
    if (!E_out) return COLATUS_OK;
    if (ctx->ntr == 0) return fail(ctx, COLATUS_E_STATE, "no tracers are being recorded");
    TRY(spec_check(ctx, nrec, ctx->ntr, dt, window));
    const long long nf = nrec / 2 + 1;
    const size_t out_bytes = (size_t)ctx->ntr * nf * sizeof(double);
    const size_t tw_bytes = (size_t)nrec * sizeof(double2);
    char *scratch = nullptr;
    CU(cudaMallocAsync(reinterpret_cast<void **>(&scratch), tw_bytes + out_bytes, ctx->stream));
    // ring rows hold (x, y, z, vx, vy, vz) per tracer; the oldest kept record first
    SpecSeries S{ctx->rec + 3, nrec, ctx->ntr, (long long)ctx->ntr * 6, 6,
                 (total - nrec) % ctx->rec_cap, ctx->rec_cap, 0};
    double *dE = reinterpret_cast<double *>(scratch + tw_bytes);
    colatus_status st = spec_launch(ctx, S, reinterpret_cast<double2 *>(scratch), dt, window, detrend,
                                    dE, ctx->stream);
    if (st == COLATUS_OK) {
        cudaError_t e = cudaMemcpyAsync(E_out, dE, out_bytes, cudaMemcpyDeviceToHost, ctx->stream);
        if (e != cudaSuccess) st = fail(ctx, COLATUS_E_CUDA, "output copy: %s", cudaGetErrorString(e));
    }
    cudaFreeAsync(scratch, ctx->stream);
    if (st == COLATUS_OK) CU(cudaStreamSynchronize(ctx->stream));
    return st;
}
