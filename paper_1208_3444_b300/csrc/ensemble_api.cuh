// ensemble_api.cuh -- host side of the batched ensemble (colatus_ensemble_*),
// included by colatus.cu after its helpers.
//
// Layout: realisation r's bodies are stored contiguously from body_off[r],
// padded with zero-mass bodies to a multiple of the 256-body tile; users pass
// and receive dense concatenated arrays (realisation r from user_off[r]).
// A step is one persistent force launch over all realisations plus one fused
// kick/drift epilogue; colatus_ensemble_step replays a captured CUDA graph of
// 16 such steps (with their FP64 schedule kernel) per launch.
#pragma once

namespace {

// 256-body i- and j-tiles.  Of six CTA shapes timed on the 64-realisation
// ensemble, 128 threads x 2 i-bodies (4 CTAs per SM) was the fastest with
// every 1/s^2 from the FMA pipe (3.75 ms per force); 64 x 4 (8 CTAs per SM)
// with one of its four i-bodies taking 1/s^2 from the MUFU pipe is faster
// still (3.69 ms) and is the built-in shape.
constexpr int kEnsJT = 256, kEnsFold = 128;
using EnsK = F32Kernel<128, 2, kEnsJT, kStages, kEnsFold, false, false>;   // SMEM: every shape's
constexpr int kEnsTile = EnsK::ITILE;   // 256 bodies: the per-realisation padding unit
constexpr int kEnsChunk = 16;           // steps per captured graph (even: ping-pong parity)
static_assert(kEnsTile == kEnsJT, "ensemble tiles pad realisations to one size");

// CTA shapes of the ensemble force kernel (threads x i-bodies per thread,
// CTAs per SM): 0-2 with 256-body i- and j-tiles, so that the padding and the
// unit list do not depend on the shape; 3 evaluates every pair once on
// 512-body tiles of each realisation (ens_sym.cuh, its own work list over the
// same storage).  The built-in choice is shape 3 where it fits (26 % faster
// than shape 2 on the 64-realisation ensemble: 2.72 against 3.69 ms per
// force), else kEnsDefault; colatus_ensemble_autotune times all of them on
// the ensemble at hand.
constexpr int kEnsShapes = 4, kEnsDefault = 2, kEnsSymShape = 3;
constexpr int kEnsSymNT = 128, kEnsSymMinB = 4, kEnsSymUnr = 8;
using EnsSymK = EnsSymKernel<kEnsSymNT>;
struct EnsVariant {
    int nt;
    const void *fn[2];   // general masses, equal masses
    void (*launch[2])(int grid, cudaStream_t, const float *, float4 *, int *, EnsLaunch);
    int smem;
};

template <int NT, int IPT, int MINB, int NRCP, bool EQM>
void ens_launch(int grid, cudaStream_t st, const float *pk, float4 *part, int *flags, EnsLaunch E) {
    static_assert(NT * IPT == kEnsTile, "one i-tile per CTA pass");
    ens_force_kernel<NT, IPT, kEnsJT, kStages, kEnsFold, MINB, EQM, NRCP><<<grid, NT, EnsK::SMEM, st>>>(
        pk, part, flags, E);
}

// NRCP: as for the single-system kernels, 1/s^2 of the first NRCP i-bodies of
// a thread from an rcp on the MUFU pipe instead of a square on the FMA pipe
template <int NT, int IPT, int MINB, int NRCP = 0>
EnsVariant make_ens() {
    return EnsVariant{NT,
                      {(const void *)ens_force_kernel<NT, IPT, kEnsJT, kStages, kEnsFold, MINB, false, NRCP>,
                       (const void *)ens_force_kernel<NT, IPT, kEnsJT, kStages, kEnsFold, MINB, true, NRCP>},
                      {&ens_launch<NT, IPT, MINB, NRCP, false>, &ens_launch<NT, IPT, MINB, NRCP, true>},
                      EnsK::SMEM};
}

template <bool EQM>
void ens_sym_launch(int grid, cudaStream_t st, const float *pk, float4 *part, int *flags, EnsLaunch E) {
    ens_sym_force_kernel<kEnsSymNT, kEnsSymMinB, EQM, kEnsSymUnr><<<grid, kEnsSymNT, EnsSymK::SMEM, st>>>(pk, part, flags, E);
}

// 64 x 4 takes one rcp per four i-bodies: 3.69 ms per force on the
// 64-realisation ensemble against 3.80 without it (and 3.75 for 128 x 2)
const EnsVariant &ens_variant(int s) {
    static const EnsVariant table[kEnsShapes] = {
        make_ens<128, 2, 4>(), make_ens<256, 1, 4>(), make_ens<64, 4, 8, 1>(),
        EnsVariant{kEnsSymNT,
                   {(const void *)ens_sym_force_kernel<kEnsSymNT, kEnsSymMinB, false, kEnsSymUnr>,
                    (const void *)ens_sym_force_kernel<kEnsSymNT, kEnsSymMinB, true, kEnsSymUnr>},
                   {&ens_sym_launch<false>, &ens_sym_launch<true>},
                   EnsSymK::SMEM}};
    return table[s];
}

}  // namespace

struct colatus_ensemble {
    int device = 0, num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int R = 0;
    long long Ntot = 0, Npad = 0;
    double G = 1.0, pairs = 0.0;
    Cosmo cosmo{};
    std::vector<long long> nbody, body_off, user_off, unit_off, tile_u0;
    std::vector<int> n_jt, tile_r;
    EnsLaunch E{};
    int shape = kEnsDefault;               // CTA shape of the force kernel (ens_variant)
    colatus_scheme scheme = COLATUS_KDK;   // colatus_ensemble_set_scheme
    int shape_G[kEnsShapes] = {0}, shape_S[kEnsShapes] = {0};   // grid and S_max per shape (0: unusable)
    int *sym_tab = nullptr;                // tables of the pair-once shape
    long long sym_col_off = 0;
    void *meta = nullptr;                  // device descriptor arrays
    long long *d_user_off = nullptr;
    float4 *xs = nullptr, *vs = nullptr, *vh = nullptr, *acc = nullptr;
    float *pk[3] = {nullptr, nullptr, nullptr};
    float4 *part = nullptr;
    int *flags = nullptr;
    DevClock *clk = nullptr;
    StepCoef *table = nullptr;             // kEnsChunk entries
    double *stage = nullptr, *stage2 = nullptr;
    bool have_state = false, spec_valid = false;
    double spec_tau = 0.0;
    int cur = 0;
    long long host_step = 0, launches = 0;
    double interactions = 0.0;
    bool profiling = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};   // per ping-pong parity
    double graph_tau[2] = {0.0, 0.0};
    // tracer records (colatus_ensemble_record_tracers): slot per padded body
    int *tslot = nullptr;
    float *rec = nullptr;
    long long rec_cap = 0, rec_base = 0;
    int ntr = 0;
    char err[512] = {0};
};

namespace {

colatus_status efail(colatus_ens_t e, colatus_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(e ? e->err : g_init_err, 512, fmt, ap);
    va_end(ap);
    return st;
}

#define ECU(call)                                                                             \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return efail(e, e_ == cudaErrorMemoryAllocation ? COLATUS_E_OOM : COLATUS_E_CUDA, \
                         "%s: %s", #call, cudaGetErrorString(e_));                            \
    } while (0)

colatus_status elaunched(colatus_ens_t e) {
    ++e->launches;
    cudaError_t r = cudaGetLastError();
    if (r != cudaSuccess) return efail(e, COLATUS_E_CUDA, "kernel launch: %s", cudaGetErrorString(r));
    return COLATUS_OK;
}

// ---- user (dense) <-> padded layout
__global__ void ens_masses_kernel(const double *m, const long long *user_off, EnsLaunch E,
                                  long long Npad, float4 *xs, int *bad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= Npad) return;
    const int r = E.tile_r[i / kEnsTile];
    const long long k = i - E.body_off[r];
    if (k >= E.nbody[r]) {
        xs[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const double mi = m[user_off[r] + k];
    if (!isfinite(mi) || mi < 0.0) atomicOr(bad, 1);
    xs[i] = make_float4(0.f, 0.f, 0.f, (float)mi);
}

__global__ void ens_load_kernel(const void *x, const void *v, int f64, const long long *user_off,
                                EnsLaunch E, long long Npad, float4 *xs, float4 *vs, int *bad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= Npad) return;
    const int r = E.tile_r[i / kEnsTile];
    const long long k = i - E.body_off[r];
    if (k >= E.nbody[r]) {
        vs[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const long long u = user_off[r] + k;
    double p[3], q[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < 3; ++c) {
        p[c] = f64 ? static_cast<const double *>(x)[3 * u + c] : static_cast<const float *>(x)[3 * u + c];
        if (v)
            q[c] = f64 ? static_cast<const double *>(v)[3 * u + c]
                       : static_cast<const float *>(v)[3 * u + c];
        if (!isfinite(p[c]) || !isfinite(q[c])) atomicOr(bad, 1);
    }
    xs[i] = make_float4((float)p[0], (float)p[1], (float)p[2], xs[i].w);
    vs[i] = make_float4((float)q[0], (float)q[1], (float)q[2], 0.f);
}

// Real bodies of a (and b) into user arrays; `scale` from the clock (G a^-3)
// when use_clock, else 1.
__global__ void ens_store_kernel(const float4 *a, const float4 *b, const long long *user_off,
                                 EnsLaunch E, long long Npad, void *oa, void *ob, int f64,
                                 const DevClock *clk, double G, int use_clock) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= Npad) return;
    const int r = E.tile_r[i / kEnsTile];
    const long long k = i - E.body_off[r];
    if (k >= E.nbody[r]) return;
    const long long u = user_off[r] + k;
    double s = 1.0;
    if (use_clock) {
        const double aa = clk->a;
        s = G / (aa * aa * aa);
    }
    const float4 pa = a[i];
    const float ca[3] = {pa.x, pa.y, pa.z};
    for (int c = 0; c < 3; ++c) {
        if (f64)
            static_cast<double *>(oa)[3 * u + c] = use_clock ? s * ca[c] : (double)ca[c];
        else
            static_cast<float *>(oa)[3 * u + c] = use_clock ? (float)(s * ca[c]) : ca[c];
    }
    if (b && ob) {
        const float4 pb = b[i];
        const float cb[3] = {pb.x, pb.y, pb.z};
        for (int c = 0; c < 3; ++c) {
            if (f64)
                static_cast<double *>(ob)[3 * u + c] = cb[c];
            else
                static_cast<float *>(ob)[3 * u + c] = cb[c];
        }
    }
}

colatus_status ens_force(colatus_ens_t e, const float *pk) {
    if (e->profiling) {
        while (e->ev.size() < e->ev_used + 2) {
            cudaEvent_t v;
            ECU(cudaEventCreate(&v));
            e->ev.push_back(v);
        }
        ECU(cudaEventRecord(e->ev[e->ev_used], e->stream));
    }
    ens_variant(e->shape).launch[e->E.meq ? 1 : 0](e->E.G, e->stream, pk, e->part, e->flags, e->E);
    colatus_status st = elaunched(e);
    if (st != COLATUS_OK) return st;
    e->interactions += e->pairs;
    if (e->profiling) {
        ECU(cudaEventRecord(e->ev[e->ev_used + 1], e->stream));
        e->ev_used += 2;
    }
    return COLATUS_OK;
}

unsigned ens_blocks(colatus_ens_t e) { return (unsigned)((e->Npad + 255) / 256); }

colatus_status ens_force_at_state(colatus_ens_t e) {
    ens_pack_kernel<<<ens_blocks(e), 256, 0, e->stream>>>(e->xs, e->pk[2], e->E, kEnsTile, e->Npad);
    colatus_status st = elaunched(e);
    if (st != COLATUS_OK) return st;
    if ((st = ens_force(e, e->pk[2])) != COLATUS_OK) return st;
    ens_forces_out_kernel<<<ens_blocks(e), 256, 0, e->stream>>>(e->part, e->E, kEnsTile, e->Npad,
                                                               e->acc);
    return elaunched(e);
}

// n <= kEnsChunk steps: their schedule, then force + epilogue per step.
colatus_status ens_steps(colatus_ens_t e, double tau, int n) {
    const int canon = e->scheme == COLATUS_KDK_CANONICAL ? 1 : 0;
    // the canonical closing kick needs the next step's opening coefficients
    ens_table_kernel<<<1, 1, 0, e->stream>>>(e->cosmo, e->clk, e->table, n + canon, tau, e->G,
                                             kFriedmannSub, canon);
    colatus_status st = elaunched(e);
    if (st != COLATUS_OK) return st;
    const Tracers tr{e->tslot, e->rec, e->rec_cap, e->rec_base, e->ntr};
    for (int j = 0; j < n; ++j) {
        const int c = e->cur, nx = c ^ 1;
        if ((st = ens_force(e, e->pk[c])) != COLATUS_OK) return st;
        if (e->scheme == COLATUS_DKD)
            ens_dkd_step_kernel<<<ens_blocks(e), 256, 0, e->stream>>>(
                e->part, e->E, kEnsTile, e->pk[c], e->xs, e->vs, e->acc, e->pk[nx], e->table, j, tau,
                e->Npad, e->flags, e->clk, tr);
        else
            ens_step_kernel<<<ens_blocks(e), 256, 0, e->stream>>>(
                e->part, e->E, kEnsTile, e->pk[c], e->xs, e->vs, e->vh, e->acc, e->pk[nx], e->table, j, tau,
                e->Npad, e->flags, e->clk, tr, canon);
        if ((st = elaunched(e)) != COLATUS_OK) return st;
        e->cur = nx;
    }
    return COLATUS_OK;
}

colatus_status ens_capture(colatus_ens_t e, double tau) {
    const int p = e->cur;
    if (e->graph[p]) {
        cudaGraphExecDestroy(e->graph[p]);
        e->graph[p] = nullptr;
    }
    const bool prof = e->profiling;
    e->profiling = false;   // no event records inside the graph
    const long long l0 = e->launches;
    const double i0 = e->interactions;
    ECU(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
    colatus_status st = ens_steps(e, tau, kEnsChunk);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
    e->profiling = prof;
    e->launches = l0;
    e->interactions = i0;
    e->cur = p;             // 16 steps return the ping-pong to its parity
    if (st != COLATUS_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (ce != cudaSuccess) return efail(e, COLATUS_E_CUDA, "graph capture: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&e->graph[p], g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return efail(e, COLATUS_E_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
    e->graph_tau[p] = tau;
    return COLATUS_OK;
}

void ens_free(colatus_ens_t e) {
    for (cudaGraphExec_t &g : e->graph)
        if (g) cudaGraphExecDestroy(g);
    for (cudaEvent_t v : e->ev) cudaEventDestroy(v);
    void *ptrs[] = {e->meta, e->xs, e->vs, e->vh, e->acc, e->pk[0], e->pk[1], e->pk[2],
                    e->part, e->flags, e->clk, e->table, e->stage, e->stage2, e->tslot, e->rec,
                    e->sym_tab};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
}

// The built-in shape: every pair once where it fits.
int ens_default_shape(colatus_ens_t e) { return e->shape_G[kEnsSymShape] > 0 ? kEnsSymShape : kEnsDefault; }

// The launch geometry and segment layout of CTA shape sh.
void ens_apply_shape(colatus_ens_t e, int sh) {
    e->shape = sh;
    e->E.G = e->shape_G[sh];
    e->E.S_max = e->shape_S[sh];
    e->E.sym = sh == kEnsSymShape ? e->sym_tab : nullptr;
    e->E.sym_col_off = sh == kEnsSymShape ? e->sym_col_off : 0;
}

// Use CTA shape sh from now on: its grid and segment layout, new graphs, and
// a new opening force (the old one was summed in the other shape's order).
void ens_set_shape(colatus_ens_t e, int sh) {
    ens_apply_shape(e, sh);
    for (cudaGraphExec_t &g : e->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    e->spec_valid = false;
}

colatus_status ens_check(colatus_ens_t e, bool clear) {
    int f[NUM_FLAGS];
    ECU(cudaStreamSynchronize(e->stream));
    ECU(cudaMemcpy(f, e->flags, sizeof(f), cudaMemcpyDeviceToHost));
    if (clear) ECU(cudaMemset(e->flags, 0, sizeof(f)));
    if (f[FLAG_TIMEOUT]) return efail(e, COLATUS_E_TIMEOUT, "a bounded device wait gave up");
    if (f[FLAG_FRIEDMANN]) return efail(e, COLATUS_E_FRIEDMANN, "H^2 < 0 while integrating Eq. 2");
    if (f[FLAG_NONFINITE]) return efail(e, COLATUS_E_NONFINITE, "non-finite position or velocity");
    return COLATUS_OK;
}

}  // namespace

extern "C" {

colatus_status colatus_ensemble_init(colatus_ens_t *out, int R, const int64_t *N_r,
                                     const double *masses, const double *eps_r, double Omega_R,
                                     double Omega_M, double Omega_K, double Omega_L, double H0,
                                     double a_start, double G, void *cuda_stream) {
    colatus_ens_t e = nullptr;
    if (!out) return efail(nullptr, COLATUS_E_ARG, "out is NULL");
    *out = nullptr;
    if (R < 1 || !N_r || !masses || !eps_r) return efail(nullptr, COLATUS_E_ARG, "bad arguments");
    if (!(a_start > 0.0) || !std::isfinite(G)) return efail(nullptr, COLATUS_E_ARG, "bad a_start or G");
    const double e2 = Omega_R / std::pow(a_start, 4) + Omega_M / std::pow(a_start, 3) +
                      Omega_K / (a_start * a_start) + Omega_L;
    if (!(e2 >= 0.0)) return efail(nullptr, COLATUS_E_ARG, "H^2(a_start) < 0");
    for (int r = 0; r < R; ++r)
        if (N_r[r] < 1 || !(eps_r[r] > 0.0) || !std::isfinite(eps_r[r]))
            return efail(nullptr, COLATUS_E_ARG, "realisation %d: N >= 1 and eps > 0 needed", r);
    e = new (std::nothrow) colatus_ensemble();
    if (!e) return efail(nullptr, COLATUS_E_OOM, "host allocation failed");
    auto bail = [&](colatus_status st) {
        snprintf(g_init_err, sizeof(g_init_err), "%s", e->err);
        ens_free(e);
        delete e;
        return st;
    };
    if (cudaGetDevice(&e->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&e->num_sms, cudaDevAttrMultiProcessorCount, e->device) != cudaSuccess)
        return bail(efail(e, COLATUS_E_CUDA, "no CUDA device"));
    e->R = R;
    e->G = G;
    e->cosmo = Cosmo{Omega_R, Omega_M, Omega_K, Omega_L, H0};
    // descriptors
    e->nbody.assign(N_r, N_r + R);
    e->body_off.assign(R + 1, 0);
    e->user_off.assign(R + 1, 0);
    e->unit_off.assign(R + 1, 0);
    e->n_jt.assign(R, 0);
    for (int r = 0; r < R; ++r) {
        const long long np = round_up(N_r[r], kEnsTile);
        const long long nt = np / kEnsTile;
        e->n_jt[r] = (int)nt;
        for (long long t = 0; t < nt; ++t) {
            e->tile_r.push_back(r);
            e->tile_u0.push_back(e->unit_off[r] + t * nt);
        }
        e->body_off[r + 1] = e->body_off[r] + np;
        e->user_off[r + 1] = e->user_off[r] + N_r[r];
        e->unit_off[r + 1] = e->unit_off[r] + nt * nt;
        e->pairs += (double)N_r[r] * (double)N_r[r];
    }
    e->Ntot = e->user_off[R];
    e->Npad = e->body_off[R];
    const int T = (int)e->tile_r.size();
    // equal masses within every realisation (as floats): the equal-mass kernel
    std::vector<float> meq(R, 0.f);
    bool eqm = true;
    for (int r = 0; r < R && eqm; ++r) {
        meq[r] = (float)masses[e->user_off[r]];
        for (long long k = 1; k < N_r[r] && eqm; ++k) eqm = (float)masses[e->user_off[r] + k] == meq[r];
    }
    EnsLaunch &E = e->E;
    E.W = e->unit_off[R];
    E.R = R;
    E.T = T;
    // grid and segment count of every shape; part is sized for the largest
    long long smax = 1;
    size_t part_bytes = 0;
    EnsSymTables sym;
    for (int sh = 0; sh < kEnsShapes; ++sh) {
        const EnsVariant &v = ens_variant(sh);
        int occ = 0, occ2 = 0;
        if (v.smem > 48 * 1024 &&
            (cudaFuncSetAttribute(v.fn[0], cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem) != cudaSuccess ||
             cudaFuncSetAttribute(v.fn[1], cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem) != cudaSuccess))
            return bail(efail(e, COLATUS_E_CUDA, "ensemble force kernel (shape %d): shared memory", sh));
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, v.fn[0], v.nt, v.smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, v.fn[1], v.nt, v.smem) != cudaSuccess ||
            std::min(occ, occ2) < 1)
            return bail(efail(e, COLATUS_E_CUDA, "ensemble force kernel (shape %d) cannot be resident", sh));
        if (sh == kEnsSymShape) {
            // every pair once: the tile pairs of 512-body tiles per realisation,
            // phases split by the cost of the kernel's form (lane-ops per
            // diagonal interaction and per symmetric pair); not usable if its
            // partial sums would take more than an eighth of the device memory
            std::vector<int> nt_r(R);
            for (int r = 0; r < R; ++r)
                nt_r[r] = (int)((e->body_off[r + 1] - e->body_off[r] + kEnsSymT - 1) / kEnsSymT);
            sym = build_ens_sym_tables(nt_r, EnsSymK::NW, (long long)std::min(occ, occ2) * e->num_sms,
                                       eqm ? 11 : 12, eqm ? 14 : 16);
            const size_t b = (size_t)((long long)sym.TT * sym.S_row + sym.slots) * kEnsSymT * sizeof(float4);
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess)
                return bail(efail(e, COLATUS_E_CUDA, "cudaMemGetInfo failed"));
            if (b <= total_b / 8) {
                e->shape_G[sh] = sym.G;
                e->shape_S[sh] = sym.S_row;
                e->sym_col_off = (long long)sym.TT * sym.S_row * kEnsSymT;
                part_bytes = std::max(part_bytes, b);
            }
            continue;
        }
        const long long G = std::min<long long>((long long)std::min(occ, occ2) * e->num_sms, E.W);
        long long sm = 1;
        for (int t = 0; t < T; ++t) {
            const long long g0 = sk_owner(e->tile_u0[t], E.W, G);
            const long long g1 = sk_owner(e->tile_u0[t] + e->n_jt[e->tile_r[t]] - 1, E.W, G);
            sm = std::max(sm, g1 - g0 + 1);
        }
        e->shape_G[sh] = (int)G;
        e->shape_S[sh] = (int)sm;
        smax = std::max(smax, sm);
    }
    part_bytes = std::max(part_bytes, (size_t)((long long)T * smax * kEnsTile) * sizeof(float4));
    E.G = e->shape_G[kEnsDefault];
    E.S_max = e->shape_S[kEnsDefault];
    // device memory
    const size_t ll = sizeof(long long);
    const size_t meta_bytes = ll * ((R + 1) * 3 + R + T) + sizeof(int) * (R + T) + sizeof(float) * 2 * R + 72;
    auto A = [&](void **p, size_t b) -> bool { return cudaMalloc(p, b) == cudaSuccess; };
    const size_t np = (size_t)e->Npad;
    bool ok = A(&e->meta, meta_bytes) && A((void **)&e->xs, np * 16) && A((void **)&e->vs, np * 16) &&
              A((void **)&e->vh, np * 16) && A((void **)&e->acc, np * 16) &&
              A((void **)&e->pk[0], np * 16) && A((void **)&e->pk[1], np * 16) &&
              A((void **)&e->pk[2], np * 16) &&
              A((void **)&e->part, part_bytes) &&
              A((void **)&e->flags, NUM_FLAGS * sizeof(int)) && A((void **)&e->clk, sizeof(DevClock)) &&
              A((void **)&e->table, (kEnsChunk + 1) * sizeof(StepCoef)) &&
              A((void **)&e->stage, (size_t)e->Ntot * 3 * sizeof(double)) &&
              A((void **)&e->stage2, (size_t)e->Ntot * 3 * sizeof(double));
    if (!ok) return bail(efail(e, COLATUS_E_OOM, "device allocation failed"));
    if (cuda_stream) {
        e->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(efail(e, COLATUS_E_CUDA, "stream creation failed"));
        e->own_stream = true;
    }
    // descriptor upload (one host block mirroring the device carve-up)
    std::vector<char> hm(meta_bytes, 0);
    char *base = static_cast<char *>(e->meta);
    size_t off = 0;
    auto put = [&](const void *src, size_t bytes) -> char * {
        std::memcpy(hm.data() + off, src, bytes);
        char *d = base + off;
        off += (bytes + 7) & ~size_t(7);
        return d;
    };
    std::vector<float> eps2(R);
    for (int r = 0; r < R; ++r) eps2[r] = (float)(eps_r[r] * eps_r[r]);
    E.unit_off = reinterpret_cast<const long long *>(put(e->unit_off.data(), ll * (R + 1)));
    E.body_off = reinterpret_cast<const long long *>(put(e->body_off.data(), ll * (R + 1)));
    e->d_user_off = reinterpret_cast<long long *>(put(e->user_off.data(), ll * (R + 1)));
    E.nbody = reinterpret_cast<const long long *>(put(e->nbody.data(), ll * R));
    E.tile_u0 = reinterpret_cast<const long long *>(put(e->tile_u0.data(), ll * T));
    E.n_jt = reinterpret_cast<const int *>(put(e->n_jt.data(), sizeof(int) * R));
    E.tile_r = reinterpret_cast<const int *>(put(e->tile_r.data(), sizeof(int) * T));
    E.eps2 = reinterpret_cast<const float *>(put(eps2.data(), sizeof(float) * R));
    E.meq = eqm ? reinterpret_cast<const float *>(put(meq.data(), sizeof(float) * R)) : nullptr;
    colatus_status st = COLATUS_OK;
    cudaError_t ce = cudaMemcpy(e->meta, hm.data(), meta_bytes, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess && e->shape_G[kEnsSymShape] > 0) {
        ce = cudaMalloc((void **)&e->sym_tab, sym.tab.size() * sizeof(int));
        if (ce == cudaSuccess)
            ce = cudaMemcpy(e->sym_tab, sym.tab.data(), sym.tab.size() * sizeof(int), cudaMemcpyHostToDevice);
    }
    if (ce == cudaSuccess) ens_apply_shape(e, ens_default_shape(e));
    DevClock clk{0.0, a_start, 0, 0};
    if (ce == cudaSuccess) ce = cudaMemcpy(e->clk, &clk, sizeof(clk), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemset(e->flags, 0, NUM_FLAGS * sizeof(int));
    for (float *p : e->pk)
        if (ce == cudaSuccess) ce = cudaMemset(p, 0, np * 16);
    if (ce == cudaSuccess)
        ce = cudaMemcpy(e->stage, masses, (size_t)e->Ntot * sizeof(double), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) return bail(efail(e, COLATUS_E_CUDA, "upload: %s", cudaGetErrorString(ce)));
    ens_masses_kernel<<<ens_blocks(e), 256, 0, e->stream>>>(e->stage, e->d_user_off, E, e->Npad,
                                                           e->xs, e->flags);
    if ((st = elaunched(e)) != COLATUS_OK) return bail(st);
    if ((st = ens_check(e, true)) != COLATUS_OK) return bail(COLATUS_E_ARG);
    *out = e;
    return COLATUS_OK;
}

colatus_status colatus_ensemble_set_state(colatus_ens_t e, const void *x, const void *v, int dtype,
                                          int on_device) {
    if (!e || !x) return COLATUS_E_ARG;
    DeviceGuard dg(e->device);
    if (dtype != COLATUS_F32 && dtype != COLATUS_F64) return efail(e, COLATUS_E_ARG, "bad dtype");
    const size_t bytes = (size_t)e->Ntot * 3 * (dtype == COLATUS_F64 ? 8 : 4);
    const void *px = x, *pv = v;
    if (!on_device) {
        ECU(cudaMemcpyAsync(e->stage, x, bytes, cudaMemcpyHostToDevice, e->stream));
        px = e->stage;
        if (v) {
            ECU(cudaMemcpyAsync(e->stage2, v, bytes, cudaMemcpyHostToDevice, e->stream));
            pv = e->stage2;
        }
    }
    TRY(ens_check(e, true));
    ens_load_kernel<<<ens_blocks(e), 256, 0, e->stream>>>(px, pv, dtype == COLATUS_F64, e->d_user_off,
                                                         e->E, e->Npad, e->xs, e->vs, e->flags);
    TRY(elaunched(e));
    TRY(ens_check(e, true));
    e->have_state = true;
    e->spec_valid = false;
    return COLATUS_OK;
}

colatus_status colatus_ensemble_get_state(colatus_ens_t e, void *x, void *v, int dtype,
                                          int on_device, double *t, double *a) {
    if (!e) return COLATUS_E_ARG;
    DeviceGuard dg(e->device);
    if (dtype != COLATUS_F32 && dtype != COLATUS_F64) return efail(e, COLATUS_E_ARG, "bad dtype");
    TRY(ens_check(e, true));
    if (x || v) {
        if (!e->have_state) return efail(e, COLATUS_E_STATE, "no state has been set");
        const size_t bytes = (size_t)e->Ntot * 3 * (dtype == COLATUS_F64 ? 8 : 4);
        void *dx = on_device ? x : (x ? (void *)e->stage : nullptr);
        void *dv = on_device ? v : (v ? (void *)e->stage2 : nullptr);
        if (dx)
            ens_store_kernel<<<ens_blocks(e), 256, 0, e->stream>>>(
                e->xs, nullptr, e->d_user_off, e->E, e->Npad, dx, nullptr, dtype == COLATUS_F64, e->clk,
                e->G, 0);
        if (dv)
            ens_store_kernel<<<ens_blocks(e), 256, 0, e->stream>>>(
                e->vs, nullptr, e->d_user_off, e->E, e->Npad, dv, nullptr, dtype == COLATUS_F64, e->clk,
                e->G, 0);
        TRY(elaunched(e));
        if (!on_device) {
            if (x) ECU(cudaMemcpyAsync(x, e->stage, bytes, cudaMemcpyDeviceToHost, e->stream));
            if (v) ECU(cudaMemcpyAsync(v, e->stage2, bytes, cudaMemcpyDeviceToHost, e->stream));
        }
        ECU(cudaStreamSynchronize(e->stream));
    }
    if (t || a) {
        DevClock c;
        ECU(cudaMemcpy(&c, e->clk, sizeof(c), cudaMemcpyDeviceToHost));
        if (t) *t = c.t;
        if (a) *a = c.a;
    }
    return COLATUS_OK;
}

colatus_status colatus_ensemble_forces(colatus_ens_t e, void *acc_out, int dtype, int on_device) {
    if (!e || !acc_out) return COLATUS_E_ARG;
    DeviceGuard dg(e->device);
    if (dtype != COLATUS_F32 && dtype != COLATUS_F64) return efail(e, COLATUS_E_ARG, "bad dtype");
    if (!e->have_state) return efail(e, COLATUS_E_STATE, "no state has been set");
    TRY(ens_force_at_state(e));
    void *dst = on_device ? acc_out : (void *)e->stage;
    ens_store_kernel<<<ens_blocks(e), 256, 0, e->stream>>>(e->acc, nullptr, e->d_user_off, e->E,
                                                          e->Npad, dst, nullptr, dtype == COLATUS_F64,
                                                          e->clk, e->G, 1);
    TRY(elaunched(e));
    if (!on_device) {
        ECU(cudaMemcpyAsync(acc_out, e->stage, (size_t)e->Ntot * 3 * (dtype == COLATUS_F64 ? 8 : 4),
                            cudaMemcpyDeviceToHost, e->stream));
        TRY(ens_check(e, true));
    }
    e->spec_valid = false;
    return COLATUS_OK;
}

colatus_status colatus_ensemble_step(colatus_ens_t e, double dt, int64_t nsteps) {
    NvtxRange nvtx_("colatus_ensemble_step");
    if (!e) return COLATUS_E_ARG;
    DeviceGuard dg(e->device);
    if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0)
        return efail(e, COLATUS_E_ARG, "dt must be > 0 and nsteps >= 0");
    if (!e->have_state) return efail(e, COLATUS_E_STATE, "no state has been set");
    if (nsteps == 0) return COLATUS_OK;
    if (!e->spec_valid || e->spec_tau != dt) {
        // the opening: KDK's half kick (force at the state) and drift, or DKD's half drift
        const bool dkd = e->scheme == COLATUS_DKD;
        if (!dkd) TRY(ens_force_at_state(e));
        ens_table_kernel<<<1, 1, 0, e->stream>>>(e->cosmo, e->clk, e->table, 1, dt, e->G, kFriedmannSub,
                                                 e->scheme == COLATUS_KDK_CANONICAL ? 1 : 0);
        TRY(elaunched(e));
        ens_open_kernel<<<ens_blocks(e), 256, 0, e->stream>>>(e->xs, e->vs, e->acc, e->vh, e->pk[e->cur],
                                                             e->table, dt, e->E, kEnsTile, e->Npad,
                                                             dkd ? 1 : 0);
        TRY(elaunched(e));
        e->spec_valid = true;
        e->spec_tau = dt;
    }
    const long long full = nsteps / kEnsChunk;
    const int rem = (int)(nsteps % kEnsChunk);
    for (long long f = 0; f < full; ++f) {
        if (!e->graph[e->cur] || e->graph_tau[e->cur] != dt) TRY(ens_capture(e, dt));
        ECU(cudaGraphLaunch(e->graph[e->cur], e->stream));
        e->launches += 1 + 2 * kEnsChunk;
        e->interactions += kEnsChunk * e->pairs;
    }
    if (rem) TRY(ens_steps(e, dt, rem));
    e->host_step += nsteps;
    return COLATUS_OK;
}

colatus_status colatus_ensemble_synchronize(colatus_ens_t e) {
    if (!e) return COLATUS_E_ARG;
    DeviceGuard dg(e->device);
    return ens_check(e, true);
}

colatus_status colatus_ensemble_set_scheme(colatus_ens_t e, colatus_scheme scheme) {
    if (!e) return COLATUS_E_ARG;
    DeviceGuard dg(e->device);
    if (scheme != COLATUS_DKD && scheme != COLATUS_KDK && scheme != COLATUS_KDK_CANONICAL)
        return efail(e, COLATUS_E_ARG, "bad scheme %d", (int)scheme);
    if (scheme == e->scheme) return COLATUS_OK;
    ECU(cudaStreamSynchronize(e->stream));
    // the captured graphs hold the other scheme's kernels; the next step re-opens
    for (cudaGraphExec_t &g : e->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    e->scheme = scheme;
    e->spec_valid = false;
    return COLATUS_OK;
}

colatus_status colatus_ensemble_record_tracers(colatus_ens_t e, const int64_t *idx, int ntr,
                                               int64_t capacity_steps) {
    if (!e) return COLATUS_E_ARG;
    DeviceGuard dg(e->device);
    if (ntr < 0) return efail(e, COLATUS_E_ARG, "ntr must be >= 0");
    if (ntr > 0 && (!idx || capacity_steps < 1))
        return efail(e, COLATUS_E_ARG, "need indices and capacity_steps >= 1");
    std::vector<int> slot;
    if (ntr > 0) {
        // dense index k of realisation r -> padded body body_off[r] + (k - user_off[r])
        slot.assign(e->Npad, -1);
        for (int q = 0; q < ntr; ++q) {
            const long long k = idx[q];
            if (k < 0 || k >= e->Ntot) return efail(e, COLATUS_E_ARG, "tracer index %lld out of range", k);
            const int r = (int)(std::upper_bound(e->user_off.begin(), e->user_off.end(), k) -
                                e->user_off.begin()) - 1;
            const long long i = e->body_off[r] + (k - e->user_off[r]);
            if (slot[i] >= 0) return efail(e, COLATUS_E_ARG, "duplicate tracer index");
            slot[i] = q;
        }
    }
    ECU(cudaStreamSynchronize(e->stream));
    // the captured graphs hold the old buffers as kernel arguments
    for (cudaGraphExec_t &g : e->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    if (e->tslot) cudaFree(e->tslot);
    if (e->rec) cudaFree(e->rec);
    e->tslot = nullptr;
    e->rec = nullptr;
    e->ntr = 0;
    e->rec_cap = 0;
    if (ntr == 0) return COLATUS_OK;
    ECU(cudaMalloc(&e->tslot, (size_t)e->Npad * sizeof(int)));
    ECU(cudaMalloc(&e->rec, (size_t)capacity_steps * ntr * 6 * sizeof(float)));
    ECU(cudaMemcpy(e->tslot, slot.data(), (size_t)e->Npad * sizeof(int), cudaMemcpyHostToDevice));
    e->ntr = ntr;
    e->rec_cap = capacity_steps;
    e->rec_base = e->host_step;
    return COLATUS_OK;
}

colatus_status colatus_ensemble_read_tracers(colatus_ens_t e, float *xv_out, int64_t *nrec_out) {
    if (!e) return COLATUS_E_ARG;
    DeviceGuard dg(e->device);
    if (!nrec_out) return efail(e, COLATUS_E_ARG, "nrec_out is NULL");
    TRY(ens_check(e, true));
    if (e->ntr == 0) {
        *nrec_out = 0;
        return COLATUS_OK;
    }
    const long long total = e->host_step - e->rec_base;
    const long long nrec = std::min(total, e->rec_cap);
    *nrec_out = nrec;
    if (!xv_out || nrec == 0) return COLATUS_OK;
    const size_t row = (size_t)e->ntr * 6;
    std::vector<float> ring((size_t)e->rec_cap * row);
    ECU(cudaMemcpy(ring.data(), e->rec, ring.size() * sizeof(float), cudaMemcpyDeviceToHost));
    for (long long k = 0; k < nrec; ++k) {
        const long long s = total - nrec + k;
        std::memcpy(xv_out + k * row, ring.data() + (s % e->rec_cap) * row, row * sizeof(float));
    }
    return COLATUS_OK;
}

colatus_status colatus_ensemble_stats(colatus_ens_t e, int profile_on, double out[6]) {
    if (!e || !out) return COLATUS_E_ARG;
    DeviceGuard dg(e->device);
    ECU(cudaStreamSynchronize(e->stream));
    double ms = 0.0;
    for (size_t k = 0; k + 1 < e->ev_used; k += 2) {
        float t = 0.f;
        ECU(cudaEventElapsedTime(&t, e->ev[k], e->ev[k + 1]));
        ms += t;
    }
    out[0] = (double)e->launches;
    out[1] = e->interactions;
    out[2] = (double)e->host_step;
    out[3] = e->pairs;
    out[4] = ms;
    out[5] = (double)(e->ev_used / 2);
    e->ev_used = 0;
    e->profiling = profile_on != 0;
    return COLATUS_OK;
}

colatus_status colatus_ensemble_set_tuning(colatus_ens_t e, int shape) {
    if (!e) return COLATUS_E_ARG;
    DeviceGuard dg(e->device);
    if (shape < -1 || shape >= kEnsShapes) return efail(e, COLATUS_E_ARG, "shape must be -1 .. %d", kEnsShapes - 1);
    if (shape >= 0 && e->shape_G[shape] < 1) return efail(e, COLATUS_E_ARG, "shape %d does not fit", shape);
    TRY(ens_check(e, true));
    ens_set_shape(e, shape < 0 ? ens_default_shape(e) : shape);
    return COLATUS_OK;
}

colatus_status colatus_ensemble_autotune(colatus_ens_t e, int reps, double out_ms[4], int *chosen) {
    if (!e) return COLATUS_E_ARG;
    DeviceGuard dg(e->device);
    if (reps < 1) return efail(e, COLATUS_E_ARG, "reps must be >= 1");
    if (!e->have_state) return efail(e, COLATUS_E_STATE, "no state has been set");
    TRY(ens_check(e, true));
    ens_pack_kernel<<<ens_blocks(e), 256, 0, e->stream>>>(e->xs, e->pk[2], e->E, kEnsTile, e->Npad);
    TRY(elaunched(e));
    cudaEvent_t ev[2] = {nullptr, nullptr};
    colatus_status st = COLATUS_OK;
    double ms[kEnsShapes];
    if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess)
        st = efail(e, COLATUS_E_CUDA, "event creation failed");
    const bool prof = e->profiling;
    e->profiling = false;
    for (int sh = 0; sh < kEnsShapes && st == COLATUS_OK; ++sh) {
        ms[sh] = 0.0;
        if (e->shape_G[sh] < 1) continue;   // does not fit
        ens_apply_shape(e, sh);
        st = ens_force(e, e->pk[2]);   // warm-up (lazy module loading)
        if (st == COLATUS_OK && cudaEventRecord(ev[0], e->stream) != cudaSuccess)
            st = efail(e, COLATUS_E_CUDA, "event record failed");
        for (int r = 0; r < reps && st == COLATUS_OK; ++r) st = ens_force(e, e->pk[2]);
        float t = 0.f;
        if (st == COLATUS_OK && (cudaEventRecord(ev[1], e->stream) != cudaSuccess ||
                                 cudaEventSynchronize(ev[1]) != cudaSuccess ||
                                 cudaEventElapsedTime(&t, ev[0], ev[1]) != cudaSuccess))
            st = efail(e, COLATUS_E_CUDA, "event timing failed");
        ms[sh] = (double)t / reps;
    }
    e->profiling = prof;
    for (cudaEvent_t v : ev)
        if (v) cudaEventDestroy(v);
    if (st == COLATUS_OK) st = ens_check(e, true);
    int best = 0;
    if (st == COLATUS_OK)
        for (int sh = 1; sh < kEnsShapes; ++sh)
            if (e->shape_G[sh] > 0 && ms[sh] < ms[best]) best = sh;
    ens_set_shape(e, st == COLATUS_OK ? best : ens_default_shape(e));
    if (st != COLATUS_OK) return st;
    for (int sh = 0; sh < kEnsShapes; ++sh)
        if (out_ms) out_ms[sh] = ms[sh];
    if (chosen) *chosen = best;
    return COLATUS_OK;
}

const char *colatus_ensemble_last_error(colatus_ens_t e) { return e ? e->err : g_init_err; }

void colatus_ensemble_destroy(colatus_ens_t e) {
    if (!e) return;
    {
        DeviceGuard dg(e->device);
        if (e->stream) cudaStreamSynchronize(e->stream);
        ens_free(e);
    }
    delete e;
}

}  // extern "C"
