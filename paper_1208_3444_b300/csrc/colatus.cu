// colatus.cu -- the C ABI of include/colatus.h: context, state, force and step
// entry points of the COLATUS hot path (arXiv 1208.3444, Eqs. 1-5) on sm_103a.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "adjoint.cuh"
#include "colatus.h"
#include "common.cuh"
#include "diagnostics.cuh"
#include "ens_sym.cuh"
#include "ensemble.cuh"
#include "ewald.cuh"
#include "ewald_adjoint.cuh"
#include "force.cuh"
#include "force_sym.cuh"
#include "integrate.cuh"
#include "probe.cuh"
#include "spectrum.cuh"
#include "tangent.cuh"

using namespace colatus;

// ------------------------------------------------------------------ kernels
// FP32 force variants: four tile shapes, each plain or compensated (TwoSum
// fold), for general or equal masses.  Shapes (threads x i-bodies per
// thread, j-tile): 0 = 512 x 4, 512 (one CTA per SM, 2048-body i-tiles) for
// large N; 1 = 256 x 4, 512 (two CTAs per SM) for medium N; 2 = 128 x 2, 64
// for small N; 3 = 512 x 4 on 2048-body tiles with every pair evaluated once
// (force_sym.cuh: Newton's third law, 14 FP32 lane-ops per pair instead of
// 2 x 11).  Unroll depth and fold length per variant come from sweeps on
// B300 (interactions per SM per clock).  colatus_autotune times the shapes
// that fit N and keeps the fastest.
namespace {

constexpr int kStages = 4;
constexpr int kShapes = 4;
constexpr int kSymShape = 3;
// pair-once force: sub-phase tables below this many whole phases per CTA
// (at 32^3, 15 phases per CTA: the slowest SM 4.7 % above the average with
// whole phases, 1.9 % with sub-phases; at 2^21 bodies, 57000 phases per CTA,
// the whole-phase loop is 2 % faster)
constexpr long long kSubPhaseBelow = 64;
constexpr int kSymNT = 512, kSymIPT = 4, kSymUnr = 8;
// The pair-once shape is the built-in choice from this many tiles up (fewer
// tiles leave most CTAs less than one unit) and while its partial sums take
// at most 1/kSymMemShare of the device's memory (they grow as N^2 / T: one
// column slot per tile pair; 17 GB in FP32 at 2^21 bodies, an eighth of a
// B300's 288 GB less 2 %).
constexpr int kSymMinTiles = 8;
constexpr int kSymMemShare = 8;

struct F32Variant {
    int nt, ipt, jt;
    bool comp, eqm;
    int nrcp;
    int smem;
    const void *fn;
    void (*launch)(int grid, cudaStream_t, const float *, float4 *, int *, ForceLaunch, float,
                   float);
    bool sym = false;                // each pair once (force_sym_f32_kernel)
    const void *fn_fine = nullptr;   // its instance for sub-phase tables
};

template <int NT, int IPT, int JT, int FOLD, bool COMP, bool EQM, int MINB, int UNR, int NRCP>
void launch_f32(int grid, cudaStream_t st, const float *pk, float4 *part, int *flags, ForceLaunch L,
                float eps2, float mass_eq) {
    using K = F32Kernel<NT, IPT, JT, kStages, FOLD, COMP, EQM>;
    force_f32_kernel<NT, IPT, JT, kStages, FOLD, COMP, EQM, MINB, UNR, NRCP>
        <<<grid, NT, K::SMEM, st>>>(pk, part, flags, L, eps2, mass_eq);
}

template <int NT, int IPT, int JT, int FOLD, bool COMP, bool EQM, int MINB, int UNR, int NRCP = 0>
F32Variant make_f32() {
    using K = F32Kernel<NT, IPT, JT, kStages, FOLD, COMP, EQM>;
    return F32Variant{NT, IPT, JT, COMP, EQM, NRCP, K::SMEM,
                      (const void *)force_f32_kernel<NT, IPT, JT, kStages, FOLD, COMP, EQM, MINB, UNR, NRCP>,
                      &launch_f32<NT, IPT, JT, FOLD, COMP, EQM, MINB, UNR, NRCP>};
}

template <bool COMP, bool EQM>
void launch_sym(int grid, cudaStream_t st, const float *pk, float4 *part, int *flags, ForceLaunch L,
                float eps2, float mass_eq) {
    using K = SymKernel<kSymNT, kSymIPT, COMP>;
    if (L.fine)
        force_sym_f32_kernel<kSymNT, kSymIPT, COMP, EQM, kSymUnr, PlummerPair, true>
            <<<grid, kSymNT, K::SMEM, st>>>(pk, part, flags, L, eps2, mass_eq, PlummerPair::Args{});
    else
        force_sym_f32_kernel<kSymNT, kSymIPT, COMP, EQM, kSymUnr, PlummerPair, false>
            <<<grid, kSymNT, K::SMEM, st>>>(pk, part, flags, L, eps2, mass_eq, PlummerPair::Args{});
}

template <bool COMP, bool EQM>
F32Variant make_sym() {
    using K = SymKernel<kSymNT, kSymIPT, COMP>;
    F32Variant v{kSymNT, kSymIPT, K::T, COMP, EQM, 0, K::SMEM,
                 (const void *)force_sym_f32_kernel<kSymNT, kSymIPT, COMP, EQM, kSymUnr>,
                 &launch_sym<COMP, EQM>};
    v.sym = true;
    v.fn_fine = (const void *)force_sym_f32_kernel<kSymNT, kSymIPT, COMP, EQM, kSymUnr, PlummerPair, true>;
    return v;
}

// index = 4 * shape + 2 * comp + eqm.  An optional last argument (NRCP)
// would move 1/s^2 of the first NRCP i-bodies of each thread from the FMA
// pipe (a square of the rsqrt) to the MUFU pipe (an rcp).  On B300 at
// N = 32^3 one i-body in four was 1 % faster for the compensated kernel
// called alone but 1 % slower inside the step loop, and slower for the plain
// kernel, so no single-system variant takes it (the ensemble's 64 x 4 does).
enum { V_COMP = 2, V_EQM = 1, NUM_F32_VARIANTS = 4 * kShapes };

const F32Variant &f32_variant(int v) {
    static const F32Variant table[NUM_F32_VARIANTS] = {
        make_f32<512, 4, 512, 256, false, false, 1, 2>(),
        make_f32<512, 4, 512, 256, false, true, 1, 4>(),
        make_f32<512, 4, 512, 256, true, false, 1, 4>(),
        make_f32<512, 4, 512, 256, true, true, 1, 2>(),
        make_f32<256, 4, 512, 256, false, false, 2, 2>(),
        make_f32<256, 4, 512, 256, false, true, 2, 2>(),
        make_f32<256, 4, 512, 128, true, false, 2, 2>(),
        make_f32<256, 4, 512, 128, true, true, 2, 2>(),
        make_f32<128, 2, 64, 32, false, false, 4, 2>(),
        make_f32<128, 2, 64, 32, false, true, 4, 2>(),
        make_f32<128, 2, 64, 32, true, false, 4, 2>(),
        make_f32<128, 2, 64, 32, true, true, 4, 2>(),
        make_sym<false, false>(),
        make_sym<false, true>(),
        make_sym<true, false>(),
        make_sym<true, true>(),
    };
    return table[v];
}

constexpr int kF64NT = 128, kF64IPT = 2, kF64JT = 64;
using F64K = F64Kernel<kF64NT, kF64IPT, kF64JT, kStages>;

// VJP kernels: FP32 256 threads x 4 i-bodies, 256-body j-tiles, one CTA per
// SM, j-loop unrolled by 4 (the fastest of a sweep of about 30 shapes and
// unroll depths on B300 at 32^3); FP64 128 x 1, 32-body tiles
constexpr int kVjpNT = 256, kVjpIPT = 4, kVjpJT = 256, kVjpMINB = 1, kVjpUnr = 4;
// Pair-once equal-mass VJP (vjp_sym.cuh): 256 threads x 4 i-bodies on
// 1024-body tiles (the general VJP's padding), one CTA per SM (about 230
// registers), rotation unrolled by 8; used from 8 tiles on, like the force's.
constexpr int kVjpSymNT = 256, kVjpSymUnr = 8;
using VjpSymK = VjpSymKernel<kVjpSymNT>;
// Pair-once VJP for any masses (vjp_sym.cuh): the same shape and tiles.
constexpr int kVjpGenNT = 256, kVjpGenUnr = 8;
using VjpGenK = VjpSymGenKernel<kVjpGenNT>;
using VjpK = VjpKernel<kVjpNT, kVjpIPT, kVjpJT, kStages>;
static_assert(kVjpIPT == 4, "the equal-mass VJP kernel shares the VJP's launch plan (4 i-bodies per thread)");
constexpr int kV64NT = 128, kV64JT = 32;
using Vjp64K = Vjp64Kernel<kV64NT, kV64JT, kStages>;

// JVP (tangent) kernel: 128 threads x 2 i-bodies, 128-body j-tiles of 64 B,
// j-loop unrolled by 4 (fastest of eight shapes timed on B300 at 32^3 with
// 64 tangents: 38.6 ms per step, 13 % less than without unrolling)
constexpr int kJvpNT = 256, kJvpIPT = 1, kJvpJT = 128, kJvpMINB = 1, kJvpUnr = 4;
using JvpK = JvpKernel<kJvpNT, kJvpIPT, kJvpJT, kStages>;
// the periodic JVP runs the same shape and plan (tiles, units, segments)
constexpr int kEwJvpMinB = 1;

// Periodic (Ewald) real-space kernels: FP32 256 threads x 2 i-bodies,
// 256-body j-tiles; FP64 128 x 1, 32-body tiles.
// 512 x 2 at one CTA per SM: 6 % faster than 256 x 2 at two, among eight
// shapes timed on B300 at 32^3 (equal masses, compensated)
constexpr int kEwNT = 512, kEwIPT = 2, kEwJT = 256, kEwFold = 32, kEwMinB = 1;
// Pair-once real space (force_sym.cuh with EwaldPair): 512 threads x 2
// i-bodies on 1024-body tiles, one CTA per SM; the built-in choice from 8
// tiles on, like the isolated force's.
constexpr int kEwSymNT = 512, kEwSymIPT = 2, kEwSymUnr = 2;
using EwSymK = SymKernel<kEwSymNT, kEwSymIPT, false>;
using EwSymKC = SymKernel<kEwSymNT, kEwSymIPT, true>;
using EwK = EwaldF32Kernel<kEwNT, kEwIPT, kEwJT, kStages, kEwFold, false>;
using EwKC = EwaldF32Kernel<kEwNT, kEwIPT, kEwJT, kStages, kEwFold, true>;
constexpr int kEw64NT = 128, kEw64JT = 32;
using Ew64K = EwaldF64Kernel<kEw64NT, kEw64JT, kStages>;
// Periodic VJP (real space): FP32 256 threads x 2 i-bodies, 256-body tiles of
// the VJP layout; FP64 128 x 1, 32-body tiles.
constexpr int kEwVjpNT = 256, kEwVjpIPT = 2, kEwVjpJT = 256, kEwVjpMinB = 1;
using EwVjpK = EwaldVjpKernel<kEwVjpNT, kEwVjpIPT, kEwVjpJT, kStages>;
// pair-once periodic VJP: the VJP for any masses with the real-space pair term
constexpr int kEwVjpSymUnr = 4;
constexpr int kEwV64NT = 128, kEwV64JT = 32;
using EwVjp64K = EwaldVjp64Kernel<kEwV64NT, kEwV64JT, kStages>;
constexpr int kEwMaxNk = 63;   // shared memory of the k-space kernels in FP64; a pencil fits one block
constexpr int kEwRhoBlocksPerSM = 8;   // structure-factor blocks per SM (k chunks x body splits)

constexpr long long kPadAlloc = 1024;   // buffers hold N rounded up to this
// threads per block of the FP32 step epilogues (one body per thread; their
// segment sums are L2-latency bound, so smaller blocks spread them over more SMs)
constexpr int kEpiThreads = 256;
constexpr int kChunk = 1024;            // steps enqueued per chunk of colatus_step
constexpr int kTabCap = 4096;           // ring of look-ahead schedule entries
constexpr int kLookahead = 256;         // schedule entries kept ahead of the state
constexpr int kFriedmannSub = 8;        // RK4 sub-steps per half step
constexpr int kTabEvents = 64;          // extension events kept in flight (one per piece)
constexpr int kReadSlots = 4;      // asynchronous read-backs in flight per context
constexpr int kTabPiece = 64;           // schedule entries per extension launch
static_assert(kChunk + 4 * kLookahead <= kTabCap, "schedule ring too small");

long long round_up(long long n, long long m) { return (n + m - 1) / m * m; }

// Segments an i-tile can have under the split of W units over G CTAs.
int max_segments(const ForceLaunch &L) {
    long long smax = 1;
    for (long long it = 0; it < L.n_it; ++it) {
        const long long g0 = sk_owner(it * L.n_jt, L.W, L.G);
        const long long g1 = sk_owner((it + 1) * L.n_jt - 1, L.W, L.G);
        smax = std::max(smax, g1 - g0 + 1);
    }
    return (int)smax;
}

ForceLaunch make_launch(long long n_pad, int itile, int jt, long long g_target) {
    ForceLaunch L{};
    L.n_it = (int)(n_pad / itile);
    L.n_jt = (int)(n_pad / jt);
    L.W = (long long)L.n_it * L.n_jt;
    L.G = (int)std::max(1LL, std::min(g_target, L.W));
    L.S_max = max_segments(L);
    return L;
}


// Launch geometry of a persistent kernel.  Its grid leaves one SM free: the
// Friedmann schedule kernel extends the look-ahead schedule on a side stream
// while steps run, and it claims a whole SM's shared memory so that no force
// CTA shares its SM (a lone FP64 thread next to a force CTA slows that CTA,
// and so the whole stream-K grid, by ~1.7x on this GPU).  The grid is the
// same whether or not an extension is running, so the segment sums, and the
// results, do not depend on timing.
struct ForcePlan {
    int variant = -1;       // F32 variant, or -1 for FP64
    long long n_pad = 0;    // bodies incl. zero-mass padding
    int itile = 0, jt = 0;
    ForceLaunch L{};
    size_t part_bytes = 0;
    bool fits = true;       // usable for this N (colatus_set_tuning, colatus_autotune)
};

// Launch geometry of a plan (n_pad, itile, jt set) on all SMs but one;
// elem_bytes per segment entry per body.
void finish_plan(ForcePlan &p, int occ, int num_sms, size_t elem_bytes) {
    p.L = make_launch(p.n_pad, p.itile, p.jt, (long long)occ * std::max(1, num_sms - 1));
    p.part_bytes = (size_t)p.L.n_it * p.L.S_max * p.itile * elem_bytes;
}

}  // namespace

// ------------------------------------------------------------------ context
struct colatus_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    long long N = 0, n_alloc = 0;
    size_t sym_max_bytes = 0;      // largest partial-sum buffer of a pair-once plan
    double eps = 0.0, G = 1.0;
    Cosmo cosmo{};
    colatus_prec prec = COLATUS_FP32;
    colatus_scheme scheme = COLATUS_KDK;

    // host-side bookkeeping (all deterministic, no device read needed)
    long long host_step = 0;
    int tuned_shape = -1;      // FP32 force shape forced by tuning (-1: built-in choice)
    double defo_C = 0.0;       // Eq. 6 deformation strength C psi (0: off)
    double defo_x[3] = {0.0, 0.0, 0.0};
    bool eq_mass = false;      // all masses equal (as floats): EQM force kernels
    float mass_eq = 0.f;
    // look-ahead Friedmann schedule: entries [tab_lo, tab_hi) for step size
    // tab_tau and G tab_G, computed on tstream ahead of the steps
    bool tab_valid = false;
    long long tab_hi = 0;
    int tab_smem = 0;          // dynamic shared memory of the schedule kernel: a whole SM's
    double tab_tau = 0.0, tab_G = 0.0;
    bool have_state = false;
    bool acc_valid = false;    // acc holds F at the state position
    bool spec_valid = false;   // pk[cur] holds the next step's force input
    double spec_tau = 0.0;
    int cur = 0;
    long long launches = 0;
    double interactions = 0.0;

    // FP32 state: xs (x,y,z,m), vs, vh (KDK half-step velocity), acc (G-less F)
    float4 *xs = nullptr, *vs = nullptr, *vh = nullptr, *acc = nullptr;
    float *pk[3] = {nullptr, nullptr, nullptr};   // [0],[1] ping-pong, [2] aux
    float *pk_ew = nullptr;                       // periodic: the force input wrapped into the box
    // FP64 state
    double4 *xs64 = nullptr, *vs64 = nullptr, *vh64 = nullptr, *acc64 = nullptr;
    double4 *pos64[3] = {nullptr, nullptr, nullptr};
    double *m64 = nullptr;

    void *part = nullptr;
    size_t part_bytes = 0;
    int *flags = nullptr;
    int *sym_tab = nullptr;        // tables of the pair-once force plans (force_sym.cuh)
    int *mstat = nullptr;          // [min, max] float bits of the masses
    DevClock *clk = nullptr;       // state clock (t, a, steps)
    DevClock *tclk = nullptr;      // schedule frontier
    StepCoef *table = nullptr;     // kTabCap ring, entry s % kTabCap
    cudaStream_t tstream = nullptr;
    cudaEvent_t main_ev = nullptr;
    // one event per schedule extension, with the step count it completes
    cudaEvent_t tab_ev[kTabEvents] = {};
    long long tab_ev_covers[kTabEvents] = {};
    int tab_ev_next = 0;
    // asynchronous state read-back (colatus_get_state_async): a copy stream
    // and kReadSlots staging slots, each with its snapshot / copy-done
    // events; the host may run that many read-backs ahead of the copies
    cudaStream_t cstream = nullptr;
    struct ReadSlot {
        void *x = nullptr, *v = nullptr;   // device staging, N x 3 doubles each
        cudaEvent_t snap = nullptr, done = nullptr;
        bool busy = false;
    } rslot[kReadSlots];
    int rnext = 0;
    double *stage = nullptr;       // N x 3 doubles for host <-> device transfers
    double *stage2 = nullptr;
    double *diag = nullptr;        // diagnostic partial sums

    // tracers
    int *tslot = nullptr;
    float *rec = nullptr;
    int ntr = 0;
    long long rec_cap = 0, rec_base = 0;
    std::vector<long long> tidx;

    ForcePlan plan32[NUM_F32_VARIANTS];
    ForcePlan plan64;
    ForcePlan plan_vjp32, plan_vjp64;
    ForcePlan plan_vjp_sym;            // pair-once equal-mass VJP (fits: usable for this N)
    int *vjp_sym_tab = nullptr;
    ForcePlan plan_vjp_gen;            // pair-once VJP for any masses
    ForcePlan plan_ewvjp_sym;          // pair-once periodic real-space VJP
    int *vjp_gen_tab = nullptr;
    int *ewvjp_sym_tab = nullptr;
    ForcePlan plan_ewvjp32, plan_ewvjp64;   // periodic VJP (real space)

    // periodic boundaries (colatus_set_periodic): Ewald parameters and buffers
    bool periodic = false;
    double box = 0.0, ew_alpha_req = 0.0;   // requested alpha (<= 0: from the precision)
    int ew_nk_req = 0;                      // requested nk (<= 0: from the precision)
    EwaldArgs ew{};
    int nkv = 0;
    double *kw = nullptr;
    double2 *rho = nullptr;
    void *rho_part = nullptr;               // [splits][nkv] partial structure factors
    size_t rho_part_bytes = 0;
    void *pot_part = nullptr;               // [splits][N] potential pair sums (diagnostics)
    size_t pot_part_bytes = 0;
    double2 *wcs = nullptr;                 // [nkv] (w C, w S) as float2 or double2
    KPencil *pen = nullptr;                 // k-vector pencils (runs of nz at fixed nx, ny)
    int *rchunk = nullptr, *fchunk = nullptr;   // first pencil of each k-space chunk (+ end)
    int npen = 0, nrchunk = 0, nfchunk = 0, rchunk_np = 0;   // rchunk_np: most pencils in one chunk
    void *lr = nullptr;                     // n_alloc float4 / double4 long-range forces
    void *lrv = nullptr;                    // n_alloc float4 / double4 reciprocal VJP (dL/dx, dL/dm)
    void *kwr = nullptr, *kwl = nullptr;    // [nkv] w_k rho(k), w_k Lambda(k) of the VJP
    size_t kwrl_cap = 0;
    void *ph = nullptr;                     // [n_alloc][3][nk+1] phase tables (float2 / double2)
    size_t ph_bytes = 0;
    size_t kv_cap = 0;
    ForcePlan plan_ew32[2], plan_ew64;
    ForcePlan plan_ew_sym[2];          // pair-once real space (plain, compensated)
    int *ew_sym_tab = nullptr;

    // tangent model (colatus_tangent_*)
    struct Tangent {
        bool ready = false, open = false;
        int B = 0, nchunk = 0;
        long long n_pad = 0, last_step = -1;
        double tau = 0.0;
        ForcePlan plan;
        float4 *dx = nullptr, *dv = nullptr, *dvh = nullptr;
        float4 *dxp = nullptr;                   // [B][n_pad] packed tangent positions (periodic)
        float *pkt = nullptr;                    // packed JVP input, pair-interleaved
        long long *seeds = nullptr;
        float *growth = nullptr;
        float4 *lrt = nullptr;                   // [B][n_pad] reciprocal-space JVP (periodic)
        long long cap = 0, base = 0;
        double dir[3] = {1.0, 0.0, 0.0};
    } tan;

    // discrete adjoint (colatus_adjoint_forward / colatus_adjoint_backward)
    struct Adjoint {
        bool ready = false;
        long long nsteps = 0, step0 = 0;
        int k = 0, nck = 0;
        double tau = 0.0;
        colatus_prec prec = COLATUS_FP32;
        colatus_scheme scheme = COLATUS_KDK;      // of the recorded pass
        double G = 1.0;
        size_t ck_bytes = 0, seg_bytes = 0, tab_bytes = 0;
        void *ck_x = nullptr, *ck_v = nullptr;   // [nck][n_alloc] checkpoints (float4 / double4)
        void *seg_x = nullptr;                   // [k][n_alloc] recomputed positions
        StepCoef *table = nullptr;               // [nsteps] schedule of the forward
        cudaEvent_t tab_ev = nullptr;            // table computed (side stream)
        DevClock *rclk = nullptr;                // scratch clock
        void *rvs = nullptr, *rvh = nullptr, *racc = nullptr;   // recompute state
        void *rpk[2] = {nullptr, nullptr};       // recompute force inputs
        void *lx = nullptr, *lv = nullptr, *lvh = nullptr, *lm = nullptr;   // adjoint variables
        void *pkw = nullptr;                     // bodies + co-vector for the VJP
        void *seg_f = nullptr;                   // [k+1][n_alloc] forces of a segment (equal-mass VJP)
        size_t segf_bytes = 0;
        void *seg_v = nullptr;                   // [k][n_alloc] recomputed velocities (DKD)
        size_t segv_bytes = 0;
    } adj;

    // force-kernel timing (colatus_profile_forces)
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_cat;      // category of each event pair: 0 force, 1 VJP, 2 adjoint update
    size_t ev_used = 0;

    char err[512] = {0};
};

namespace {

char g_init_err[512] = {0};

colatus_status fail(colatus_t ctx, colatus_status st, const char *fmt, ...) {
    char *buf = ctx ? ctx->err : g_init_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return st;
}

#define CU(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? COLATUS_E_OOM : COLATUS_E_CUDA, \
                        "%s: %s", #call, cudaGetErrorString(e_));                         \
    } while (0)

#define TRY(expr)                              \
    do {                                       \
        colatus_status s_ = (expr);            \
        if (s_ != COLATUS_OK) return s_;       \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

colatus_status launched(colatus_t ctx) {
    ++ctx->launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, COLATUS_E_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    return COLATUS_OK;
}

// ---- plans
// Whether a pair-once plan of tiles of T bodies (pl planes) could fit the
// partial-sum budget: its column slots alone, one per tile pair it < jt.
bool sym_may_fit(colatus_t ctx, long long n_pad, int T, int pl) {
    const long long n = n_pad / T;
    const double slots = 0.5 * (double)n * (double)(n - 1);
    return n >= 2 && slots * pl * T * sizeof(float4) <= (double)ctx->sym_max_bytes;
}

colatus_status build_plans(colatus_t ctx) {
    SymTables st;
    for (int v = 0; v < NUM_F32_VARIANTS; ++v) {
        const F32Variant &fv = f32_variant(v);
        if (fv.smem > 48 * 1024) {
            CU(cudaFuncSetAttribute(fv.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, fv.smem));
            if (fv.fn_fine)
                CU(cudaFuncSetAttribute(fv.fn_fine, cudaFuncAttributeMaxDynamicSharedMemorySize, fv.smem));
        }
        int occ = 0;
        CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fv.fn, fv.nt, fv.smem));
        if (occ < 1) return fail(ctx, COLATUS_E_CUDA, "force variant %d cannot be resident", v);
        ForcePlan &p = ctx->plan32[v];
        p.variant = v;
        p.itile = fv.nt * fv.ipt;
        p.jt = fv.jt;
        p.n_pad = round_up(ctx->N, std::max(p.itile, p.jt));
        if (!fv.sym) {
            finish_plan(p, occ, ctx->num_sms, sizeof(float4) * (fv.comp ? 2 : 1));
            p.fits = p.L.W >= p.L.G;
            continue;
        }
        // pair-once plan: one set of tables for all four variants, the phase
        // costs of the equal-mass form (11 lane-ops per diagonal interaction,
        // 14 per symmetric pair), on all SMs but the schedule kernel's; in
        // sub-phases (one 32-pair block of every warp's slice) where a CTA
        // would get fewer than kSubPhaseBelow whole phases, so that shares end
        // closer to their cost quantiles; not built when even its column slots
        // alone would not fit
        const int pl = fv.comp ? 2 : 1;
        if (!sym_may_fit(ctx, p.n_pad, p.itile, pl)) {
            p.fits = false;
            continue;
        }
        if (st.tab.empty()) {
            using SK = SymKernel<kSymNT, kSymIPT, false>;
            const long long grid = (long long)occ * std::max(1, ctx->num_sms - 1);
            const long long nt = p.n_pad / p.itile, phases = nt * (nt + 1) / 2 * SK::NW;
            const int units = phases < kSubPhaseBelow * grid ? SK::PH : SK::NW;
            st = build_sym_tables(p.n_pad, p.itile, units, grid, 11, 14);
        }
        p.L = ForceLaunch{};
        p.L.W = st.U;
        p.L.n_it = p.L.n_jt = st.n;
        p.L.G = st.G;
        p.L.S_max = st.S_row;
        p.L.col_off = (long long)st.n * st.S_row * pl * p.itile;
        p.L.fine = st.tab[1] != SymKernel<kSymNT, kSymIPT, false>::NW;   // the tables' granularity
        p.part_bytes = (size_t)((long long)st.n * st.S_row + st.slots) * pl * p.itile * sizeof(float4);
        p.fits = st.n >= 2 && p.part_bytes <= ctx->sym_max_bytes;
    }
    if (!st.tab.empty()) {
        CU(cudaMalloc(&ctx->sym_tab, st.tab.size() * sizeof(int)));
        CU(cudaMemcpy(ctx->sym_tab, st.tab.data(), st.tab.size() * sizeof(int), cudaMemcpyHostToDevice));
        for (int v = 4 * kSymShape; v < 4 * kSymShape + 4; ++v) ctx->plan32[v].L.sym = ctx->sym_tab;
    }
    int occ = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, force_f64_kernel<kF64NT, kF64IPT, kF64JT, kStages>, kF64NT, F64K::SMEM));
    if (occ < 1) return fail(ctx, COLATUS_E_CUDA, "FP64 force kernel cannot be resident");
    ForcePlan &p = ctx->plan64;
    p.variant = -1;
    p.itile = F64K::ITILE;
    p.jt = kF64JT;
    p.n_pad = round_up(ctx->N, std::max(p.itile, p.jt));
    finish_plan(p, occ, ctx->num_sms, sizeof(double4));

    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, vjp_f32_kernel<kVjpNT, kVjpIPT, kVjpJT, kStages, kVjpMINB, kVjpUnr>, kVjpNT, VjpK::SMEM));
    if (occ < 1) return fail(ctx, COLATUS_E_CUDA, "VJP kernel cannot be resident");
    ForcePlan &v = ctx->plan_vjp32;
    v.itile = VjpK::ITILE;
    v.jt = kVjpJT;
    v.n_pad = round_up(ctx->N, std::max(v.itile, v.jt));
    finish_plan(v, occ, ctx->num_sms, sizeof(float4));
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, vjp_f64_kernel<kV64NT, kV64JT, kStages>, kV64NT, Vjp64K::SMEM));
    if (occ < 1) return fail(ctx, COLATUS_E_CUDA, "FP64 VJP kernel cannot be resident");
    {
        // the pair-once equal-mass VJP: tables with its phase costs (23
        // lane-ops per diagonal interaction, 27 per symmetric pair)
        auto fn = vjp_sym_eqm_f32_kernel<kVjpSymNT, kVjpSymUnr>;
        CU(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, VjpSymK::SMEM));
        CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kVjpSymNT, VjpSymK::SMEM));
        if (occ < 1) return fail(ctx, COLATUS_E_CUDA, "pair-once VJP kernel cannot be resident");
        ForcePlan &q = ctx->plan_vjp_sym;
        q.itile = q.jt = VjpSymK::T;
        q.n_pad = round_up(ctx->N, VjpSymK::T);
        const bool may = sym_may_fit(ctx, q.n_pad, VjpSymK::T, 1);
        const SymTables st = may ? build_sym_tables(q.n_pad, VjpSymK::T, VjpSymK::NW,
                                                    (long long)occ * std::max(1, ctx->num_sms - 1), 23, 27)
                                 : SymTables{};
        q.L = ForceLaunch{};
        q.L.W = st.U;
        q.L.n_it = q.L.n_jt = st.n;
        q.L.G = st.G;
        q.L.S_max = st.S_row;
        q.L.col_off = (long long)st.n * st.S_row * q.itile;
        q.part_bytes = (size_t)((long long)st.n * st.S_row + st.slots) * q.itile * sizeof(float4);
        q.fits = may && st.n >= kSymMinTiles && q.part_bytes <= ctx->sym_max_bytes;
        if (q.fits) {
            CU(cudaMalloc(&ctx->vjp_sym_tab, st.tab.size() * sizeof(int)));
            CU(cudaMemcpy(ctx->vjp_sym_tab, st.tab.data(), st.tab.size() * sizeof(int), cudaMemcpyHostToDevice));
            q.L.sym = ctx->vjp_sym_tab;
        }
    }
    {
        // the pair-once VJP for any masses: tables with its phase costs (36
        // lane-ops per diagonal interaction, 40 per symmetric pair; 27 and 31
        // in the equal-mass form)
        auto fn = vjp_sym_f32_kernel<kVjpGenNT, kVjpGenUnr, false>;
        CU(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, VjpGenK::SMEM));
        CU(cudaFuncSetAttribute(vjp_sym_f32_kernel<kVjpGenNT, kVjpGenUnr, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, VjpGenK::SMEM));
        CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kVjpGenNT, VjpGenK::SMEM));
        if (occ < 1) return fail(ctx, COLATUS_E_CUDA, "pair-once VJP kernel (any masses) cannot be resident");
        ForcePlan &q = ctx->plan_vjp_gen;
        q.itile = q.jt = VjpGenK::T;
        q.n_pad = round_up(ctx->N, VjpGenK::T);
        const bool may = sym_may_fit(ctx, q.n_pad, VjpGenK::T, 1);
        const SymTables st = may ? build_sym_tables(q.n_pad, VjpGenK::T, VjpGenK::NW,
                                                    (long long)occ * std::max(1, ctx->num_sms - 1), 36, 40)
                                 : SymTables{};
        q.L = ForceLaunch{};
        q.L.W = st.U;
        q.L.n_it = q.L.n_jt = st.n;
        q.L.G = st.G;
        q.L.S_max = st.S_row;
        q.L.col_off = (long long)st.n * st.S_row * q.itile;
        q.part_bytes = (size_t)((long long)st.n * st.S_row + st.slots) * q.itile * sizeof(float4);
        q.fits = may && st.n >= kSymMinTiles && q.part_bytes <= ctx->sym_max_bytes;
        if (q.fits) {
            CU(cudaMalloc(&ctx->vjp_gen_tab, st.tab.size() * sizeof(int)));
            CU(cudaMemcpy(ctx->vjp_gen_tab, st.tab.data(), st.tab.size() * sizeof(int), cudaMemcpyHostToDevice));
            q.L.sym = ctx->vjp_gen_tab;
        }
    }
    {
        // the same kernel with the periodic real-space pair term: tables with
        // its phase costs (68 lane-ops per diagonal interaction, 72 per
        // symmetric pair; 59 and 63 in the equal-mass form)
        auto fn = vjp_sym_f32_kernel<kVjpGenNT, kEwVjpSymUnr, false, EwaldVjpPair>;
        CU(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, VjpGenK::SMEM));
        CU(cudaFuncSetAttribute(vjp_sym_f32_kernel<kVjpGenNT, kEwVjpSymUnr, true, EwaldVjpPair>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, VjpGenK::SMEM));
        CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kVjpGenNT, VjpGenK::SMEM));
        if (occ < 1) return fail(ctx, COLATUS_E_CUDA, "pair-once periodic VJP kernel cannot be resident");
        ForcePlan &q = ctx->plan_ewvjp_sym;
        q.itile = q.jt = VjpGenK::T;
        q.n_pad = round_up(ctx->N, VjpGenK::T);
        const bool may = sym_may_fit(ctx, q.n_pad, VjpGenK::T, 1);
        const SymTables st = may ? build_sym_tables(q.n_pad, VjpGenK::T, VjpGenK::NW,
                                                    (long long)occ * std::max(1, ctx->num_sms - 1), 68, 72)
                                 : SymTables{};
        q.L = ForceLaunch{};
        q.L.W = st.U;
        q.L.n_it = q.L.n_jt = st.n;
        q.L.G = st.G;
        q.L.S_max = st.S_row;
        q.L.col_off = (long long)st.n * st.S_row * q.itile;
        q.part_bytes = (size_t)((long long)st.n * st.S_row + st.slots) * q.itile * sizeof(float4);
        q.fits = may && st.n >= kSymMinTiles && q.part_bytes <= ctx->sym_max_bytes;
        if (q.fits) {
            CU(cudaMalloc(&ctx->ewvjp_sym_tab, st.tab.size() * sizeof(int)));
            CU(cudaMemcpy(ctx->ewvjp_sym_tab, st.tab.data(), st.tab.size() * sizeof(int), cudaMemcpyHostToDevice));
            q.L.sym = ctx->ewvjp_sym_tab;
        }
    }
    ForcePlan &w = ctx->plan_vjp64;
    w.itile = Vjp64K::ITILE;
    w.jt = kV64JT;
    w.n_pad = round_up(ctx->N, std::max(w.itile, w.jt));
    finish_plan(w, occ, ctx->num_sms, sizeof(double4));
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, ewald_vjp_f32_kernel<kEwVjpNT, kEwVjpIPT, kEwVjpJT, kStages, kEwVjpMinB>, kEwVjpNT,
        EwVjpK::SMEM));
    if (occ < 1) return fail(ctx, COLATUS_E_CUDA, "periodic VJP kernel cannot be resident");
    ForcePlan &ev = ctx->plan_ewvjp32;
    ev.itile = EwVjpK::ITILE;
    ev.jt = kEwVjpJT;
    ev.n_pad = round_up(ctx->N, std::max(ev.itile, ev.jt));
    finish_plan(ev, occ, ctx->num_sms, sizeof(float4));
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, ewald_vjp_f64_kernel<kEwV64NT, kEwV64JT, kStages>, kEwV64NT, EwVjp64K::SMEM));
    if (occ < 1) return fail(ctx, COLATUS_E_CUDA, "FP64 periodic VJP kernel cannot be resident");
    ForcePlan &ew = ctx->plan_ewvjp64;
    ew.itile = EwVjp64K::ITILE;
    ew.jt = kEwV64JT;
    ew.n_pad = round_up(ctx->N, std::max(ew.itile, ew.jt));
    finish_plan(ew, occ, ctx->num_sms, sizeof(double4));

    for (int comp = 0; comp < 2; ++comp) {
        const void *fn = comp ? (const void *)ewald_f32_kernel<kEwNT, kEwIPT, kEwJT, kStages, kEwFold,
                                                              true, kEwMinB, false>
                              : (const void *)ewald_f32_kernel<kEwNT, kEwIPT, kEwJT, kStages, kEwFold,
                                                              false, kEwMinB, false>;
        CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kEwNT, EwK::SMEM));
        if (occ < 1) return fail(ctx, COLATUS_E_CUDA, "Ewald kernel cannot be resident");
        ForcePlan &e = ctx->plan_ew32[comp];
        e.itile = EwK::ITILE;
        e.jt = kEwJT;
        e.n_pad = round_up(ctx->N, std::max(e.itile, e.jt));
        finish_plan(e, occ, ctx->num_sms, sizeof(float4) * (comp ? 2 : 1));
    }
    {
        // pair-once real space: tables with its phase costs (35 lane-ops per
        // diagonal interaction, 38 per symmetric pair)
        SymTables st;
        for (int comp = 0; comp < 2; ++comp) {
            const void *fn = comp ? (const void *)force_sym_f32_kernel<kEwSymNT, kEwSymIPT, true, false, kEwSymUnr, EwaldPair>
                                  : (const void *)force_sym_f32_kernel<kEwSymNT, kEwSymIPT, false, false, kEwSymUnr, EwaldPair>;
            const void *fe = comp ? (const void *)force_sym_f32_kernel<kEwSymNT, kEwSymIPT, true, true, kEwSymUnr, EwaldPair>
                                  : (const void *)force_sym_f32_kernel<kEwSymNT, kEwSymIPT, false, true, kEwSymUnr, EwaldPair>;
            const int smem = comp ? EwSymKC::SMEM : EwSymK::SMEM;
            CU(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            CU(cudaFuncSetAttribute(fe, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kEwSymNT, smem));
            if (occ < 1) return fail(ctx, COLATUS_E_CUDA, "pair-once Ewald kernel cannot be resident");
            ForcePlan &q = ctx->plan_ew_sym[comp];
            q.itile = q.jt = EwSymK::T;
            q.n_pad = round_up(ctx->N, EwSymK::T);
            if (!sym_may_fit(ctx, q.n_pad, EwSymK::T, comp + 1)) {
                q.fits = false;
                continue;
            }
            if (st.tab.empty())
                st = build_sym_tables(q.n_pad, EwSymK::T, EwSymK::PH,
                                      (long long)occ * std::max(1, ctx->num_sms - 1), 35, 38);
            q.L = ForceLaunch{};
            q.L.W = st.U;
            q.L.n_it = q.L.n_jt = st.n;
            q.L.G = st.G;
            q.L.S_max = st.S_row;
            q.L.col_off = (long long)st.n * st.S_row * (comp + 1) * q.itile;
            q.part_bytes = (size_t)((long long)st.n * st.S_row + st.slots) * (comp + 1) * q.itile * sizeof(float4);
            q.fits = st.n >= kSymMinTiles && q.part_bytes <= ctx->sym_max_bytes;
        }
        if (ctx->plan_ew_sym[0].fits || ctx->plan_ew_sym[1].fits) {
            CU(cudaMalloc(&ctx->ew_sym_tab, st.tab.size() * sizeof(int)));
            CU(cudaMemcpy(ctx->ew_sym_tab, st.tab.data(), st.tab.size() * sizeof(int), cudaMemcpyHostToDevice));
            ctx->plan_ew_sym[0].L.sym = ctx->plan_ew_sym[1].L.sym = ctx->ew_sym_tab;
        }
    }
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, ewald_f64_kernel<kEw64NT, kEw64JT, kStages>, kEw64NT, Ew64K::SMEM));
    if (occ < 1) return fail(ctx, COLATUS_E_CUDA, "FP64 Ewald kernel cannot be resident");
    ForcePlan &e64 = ctx->plan_ew64;
    e64.itile = Ew64K::ITILE;
    e64.jt = kEw64JT;
    e64.n_pad = round_up(ctx->N, std::max(e64.itile, e64.jt));
    finish_plan(e64, occ, ctx->num_sms, sizeof(double4));
    return COLATUS_OK;
}

// FP32 variant for the current precision and masses: wide tiles when every
// CTA still gets at least four units, narrow tiles otherwise.
// The equal-mass kernels ignore m_j, so they are used only when no zero-mass
// padding body enters the sum (N_pad == N).
// Built-in shape choice: the largest shape that still gives every CTA at
// least four units; colatus_autotune / colatus_set_tuning override it.
int default_shape(colatus_t ctx, int comp) {
    const ForcePlan &ps = ctx->plan32[4 * kSymShape + comp];
    if (ps.fits && ps.L.n_it >= kSymMinTiles) return kSymShape;
    for (int sh = 0; sh < 2; ++sh) {
        const ForcePlan &p = ctx->plan32[4 * sh + comp];
        if (p.L.W >= 4LL * p.L.G) return sh;
    }
    return 2;
}

const ForcePlan &plan_f32(colatus_t ctx) {
    if (ctx->periodic) {
        // real space: the pair-once kernel where it fits (tuning shape 3 or the
        // built-in choice), else the per-ordered-pair one (any other shape)
        const int c = ctx->prec == COLATUS_FP32_COMP ? 1 : 0;
        const ForcePlan &q = ctx->plan_ew_sym[c];
        const bool sym = q.fits && (ctx->tuned_shape < 0 || ctx->tuned_shape == kSymShape);
        return sym ? q : ctx->plan_ew32[c];
    }
    const int comp = ctx->prec == COLATUS_FP32_COMP ? V_COMP : 0;
    const int sh = ctx->tuned_shape >= 0 ? ctx->tuned_shape : default_shape(ctx, comp);
    const ForcePlan *w = &ctx->plan32[4 * sh + comp];
    if (ctx->eq_mass && w->n_pad == ctx->N) w += V_EQM;
    return *w;
}

const ForcePlan &plan_f64(colatus_t ctx) { return ctx->periodic ? ctx->plan_ew64 : ctx->plan64; }

colatus_status ensure_part(colatus_t ctx, size_t bytes) {
    if (bytes <= ctx->part_bytes) return COLATUS_OK;
    if (ctx->part) cudaFree(ctx->part);
    ctx->part = nullptr;
    ctx->part_bytes = 0;
    CU(cudaMalloc(&ctx->part, bytes));
    ctx->part_bytes = bytes;
    return COLATUS_OK;
}

// Bracket one force (cat 0) or VJP (cat 1) launch with a pair of events
// when profiling.
colatus_status prof_begin(colatus_t ctx) {
    if (!ctx->profiling) return COLATUS_OK;
    while (ctx->ev_pool.size() < ctx->ev_used + 2) {
        cudaEvent_t e;
        CU(cudaEventCreate(&e));
        ctx->ev_pool.push_back(e);
        ctx->ev_cat.push_back(0);
    }
    CU(cudaEventRecord(ctx->ev_pool[ctx->ev_used], ctx->stream));
    return COLATUS_OK;
}

colatus_status prof_end(colatus_t ctx, int cat = 0) {
    if (!ctx->profiling) return COLATUS_OK;
    CU(cudaEventRecord(ctx->ev_pool[ctx->ev_used + 1], ctx->stream));
    ctx->ev_cat[ctx->ev_used] = cat;
    ctx->ev_used += 2;
    return COLATUS_OK;
}

colatus_status grow(colatus_t ctx, void **p, size_t *have, size_t need);

// Ewald parameters for the current precision.  alpha (unless requested) from
// the real-space truncation: the images beyond the nearest are at r >= L/2,
// where the pair term is below erfc(x) + (2x/sqrt(pi)) exp(-x^2), x = alpha L/2;
// nk (unless requested) from exp(-(pi nk / (alpha L))^2), the largest k-space
// weight left out.  Both at tol = 1e-8 (FP32 modes) or 1e-15 (FP64).
colatus_status ewald_setup(colatus_t ctx) {
    const double L = ctx->box, pi = std::acos(-1.0);
    const bool f64 = ctx->prec == COLATUS_FP64;
    const double tol = f64 ? 1e-15 : 1e-8;
    double alpha = ctx->ew_alpha_req;
    if (!(alpha > 0.0)) {
        double lo = 0.5, hi = 10.0;
        for (int it = 0; it < 100; ++it) {
            const double x = 0.5 * (lo + hi);
            const double err = std::erfc(x) + 2.0 * x / std::sqrt(pi) * std::exp(-x * x);
            (err > tol ? lo : hi) = x;
        }
        alpha = 2.0 * hi / L;
    }
    int nk = ctx->ew_nk_req;
    if (nk <= 0) nk = (int)std::ceil(alpha * L / pi * std::sqrt(std::log(1.0 / tol)));
    if (nk > kEwMaxNk) return fail(ctx, COLATUS_E_ARG, "Ewald needs nk = %d > %d", nk, kEwMaxNk);
    std::vector<KVec> kv;
    std::vector<double> w;
    const double V = L * L * L, tk = 2.0 * pi / L;
    for (int nx = 0; nx <= nk; ++nx)
        for (int ny = -nk; ny <= nk; ++ny)
            for (int nz = -nk; nz <= nk; ++nz) {
                const int n2 = nx * nx + ny * ny + nz * nz;
                if (n2 == 0 || n2 > nk * nk) continue;
                if (!(nx > 0 || (nx == 0 && (ny > 0 || (ny == 0 && nz > 0))))) continue;
                const double k2 = tk * tk * n2;
                kv.push_back(KVec{nx, ny, nz, 0});
                w.push_back(2.0 * 4.0 * pi / V * std::exp(-k2 / (4.0 * alpha * alpha)) / k2);
            }
    const size_t nkv = kv.size();
    // pencils: runs of consecutive nz at fixed (nx, ny), in k order
    std::vector<KPencil> pen;
    for (size_t k = 0; k < nkv; ++k) {
        if (pen.empty() || pen.back().nx != kv[k].nx || pen.back().ny != kv[k].ny ||
            pen.back().nz0 + pen.back().len != kv[k].nz)
            pen.push_back(KPencil{kv[k].nx, kv[k].ny, kv[k].nz, 0, (int)k, 0, 0, 0});
        ++pen.back().len;
    }
    // chunks of whole pencils holding at most `cap` k-vectors: first pencil of each, then the end
    auto chunks = [&](int cap) {
        std::vector<int> c{0};
        int have = 0;
        for (int p = 0; p < (int)pen.size(); ++p) {
            if (have + pen[p].len > cap) {
                c.push_back(p);
                have = 0;
            }
            have += pen[p].len;
        }
        c.push_back((int)pen.size());
        return c;
    };
    const std::vector<int> rch = chunks(kEwKThreads);
    const std::vector<int> fch = chunks(f64 ? ew_fk<double>() : ew_fk<float>());
    if (nkv > ctx->kv_cap) {
        for (void *q : {(void *)ctx->kw, (void *)ctx->rho, (void *)ctx->wcs, (void *)ctx->pen,
                        (void *)ctx->rchunk, (void *)ctx->fchunk})
            if (q) cudaFree(q);
        ctx->kw = nullptr;
        ctx->rho = nullptr;
        ctx->wcs = nullptr;
        ctx->pen = nullptr;
        ctx->rchunk = ctx->fchunk = nullptr;
        ctx->kv_cap = 0;
        CU(cudaMalloc(&ctx->kw, nkv * sizeof(double)));
        CU(cudaMalloc(&ctx->rho, nkv * sizeof(double2)));
        CU(cudaMalloc(&ctx->wcs, nkv * sizeof(double2)));
        // at most one pencil (and chunk) per k-vector
        CU(cudaMalloc(&ctx->pen, nkv * sizeof(KPencil)));
        CU(cudaMalloc(&ctx->rchunk, (nkv + 1) * sizeof(int)));
        CU(cudaMalloc(&ctx->fchunk, (nkv + 1) * sizeof(int)));
        ctx->kv_cap = nkv;
    }
    CU(cudaMemcpyAsync(ctx->pen, pen.data(), pen.size() * sizeof(KPencil), cudaMemcpyHostToDevice,
                       ctx->stream));
    CU(cudaMemcpyAsync(ctx->rchunk, rch.data(), rch.size() * sizeof(int), cudaMemcpyHostToDevice,
                       ctx->stream));
    CU(cudaMemcpyAsync(ctx->fchunk, fch.data(), fch.size() * sizeof(int), cudaMemcpyHostToDevice,
                       ctx->stream));
    ctx->npen = (int)pen.size();
    ctx->nrchunk = (int)rch.size() - 1;
    ctx->rchunk_np = 1;
    for (int c = 0; c < ctx->nrchunk; ++c) ctx->rchunk_np = std::max(ctx->rchunk_np, rch[c + 1] - rch[c]);
    ctx->nfchunk = (int)fch.size() - 1;
    if (!ctx->lr) CU(cudaMalloc(&ctx->lr, (size_t)ctx->n_alloc * sizeof(double4)));
    if (!f64 && !ctx->pk_ew) {
        // the padding bodies stay zero: the phase kernel writes bodies 0 .. N-1
        CU(cudaMalloc(&ctx->pk_ew, (size_t)ctx->n_alloc * 4 * sizeof(float)));
        CU(cudaMemsetAsync(ctx->pk_ew, 0, (size_t)ctx->n_alloc * 4 * sizeof(float), ctx->stream));
    }
    TRY(grow(ctx, &ctx->ph, &ctx->ph_bytes,
             (size_t)ctx->n_alloc * 3 * (nk + 1) * (f64 ? sizeof(double2) : sizeof(float2))));
    CU(cudaMemcpyAsync(ctx->kw, w.data(), nkv * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));   // the host vectors go out of scope
    ctx->nkv = (int)nkv;
    EwaldArgs &A = ctx->ew;
    A.L = L;
    A.alpha = alpha;
    A.Lf = (float)L;
    A.invLf = (float)(1.0 / L);
    A.alpha_f = (float)alpha;
    A.alpha2_log2e = (float)(alpha * alpha / std::log(2.0));
    A.cg = (float)(2.0 * alpha / std::sqrt(pi));
    A.p_alpha = (float)((double)kAsP * alpha);
    A.s0 = (float)(-4.0 / 3.0 * alpha * alpha * alpha / std::sqrt(pi));
    A.s1 = (float)(0.8 * std::pow(alpha, 5) / std::sqrt(pi));
    A.x2_series = (float)((0.05 / alpha) * (0.05 / alpha));
    A.nk = nk;
    A.c2ag = (float)(2.0 * alpha * alpha * 2.0 * alpha / std::sqrt(pi));
    A.ncs0 = (float)(-1.6 * std::pow(alpha, 5) / std::sqrt(pi));
    A.ncs1 = (float)(8.0 / 7.0 * std::pow(alpha, 7) / std::sqrt(pi));
    // shared memory of the k-space kernels grows with nk
    const int nt = nk + 1;
    const size_t es = f64 ? sizeof(double) : sizeof(float);
    const size_t smem_rho = f64 ? ew_rho_smem<double>(nk, ctx->rchunk_np) : ew_rho_smem<float>(nk, ctx->rchunk_np);
    const size_t smem_f = kEwFKBytes + (size_t)kEwFThreads * 3 * nt * 2 * es;
    const void *frho = f64 ? (const void *)ewald_rho_kernel<double> : (const void *)ewald_rho_kernel<float>;
    const void *fk = f64 ? (const void *)ewald_kforce_kernel<double, double4>
                         : (const void *)ewald_kforce_kernel<float, float4>;
    CU(cudaFuncSetAttribute(frho, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rho));
    CU(cudaFuncSetAttribute(fk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_f));
    // the derivatives' reciprocal passes (VJP in this precision; the tangent
    // model's multi-tangent passes in FP32)
    const void *fkv = f64 ? (const void *)ewald_kvjp_kernel<double, double4, 1>
                          : (const void *)ewald_kvjp_kernel<float, float4, 1>;
    const size_t smem_kv = f64 ? ew_kvjp_smem<double, 1>(nk) : ew_kvjp_smem<float, 1>(nk);
    CU(cudaFuncSetAttribute(fkv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_kv));
    const void *fm4 = f64 ? (const void *)ewald_rho_multi_kernel<double, 4>
                          : (const void *)ewald_rho_multi_kernel<float, 4>;
    const size_t smem_m4 = f64 ? ew_rho_multi_smem<double, 4>(nk, ctx->rchunk_np)
                               : ew_rho_multi_smem<float, 4>(nk, ctx->rchunk_np);
    CU(cudaFuncSetAttribute(fm4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_m4));
    if (!f64) {
        CU(cudaFuncSetAttribute(ewald_rho_multi_kernel<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ew_rho_multi_smem<float, 1>(nk, ctx->rchunk_np)));
        CU(cudaFuncSetAttribute(ewald_rho_multi_kernel<float, 3 * kTB>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ew_rho_multi_smem<float, 3 * kTB>(nk, ctx->rchunk_np)));
        CU(cudaFuncSetAttribute(ewald_kvjp_kernel<float, float4, kTB>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ew_kvjp_smem<float, kTB>(nk)));
    }
    return COLATUS_OK;
}

// Periodic boundaries: the phase tables of every body (FP32: also the
// wrapped force input pk_ew), before the real-space kernel.
template <typename T>
colatus_status run_ewald_phases(colatus_t ctx, const float *pk, const double4 *pos) {
    using T2 = typename Vec2<T>::type;
    ewald_phase_kernel<T><<<blocks_for(3 * ctx->N, 128), 128, 0, ctx->stream>>>(
        masses_of(pk, pos), ctx->N, ctx->ew, static_cast<T2 *>(ctx->ph), pos ? nullptr : ctx->pk_ew);
    return launched(ctx);
}

// The k-space part, after the real-space kernel: structure factors into
// ctx->rho, then the long-range force at every body into ctx->lr.  pk (FP32
// packed) or pos (FP64) holds the positions; the phase tables are current.
template <typename T, typename T4>
colatus_status run_ewald_kspace(colatus_t ctx, const float *pk, const double4 *pos) {
    using T2 = typename Vec2<T>::type;
    const int nt = ctx->ew.nk + 1;
    T2 *ph = static_cast<T2 *>(ctx->ph);
    const int kchunks = ctx->nrchunk;
    const long long max_split = std::max(1LL, ctx->N / ew_bodies<T>());
    const int splits = (int)std::min<long long>(std::max(1, kEwRhoBlocksPerSM * ctx->num_sms / kchunks),
                                                max_split);
    TRY(grow(ctx, &ctx->rho_part, &ctx->rho_part_bytes, (size_t)splits * ctx->nkv * sizeof(double2)));
    const size_t smem_rho = ew_rho_smem<T>(ctx->ew.nk, ctx->rchunk_np);
    ewald_rho_kernel<T><<<dim3(kchunks, splits), kEwKThreads, smem_rho, ctx->stream>>>(
        masses_of(pk, pos), ctx->N, ph, ctx->pen, ctx->rchunk, ctx->rchunk_np, ctx->nkv, ctx->ew,
        static_cast<double2 *>(ctx->rho_part));
    TRY(launched(ctx));
    T2 *wcs = reinterpret_cast<T2 *>(ctx->wcs);
    ewald_rho_sum_kernel<T><<<blocks_for(ctx->nkv, 256), 256, 0, ctx->stream>>>(
        static_cast<const double2 *>(ctx->rho_part), splits, ctx->nkv, ctx->kw, ctx->rho, wcs);
    TRY(launched(ctx));
    const size_t smem_f = kEwFKBytes + (size_t)kEwFThreads * 3 * nt * sizeof(T2);
    ewald_kforce_kernel<T, T4><<<blocks_for(ctx->N, kEwFThreads), kEwFThreads * kEwFSlices, smem_f,
                                 ctx->stream>>>(ctx->N, ph, ctx->pen, ctx->fchunk, ctx->nfchunk, wcs,
                                                ctx->ew, static_cast<T4 *>(ctx->lr));
    return launched(ctx);
}

colatus_status run_ewald_f32(colatus_t ctx, const ForcePlan &p, const float *pk) {
    TRY(ensure_part(ctx, p.part_bytes));
    const float eps2 = (float)(ctx->eps * ctx->eps);
    TRY(run_ewald_phases<float>(ctx, pk, nullptr));
    const float *pkw = ctx->pk_ew;
    TRY(prof_begin(ctx));
    // equal masses and no zero-mass padding: the equal-mass form
    const bool eqm = ctx->eq_mass && p.n_pad == ctx->N;
    float4 *part = static_cast<float4 *>(ctx->part);
    const float me = ctx->mass_eq;
    const bool comp = ctx->prec == COLATUS_FP32_COMP;
    if (p.L.sym) {
        // pair-once real space
        const int smem = comp ? EwSymKC::SMEM : EwSymK::SMEM;
        if (comp && eqm)
            force_sym_f32_kernel<kEwSymNT, kEwSymIPT, true, true, kEwSymUnr, EwaldPair>
                <<<p.L.G, kEwSymNT, smem, ctx->stream>>>(pkw, part, ctx->flags, p.L, eps2, me, ctx->ew);
        else if (comp)
            force_sym_f32_kernel<kEwSymNT, kEwSymIPT, true, false, kEwSymUnr, EwaldPair>
                <<<p.L.G, kEwSymNT, smem, ctx->stream>>>(pkw, part, ctx->flags, p.L, eps2, me, ctx->ew);
        else if (eqm)
            force_sym_f32_kernel<kEwSymNT, kEwSymIPT, false, true, kEwSymUnr, EwaldPair>
                <<<p.L.G, kEwSymNT, smem, ctx->stream>>>(pkw, part, ctx->flags, p.L, eps2, me, ctx->ew);
        else
            force_sym_f32_kernel<kEwSymNT, kEwSymIPT, false, false, kEwSymUnr, EwaldPair>
                <<<p.L.G, kEwSymNT, smem, ctx->stream>>>(pkw, part, ctx->flags, p.L, eps2, me, ctx->ew);
    } else if (ctx->prec == COLATUS_FP32_COMP && eqm)
        ewald_f32_kernel<kEwNT, kEwIPT, kEwJT, kStages, kEwFold, true, kEwMinB, true>
            <<<p.L.G, kEwNT, EwKC::SMEM, ctx->stream>>>(pkw, part, ctx->flags, p.L, eps2, ctx->ew, me);
    else if (ctx->prec == COLATUS_FP32_COMP)
        ewald_f32_kernel<kEwNT, kEwIPT, kEwJT, kStages, kEwFold, true, kEwMinB, false>
            <<<p.L.G, kEwNT, EwKC::SMEM, ctx->stream>>>(pkw, part, ctx->flags, p.L, eps2, ctx->ew, me);
    else if (eqm)
        ewald_f32_kernel<kEwNT, kEwIPT, kEwJT, kStages, kEwFold, false, kEwMinB, true>
            <<<p.L.G, kEwNT, EwK::SMEM, ctx->stream>>>(pkw, part, ctx->flags, p.L, eps2, ctx->ew, me);
    else
        ewald_f32_kernel<kEwNT, kEwIPT, kEwJT, kStages, kEwFold, false, kEwMinB, false>
            <<<p.L.G, kEwNT, EwK::SMEM, ctx->stream>>>(pkw, part, ctx->flags, p.L, eps2, ctx->ew, me);
    TRY(launched(ctx));
    ctx->interactions += (double)ctx->N * (double)ctx->N;
    TRY(prof_end(ctx));
    return run_ewald_kspace<float, float4>(ctx, pk, nullptr);
}

// Launch the force sum on packed FP32 bodies; segments land in ctx->part.
colatus_status run_force_f32(colatus_t ctx, const ForcePlan &p, const float *pk) {
    if (ctx->periodic) return run_ewald_f32(ctx, p, pk);
    TRY(ensure_part(ctx, p.part_bytes));
    const F32Variant &fv = f32_variant(p.variant);
    const float eps2 = (float)(ctx->eps * ctx->eps);
    TRY(prof_begin(ctx));
    fv.launch(p.L.G, ctx->stream, pk, static_cast<float4 *>(ctx->part), ctx->flags, p.L, eps2,
              ctx->mass_eq);
    TRY(launched(ctx));
    ctx->interactions += (double)ctx->N * (double)ctx->N;
    return prof_end(ctx);
}

colatus_status run_force_f64(colatus_t ctx, const double4 *pos) {
    if (ctx->periodic) {
        const ForcePlan &p = ctx->plan_ew64;
        TRY(ensure_part(ctx, p.part_bytes));
        TRY(run_ewald_phases<double>(ctx, nullptr, pos));
        TRY(prof_begin(ctx));
        ewald_f64_kernel<kEw64NT, kEw64JT, kStages><<<p.L.G, kEw64NT, Ew64K::SMEM, ctx->stream>>>(
            pos, static_cast<double4 *>(ctx->part), ctx->flags, p.L, ctx->eps * ctx->eps, ctx->ew);
        TRY(launched(ctx));
        ctx->interactions += (double)ctx->N * (double)ctx->N;
        TRY(prof_end(ctx));
        return run_ewald_kspace<double, double4>(ctx, nullptr, pos);
    }
    const ForcePlan &p = ctx->plan64;
    TRY(ensure_part(ctx, p.part_bytes));
    TRY(prof_begin(ctx));
    force_f64_kernel<kF64NT, kF64IPT, kF64JT, kStages><<<p.L.G, kF64NT, F64K::SMEM, ctx->stream>>>(
        pos, static_cast<double4 *>(ctx->part), ctx->flags, p.L, ctx->eps * ctx->eps);
    TRY(launched(ctx));
    ctx->interactions += (double)ctx->N * (double)ctx->N;
    return prof_end(ctx);
}

// Self-test of the bounded waits: one CTA waits on an mbarrier that nothing
// ever completes, with a short limit, and raises FLAG_TIMEOUT as the
// pipelined kernels do when a wait gives up.  Nothing faults or hangs.
__global__ void wait_selftest_kernel(int *flags, long long limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, limit);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(&flags[FLAG_TIMEOUT], 1);
}

// ---- state conversion kernels (I/O only)
__global__ void load_state_kernel(const void *x, const void *v, int f64, const double *m64,
                                  long long N, float4 *xs, float4 *vs, double4 *xs64,
                                  double4 *vs64, int *bad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double p[3], q[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < 3; ++c) {
        p[c] = f64 ? static_cast<const double *>(x)[3 * i + c] : static_cast<const float *>(x)[3 * i + c];
        if (v) q[c] = f64 ? static_cast<const double *>(v)[3 * i + c]
                          : static_cast<const float *>(v)[3 * i + c];
    }
    const double m = m64[i];
    bool ok = true;
    for (int c = 0; c < 3; ++c) ok = ok && isfinite(p[c]) && isfinite(q[c]);
    if (!ok) atomicOr(bad, 1);
    xs[i] = make_float4((float)p[0], (float)p[1], (float)p[2], (float)m);
    vs[i] = make_float4((float)q[0], (float)q[1], (float)q[2], 0.f);
    xs64[i] = make_double4(p[0], p[1], p[2], m);
    vs64[i] = make_double4(q[0], q[1], q[2], 0.0);
}

__global__ void store_state_kernel(const float4 *xs, const float4 *vs, const double4 *xs64,
                                   const double4 *vs64, int from64, long long N, void *x, void *v,
                                   int f64) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double p[3], q[3];
    if (from64) {
        const double4 a = xs64[i], b = vs64[i];
        p[0] = a.x; p[1] = a.y; p[2] = a.z;
        q[0] = b.x; q[1] = b.y; q[2] = b.z;
    } else {
        const float4 a = xs[i], b = vs[i];
        p[0] = a.x; p[1] = a.y; p[2] = a.z;
        q[0] = b.x; q[1] = b.y; q[2] = b.z;
    }
    for (int c = 0; c < 3; ++c) {
        if (f64) {
            if (x) static_cast<double *>(x)[3 * i + c] = p[c];
            if (v) static_cast<double *>(v)[3 * i + c] = q[c];
        } else {
            if (x) static_cast<float *>(x)[3 * i + c] = (float)p[c];
            if (v) static_cast<float *>(v)[3 * i + c] = (float)q[c];
        }
    }
}

// Copy the state of one precision into the other (precision switch).
__global__ void convert_state_kernel(float4 *xs, float4 *vs, double4 *xs64, double4 *vs64,
                                     int to64, long long N) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (to64) {
        const float4 a = xs[i], b = vs[i];
        xs64[i] = make_double4(a.x, a.y, a.z, xs64[i].w);
        vs64[i] = make_double4(b.x, b.y, b.z, 0.0);
    } else {
        const double4 a = xs64[i], b = vs64[i];
        xs[i] = make_float4((float)a.x, (float)a.y, (float)a.z, xs[i].w);
        vs[i] = make_float4((float)b.x, (float)b.y, (float)b.z, 0.f);
    }
}

// Store the masses and record the extreme float masses (non-negative floats
// order like their bit patterns) to detect the equal-mass case.
__global__ void load_masses_kernel(const void *m, int f64, long long N, double *m64, float4 *xs,
                                   double4 *xs64, int *bad, int *mstat) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double mi = f64 ? static_cast<const double *>(m)[i] : static_cast<const float *>(m)[i];
    if (!isfinite(mi) || mi < 0.0) atomicOr(bad, 1);
    m64[i] = mi;
    xs[i].w = (float)mi;
    xs64[i].w = mi;
    const int bits = __float_as_int((float)mi);
    atomicMin(&mstat[0], bits);
    atomicMax(&mstat[1], bits);
}

colatus_status read_flags(colatus_t ctx, bool clear) {
    int f[NUM_FLAGS];
    CU(cudaMemcpy(f, ctx->flags, sizeof(f), cudaMemcpyDeviceToHost));
    if (clear) CU(cudaMemset(ctx->flags, 0, sizeof(f)));
    if (f[FLAG_TIMEOUT]) return fail(ctx, COLATUS_E_TIMEOUT, "a bounded device wait gave up");
    if (f[FLAG_FRIEDMANN])
        return fail(ctx, COLATUS_E_FRIEDMANN, "H^2 < 0 or a <= 0 while integrating Eq. 2");
    if (f[FLAG_NONFINITE]) return fail(ctx, COLATUS_E_NONFINITE, "non-finite position or velocity");
    return COLATUS_OK;
}

colatus_status sync_and_check(colatus_t ctx) {
    CU(cudaStreamSynchronize(ctx->stream));
    return read_flags(ctx, true);
}

size_t elem_size(int dtype) { return dtype == COLATUS_F64 ? 8 : 4; }

// Both kick-drift-kick schemes share every kernel; only the schedule differs.
bool is_kdk(colatus_t ctx) { return ctx->scheme != COLATUS_DKD; }
int canonical(colatus_t ctx) { return ctx->scheme == COLATUS_KDK_CANONICAL ? 1 : 0; }

// Deformation term for the kernels: the G-less kappa = C psi / G.
Extra extra_args(colatus_t ctx) {
    Extra D{};
    D.on = ctx->defo_C != 0.0 && ctx->G != 0.0;
    D.kappa = D.on ? ctx->defo_C / ctx->G : 0.0;
    D.x = ctx->defo_x[0];
    D.y = ctx->defo_x[1];
    D.z = ctx->defo_x[2];
    D.eps2 = ctx->eps * ctx->eps;
    D.lr32 = ctx->periodic && ctx->prec != COLATUS_FP64 ? static_cast<const float4 *>(ctx->lr) : nullptr;
    D.lr64 = ctx->periodic && ctx->prec == COLATUS_FP64 ? static_cast<const double4 *>(ctx->lr) : nullptr;
    return D;
}

colatus_status check_dtype(colatus_t ctx, int dtype) {
    if (dtype != COLATUS_F32 && dtype != COLATUS_F64) return fail(ctx, COLATUS_E_ARG, "bad dtype %d", dtype);
    return COLATUS_OK;
}

void free_all(colatus_t ctx) {
    void *ptrs[] = {ctx->xs, ctx->vs, ctx->vh, ctx->acc, ctx->pk[0], ctx->pk[1], ctx->pk[2],
                    ctx->xs64, ctx->vs64, ctx->vh64, ctx->acc64, ctx->pos64[0], ctx->pos64[1],
                    ctx->pos64[2], ctx->m64, ctx->part, ctx->flags, ctx->sym_tab, ctx->mstat, ctx->clk,
                    ctx->tclk, ctx->table, ctx->stage, ctx->stage2, ctx->diag, ctx->tslot,
                    ctx->rec, ctx->kw, ctx->rho, ctx->rho_part, ctx->wcs, ctx->pen,
                    ctx->rchunk, ctx->fchunk, ctx->lr, ctx->ph, ctx->pot_part, ctx->lrv,
                    ctx->kwr, ctx->kwl, ctx->pk_ew, ctx->vjp_sym_tab, ctx->ew_sym_tab, ctx->vjp_gen_tab,
                    ctx->ewvjp_sym_tab};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    void *tptrs[] = {ctx->tan.dx, ctx->tan.dv, ctx->tan.dvh, ctx->tan.dxp, ctx->tan.pkt,
                     ctx->tan.seeds, ctx->tan.growth, ctx->tan.lrt};
    for (void *p : tptrs)
        if (p) cudaFree(p);
    void *aptrs[] = {ctx->adj.ck_x, ctx->adj.ck_v, ctx->adj.seg_x, ctx->adj.table, ctx->adj.rclk,
                     ctx->adj.rvs, ctx->adj.rvh, ctx->adj.racc, ctx->adj.rpk[0], ctx->adj.rpk[1],
                     ctx->adj.lx, ctx->adj.lv, ctx->adj.lvh, ctx->adj.lm, ctx->adj.pkw,
                     ctx->adj.seg_f, ctx->adj.seg_v};
    for (void *p : aptrs)
        if (p) cudaFree(p);
    if (ctx->cstream) cudaStreamSynchronize(ctx->cstream);
    for (auto &r : ctx->rslot) {
        if (r.x) cudaFree(r.x);
        if (r.v) cudaFree(r.v);
        if (r.snap) cudaEventDestroy(r.snap);
        if (r.done) cudaEventDestroy(r.done);
    }
    if (ctx->cstream) cudaStreamDestroy(ctx->cstream);
    for (cudaEvent_t e : ctx->tab_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->adj.tab_ev) cudaEventDestroy(ctx->adj.tab_ev);
    if (ctx->main_ev) cudaEventDestroy(ctx->main_ev);
    if (ctx->tstream) cudaStreamDestroy(ctx->tstream);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    ctx->ev_pool.clear();
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
}

// Load masses (device pointer src) and refresh the equal-mass flag.
colatus_status load_masses(colatus_t ctx, const void *src, int f64) {
    const int init[2] = {0x7fffffff, 0};
    CU(cudaMemcpyAsync(ctx->mstat, init, sizeof(init), cudaMemcpyHostToDevice, ctx->stream));
    load_masses_kernel<<<blocks_for(ctx->N, 256), 256, 0, ctx->stream>>>(
        src, f64, ctx->N, ctx->m64, ctx->xs, ctx->xs64, ctx->flags, ctx->mstat);
    TRY(launched(ctx));
    int st[2];
    CU(cudaMemcpyAsync(st, ctx->mstat, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->eq_mass = st[0] == st[1];
    float me;
    std::memcpy(&me, &st[0], sizeof(me));
    ctx->mass_eq = me;
    return COLATUS_OK;
}

// Extend the look-ahead schedule by n entries on the schedule stream, in
// launches of kTabPiece entries, each followed by an event that records how
// far the schedule then reaches; steps wait only for the piece they need.
colatus_status extend_table(colatus_t ctx, int n) {
    for (int done = 0; done < n; done += kTabPiece) {
        const int m = std::min(kTabPiece, n - done);
        friedmann_table_kernel<<<1, 1, ctx->tab_smem, ctx->tstream>>>(
            ctx->cosmo, ctx->tclk, ctx->table, kTabCap, m, ctx->tab_tau, ctx->tab_G, kFriedmannSub,
            canonical(ctx));
        TRY(launched(ctx));
        ctx->tab_hi += m;
        const int k = ctx->tab_ev_next;
        ctx->tab_ev_next = (k + 1) % kTabEvents;
        CU(cudaEventRecord(ctx->tab_ev[k], ctx->tstream));
        ctx->tab_ev_covers[k] = ctx->tab_hi;
    }
    return COLATUS_OK;
}

// Make the main stream wait until the schedule holds the entries below
// `need` (the earliest extension piece that reaches it).
colatus_status wait_table(colatus_t ctx, long long need) {
    int best = -1;
    for (int k = 0; k < kTabEvents; ++k)
        if (ctx->tab_ev_covers[k] >= need &&
            (best < 0 || ctx->tab_ev_covers[k] < ctx->tab_ev_covers[best]))
            best = k;
    if (best < 0) return fail(ctx, COLATUS_E_STATE, "schedule bookkeeping lost its extension");
    CU(cudaStreamWaitEvent(ctx->stream, ctx->tab_ev[best], 0));
    return COLATUS_OK;
}

// Make schedule entries [host_step, host_step + n] available for step size
// tau: extend the schedule to cover them (plus the look-ahead), and make the
// main stream wait for the first `first` steps' entries only; a caller that
// passes first < n waits for the rest with wait_table as it goes.  The
// schedule stream first waits for all work already enqueued on the main
// stream, so an extension never overwrites ring entries that enqueued steps
// still read (the ring holds kTabCap entries and at most kChunk +
// 4 kLookahead are live).
colatus_status need_table(colatus_t ctx, double tau, int n, int first) {
    CU(cudaEventRecord(ctx->main_ev, ctx->stream));
    CU(cudaStreamWaitEvent(ctx->tstream, ctx->main_ev, 0));
    if (!ctx->tab_valid || ctx->tab_tau != tau || ctx->tab_G != ctx->G) {
        clock_copy_kernel<<<1, 1, 0, ctx->tstream>>>(ctx->clk, ctx->tclk);
        TRY(launched(ctx));
        ctx->tab_valid = true;
        ctx->tab_tau = tau;
        ctx->tab_G = ctx->G;
        ctx->tab_hi = ctx->host_step;
        for (long long &c : ctx->tab_ev_covers) c = -1;
    }
    // steps [host_step, host_step + n) and the entry after them, whose
    // opening coefficients the last step's epilogue applies
    const long long need = ctx->host_step + n + 1;
    if (ctx->tab_hi < need) TRY(extend_table(ctx, (int)(need + kLookahead - ctx->tab_hi)));
    return wait_table(ctx, ctx->host_step + std::min(first, n) + 1);
}

// Before step j of a chunk of n steps enqueued after need_table(.., n,
// kTabPiece): every kTabPiece steps, wait for the next piece's entries.
colatus_status wait_table_at(colatus_t ctx, int j, int n) {
    if (j == 0 || j % kTabPiece != 0) return COLATUS_OK;
    return wait_table(ctx, ctx->host_step + std::min(j + kTabPiece, n) + 1);
}

// After enqueuing steps: keep kLookahead entries ahead, computed on the
// schedule stream while the main stream runs the force kernels.
colatus_status refill_table(colatus_t ctx) {
    if (ctx->tab_hi < ctx->host_step + kLookahead) {
        CU(cudaEventRecord(ctx->main_ev, ctx->stream));
        CU(cudaStreamWaitEvent(ctx->tstream, ctx->main_ev, 0));
        TRY(extend_table(ctx, (int)(ctx->host_step + 2 * kLookahead - ctx->tab_hi)));
    }
    return COLATUS_OK;
}

// Pack the state for a force evaluation at the state position into the aux
// buffer and run the force sum (segments in ctx->part).
colatus_status force_at_state(colatus_t ctx) {
    if (ctx->prec == COLATUS_FP64) {
        const ForcePlan &p = plan_f64(ctx);
        pack_f64_kernel<<<blocks_for(p.n_pad, 256), 256, 0, ctx->stream>>>(ctx->xs64, ctx->pos64[2],
                                                                           ctx->N, p.n_pad);
        TRY(launched(ctx));
        return run_force_f64(ctx, ctx->pos64[2]);
    }
    const ForcePlan &p = plan_f32(ctx);
    pack_f32_kernel<<<blocks_for(p.n_pad, 256), 256, 0, ctx->stream>>>(ctx->xs, ctx->pk[2], ctx->N,
                                                                       p.n_pad);
    TRY(launched(ctx));
    return run_force_f32(ctx, p, ctx->pk[2]);
}

// forces_out_f32_kernel for plan p (its pair-once or ordered-pair sums).
template <bool COMP>
void launch_forces_out_f32(colatus_t ctx, const ForcePlan &p, void *out, int out_f64, float4 *acc,
                           const float *pk) {
    const float4 *part = static_cast<const float4 *>(ctx->part);
    if (p.L.sym)
        forces_out_f32_kernel<COMP, true><<<blocks_for(ctx->N, 256), 256, 0, ctx->stream>>>(
            part, p.L, p.itile, ctx->N, ctx->clk, ctx->G, out, out_f64, acc, pk, extra_args(ctx));
    else
        forces_out_f32_kernel<COMP, false><<<blocks_for(ctx->N, 256), 256, 0, ctx->stream>>>(
            part, p.L, p.itile, ctx->N, ctx->clk, ctx->G, out, out_f64, acc, pk, extra_args(ctx));
}

// Reduce the segments of the last force sum into acc and/or out.
colatus_status force_output(colatus_t ctx, void *out, int out_f64, bool to_acc) {
    if (ctx->prec == COLATUS_FP64) {
        const ForcePlan &p = plan_f64(ctx);
        forces_out_f64_kernel<<<blocks_for(ctx->N, 256), 256, 0, ctx->stream>>>(
            static_cast<const double4 *>(ctx->part), p.L, p.itile, ctx->N, ctx->clk, ctx->G, out,
            out_f64, to_acc ? ctx->acc64 : nullptr, ctx->pos64[2], extra_args(ctx));
        return launched(ctx);
    }
    const ForcePlan &p = plan_f32(ctx);
    if (ctx->prec == COLATUS_FP32_COMP)
        launch_forces_out_f32<true>(ctx, p, out, out_f64, to_acc ? ctx->acc : nullptr, ctx->pk[2]);
    else
        launch_forces_out_f32<false>(ctx, p, out, out_f64, to_acc ? ctx->acc : nullptr, ctx->pk[2]);
    return launched(ctx);
}

Tracers tracer_args(colatus_t ctx) {
    Tracers t;
    t.slot = ctx->tslot;
    t.rec = ctx->rec;
    t.cap = ctx->rec_cap > 0 ? ctx->rec_cap : 1;
    t.base = ctx->rec_base;
    t.ntr = ctx->ntr;
    return t;
}

// Explicit buffers of one KDK/DKD trajectory: the context's own, or the
// scratch of an adjoint recomputation.
struct StepBufs {
    float4 *xs, *vs, *vh, *acc;
    float *pk[2];
    double4 *xs64, *vs64, *vh64, *acc64;
    double4 *pos64[2];
    const StepCoef *table;
    int tcap;
    DevClock *clk;
    Tracers tr;
};

StepBufs ctx_bufs(colatus_t ctx) {
    StepBufs b;
    b.xs = ctx->xs; b.vs = ctx->vs; b.vh = ctx->vh; b.acc = ctx->acc;
    b.pk[0] = ctx->pk[0]; b.pk[1] = ctx->pk[1];
    b.xs64 = ctx->xs64; b.vs64 = ctx->vs64; b.vh64 = ctx->vh64; b.acc64 = ctx->acc64;
    b.pos64[0] = ctx->pos64[0]; b.pos64[1] = ctx->pos64[1];
    b.table = ctx->table;
    b.tcap = kTabCap;
    b.clk = ctx->clk;
    b.tr = tracer_args(ctx);
    return b;
}

// KDK opening (half kick + drift) from (xs, vs) with F = acc into pk[c].
colatus_status launch_kdk_open(colatus_t ctx, const StepBufs &b, int c, long long step, double tau) {
    if (ctx->prec == COLATUS_FP64) {
        const ForcePlan &p = plan_f64(ctx);
        kdk_open_f64_kernel<<<blocks_for(p.n_pad, 256), 256, 0, ctx->stream>>>(
            b.xs64, b.vs64, b.acc64, b.vh64, b.pos64[c], b.table, b.tcap, step, tau, ctx->N, p.n_pad);
    } else {
        const ForcePlan &p = plan_f32(ctx);
        kdk_open_f32_kernel<<<blocks_for(p.n_pad, 256), 256, 0, ctx->stream>>>(
            b.xs, b.vs, b.acc, b.vh, b.pk[c], b.table, b.tcap, step, tau, ctx->N, p.n_pad);
    }
    return launched(ctx);
}

// The FP32 step epilogue of plan p (SYM: its pair-once sums).
template <bool COMP, bool SYM>
void launch_step_f32(colatus_t ctx, const ForcePlan &p, const StepBufs &b, int c, long long step, double tau,
                     const Extra &D) {
    const int n = c ^ 1;
    const float4 *part = static_cast<const float4 *>(ctx->part);
    const unsigned nb = blocks_for(p.n_pad, kEpiThreads);
    if (is_kdk(ctx))
        kdk_step_f32_kernel<COMP, SYM><<<nb, kEpiThreads, 0, ctx->stream>>>(
            part, p.L, p.itile, b.pk[c], b.xs, b.vs, b.vh, b.acc, b.pk[n], b.table, b.tcap, step, tau, ctx->N,
            p.n_pad, b.tr, ctx->flags, b.clk, D);
    else
        dkd_step_f32_kernel<COMP, SYM><<<nb, kEpiThreads, 0, ctx->stream>>>(
            part, p.L, p.itile, b.pk[c], b.xs, b.vs, b.acc, b.pk[n], b.table, b.tcap, step, tau, ctx->N, p.n_pad,
            b.tr, ctx->flags, b.clk, D);
}

// One step: force on pk[c], then the fused epilogue that writes the state
// (xs, vs), the next force input pk[c ^ 1] and, for KDK, vh and acc.
colatus_status launch_step(colatus_t ctx, const StepBufs &b, int c, long long step, double tau) {
    const int n = c ^ 1;
    const Tracers &tr = b.tr;
    const Extra D = extra_args(ctx);
    if (ctx->prec == COLATUS_FP64) {
        const ForcePlan &p = plan_f64(ctx);
        TRY(run_force_f64(ctx, b.pos64[c]));
        const double4 *part = static_cast<const double4 *>(ctx->part);
        if (is_kdk(ctx))
            kdk_step_f64_kernel<<<blocks_for(p.n_pad, 256), 256, 0, ctx->stream>>>(
                part, p.L, p.itile, b.pos64[c], b.xs64, b.vs64, b.vh64, b.acc64, b.pos64[n], b.table,
                b.tcap, step, tau, ctx->N, p.n_pad, tr, ctx->flags, b.clk, D);
        else
            dkd_step_f64_kernel<<<blocks_for(p.n_pad, 256), 256, 0, ctx->stream>>>(
                part, p.L, p.itile, b.pos64[c], b.xs64, b.vs64, b.acc64, b.pos64[n], b.table, b.tcap,
                step, tau, ctx->N, p.n_pad, tr, ctx->flags, b.clk, D);
    } else {
        const ForcePlan &p = plan_f32(ctx);
        TRY(run_force_f32(ctx, p, b.pk[c]));
        const bool comp = ctx->prec == COLATUS_FP32_COMP;
        if (p.L.sym) {
            if (comp)
                launch_step_f32<true, true>(ctx, p, b, c, step, tau, D);
            else
                launch_step_f32<false, true>(ctx, p, b, c, step, tau, D);
        } else {
            if (comp)
                launch_step_f32<true, false>(ctx, p, b, c, step, tau, D);
            else
                launch_step_f32<false, false>(ctx, p, b, c, step, tau, D);
        }
    }
    return launched(ctx);
}

// Opening of the first step of a call: the KDK half kick + drift, or the
// DKD half drift, from the state into the force input pk[cur].
colatus_status open_step(colatus_t ctx, double tau) {
    const bool f64 = ctx->prec == COLATUS_FP64;
    if (is_kdk(ctx)) {
        if (!ctx->acc_valid) {
            TRY(force_at_state(ctx));
            TRY(force_output(ctx, nullptr, 0, true));
            ctx->acc_valid = true;
        }
        return launch_kdk_open(ctx, ctx_bufs(ctx), ctx->cur, ctx->host_step, tau);
    }
    if (f64) {
        const ForcePlan &p = plan_f64(ctx);
        dkd_open_f64_kernel<<<blocks_for(p.n_pad, 256), 256, 0, ctx->stream>>>(
            ctx->xs64, ctx->vs64, ctx->pos64[ctx->cur], tau, ctx->N, p.n_pad);
    } else {
        const ForcePlan &p = plan_f32(ctx);
        dkd_open_f32_kernel<<<blocks_for(p.n_pad, 256), 256, 0, ctx->stream>>>(
            ctx->xs, ctx->vs, ctx->pk[ctx->cur], tau, ctx->N, p.n_pad);
    }
    return launched(ctx);
}

// One step j of the current chunk on the context's own buffers.
colatus_status one_step(colatus_t ctx, int j, double tau) {
    TRY(launch_step(ctx, ctx_bufs(ctx), ctx->cur, ctx->host_step + j, tau));
    ctx->cur ^= 1;
    return COLATUS_OK;
}


// ------------------------------------------------------------------ adjoint
// Allocate the fixed-size adjoint buffers (first use only).
colatus_status adj_alloc(colatus_t ctx) {
    auto &a = ctx->adj;
    if (a.pkw) return COLATUS_OK;
    const size_t na = (size_t)ctx->n_alloc;
    void **bufs32[] = {&a.rvs, &a.rvh, &a.racc, &a.rpk[0], &a.rpk[1], &a.lx, &a.lv, &a.lvh};
    for (void **b : bufs32) CU(cudaMalloc(b, na * 32));
    CU(cudaMalloc(&a.lm, na * 8));
    CU(cudaMalloc(&a.rclk, sizeof(DevClock)));
    CU(cudaMalloc(&a.pkw, na * 64));
    CU(cudaEventCreateWithFlags(&a.tab_ev, cudaEventDisableTiming));
    return COLATUS_OK;
}

colatus_status grow(colatus_t ctx, void **p, size_t *have, size_t need) {
    if (need <= *have) return COLATUS_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *have = 0;
    CU(cudaMalloc(p, need));
    *have = need;
    return COLATUS_OK;
}

// The VJP's launch plan: the periodic kernel's when the boundaries are periodic
// (in FP32 the pair-once one where it fits, under tuning shape 3 or the
// built-in choice, as the periodic force); in FP32 the pair-once kernels'
// where they fit (same padding as the per-ordered-pair VJP): the equal-mass
// one for eqm (the KDK adjoint's), the one for any masses otherwise.
const ForcePlan &vjp_plan(colatus_t ctx, bool eqm = false) {
    const bool f64 = ctx->prec == COLATUS_FP64;
    if (ctx->periodic && f64) return ctx->plan_ewvjp64;
    if (ctx->periodic) {
        const ForcePlan &q = ctx->plan_ewvjp_sym;
        const bool sym = q.fits && (ctx->tuned_shape < 0 || ctx->tuned_shape == kSymShape);
        return sym ? q : ctx->plan_ewvjp32;
    }
    if (f64) return ctx->plan_vjp64;
    if (eqm && ctx->plan_vjp_sym.fits) return ctx->plan_vjp_sym;
    if (!eqm && ctx->plan_vjp_gen.fits) return ctx->plan_vjp_gen;
    return ctx->plan_vjp32;
}

// Per-body terms of the VJP consumers: the deformation term and, with
// periodic boundaries, the reciprocal-space VJP (lrv).
Extra vjp_extra(colatus_t ctx) {
    Extra D = extra_args(ctx);
    D.lr32 = ctx->periodic && ctx->prec != COLATUS_FP64 ? static_cast<const float4 *>(ctx->lrv) : nullptr;
    D.lr64 = ctx->periodic && ctx->prec == COLATUS_FP64 ? static_cast<const double4 *>(ctx->lrv) : nullptr;
    return D;
}

// The per-k weights of the reciprocal-space VJP and JVP (kwr, kwl).
colatus_status kweight_bufs(colatus_t ctx) {
    if (ctx->kwrl_cap >= (size_t)ctx->nkv) return COLATUS_OK;
    if (ctx->kwr) cudaFree(ctx->kwr);
    if (ctx->kwl) cudaFree(ctx->kwl);
    ctx->kwr = ctx->kwl = nullptr;
    ctx->kwrl_cap = 0;
    CU(cudaMalloc(&ctx->kwr, ctx->nkv * sizeof(double2)));
    CU(cudaMalloc(&ctx->kwl, (size_t)kTB * ctx->nkv * sizeof(double2)));   // a plane per tangent
    ctx->kwrl_cap = ctx->nkv;
    return COLATUS_OK;
}

// Splits of the bodies in the structure-factor passes: enough blocks to
// fill the GPU, at least ew_bodies<T>() bodies per split.
template <typename T>
int ew_splits(colatus_t ctx) {
    const long long max_split = std::max(1LL, ctx->N / ew_bodies<T>());
    return (int)std::min<long long>(std::max(1, kEwRhoBlocksPerSM * ctx->num_sms / ctx->nrchunk), max_split);
}

// Reciprocal-space VJP of the bodies and co-vectors packed in adj.pkw, into
// lrv: phase tables of the packed positions, one pass for the structure
// factors weighted by m, w_x, w_y, w_z, their weights per k, then one pass
// per body.
template <typename T, typename T4>
colatus_status run_ewald_kspace_vjp(colatus_t ctx) {
    using T2 = typename Vec2<T>::type;
    const bool f64 = sizeof(T) == 8;
    if (!ctx->lrv) CU(cudaMalloc(&ctx->lrv, (size_t)ctx->n_alloc * sizeof(double4)));
    TRY(kweight_bufs(ctx));
    ChanSrc C{};
    C.src = BodySrc{f64 ? nullptr : static_cast<const float *>(ctx->adj.pkw),
                    f64 ? static_cast<const double4 *>(ctx->adj.pkw) : nullptr, f64 ? 2 : 16, f64 ? 3 : 6};
    C.mode = 0;
    const int widx[4] = {f64 ? 3 : 6, f64 ? 4 : 8, f64 ? 5 : 10, f64 ? 6 : 12};
    for (int c = 0; c < 4; ++c) C.widx[c] = widx[c];
    T2 *ph = static_cast<T2 *>(ctx->ph);
    ewald_phase_kernel<T><<<blocks_for(3 * ctx->N, 128), 128, 0, ctx->stream>>>(C.src, ctx->N, ctx->ew,
                                                                                ph, nullptr);
    TRY(launched(ctx));
    const int splits = ew_splits<T>(ctx);
    const size_t plane = (size_t)splits * ctx->nkv;
    TRY(grow(ctx, &ctx->rho_part, &ctx->rho_part_bytes, 4 * plane * sizeof(double2)));
    double2 *rp = static_cast<double2 *>(ctx->rho_part);
    ewald_rho_multi_kernel<T, 4><<<dim3(ctx->nrchunk, splits), kEwKThreads,
                                   ew_rho_multi_smem<T, 4>(ctx->ew.nk, ctx->rchunk_np), ctx->stream>>>(
        C, ctx->N, ph, ctx->pen, ctx->rchunk, ctx->rchunk_np, ctx->nkv, ctx->ew, rp);
    TRY(launched(ctx));
    ewald_vjp_weights_kernel<T><<<blocks_for(ctx->nkv, 128), 128, 0, ctx->stream>>>(
        rp, rp + plane, splits, ctx->nkv, ctx->kw, ctx->pen, ctx->npen, 2.0 * std::acos(-1.0) / ctx->ew.L,
        static_cast<T2 *>(ctx->kwr), static_cast<T2 *>(ctx->kwl));
    TRY(launched(ctx));
    ewald_kvjp_kernel<T, T4, 1><<<blocks_for(ctx->N, kEwFThreads), kEwFThreads * kEwFSlices,
                                  ew_kvjp_smem<T, 1>(ctx->ew.nk), ctx->stream>>>(
        ctx->N, ph, ctx->pen, ctx->npen, ctx->nkv, static_cast<const T2 *>(ctx->kwr),
        static_cast<const T2 *>(ctx->kwl), C.src, nullptr, 0, 1, ctx->ew, static_cast<T4 *>(ctx->lrv), 0);
    return launched(ctx);
}

// One VJP launch on the packed bodies + co-vectors in adj.pkw (with periodic
// boundaries: the real-space kernel, then the reciprocal-space VJP; eqm: the
// equal-mass FP32 kernel, whose consumers need the forces at the positions).
colatus_status run_vjp(colatus_t ctx, bool eqm = false) {
    const bool f64 = ctx->prec == COLATUS_FP64;
    const ForcePlan &p = vjp_plan(ctx, eqm);
    TRY(ensure_part(ctx, p.part_bytes));
    TRY(prof_begin(ctx));
    if (ctx->periodic && f64)
        ewald_vjp_f64_kernel<kEwV64NT, kEwV64JT, kStages><<<p.L.G, kEwV64NT, EwVjp64K::SMEM, ctx->stream>>>(
            static_cast<const double4 *>(ctx->adj.pkw), static_cast<double4 *>(ctx->part), ctx->flags,
            p.L, ctx->eps * ctx->eps, ctx->ew);
    else if (ctx->periodic && p.L.sym && ctx->eq_mass && p.n_pad == ctx->N)
        vjp_sym_f32_kernel<kVjpGenNT, kEwVjpSymUnr, true, EwaldVjpPair>
            <<<p.L.G, kVjpGenNT, VjpGenK::SMEM, ctx->stream>>>(
                static_cast<const float *>(ctx->adj.pkw), static_cast<float4 *>(ctx->part), ctx->flags, p.L,
                (float)(ctx->eps * ctx->eps), ctx->mass_eq, ctx->ew);
    else if (ctx->periodic && p.L.sym)
        vjp_sym_f32_kernel<kVjpGenNT, kEwVjpSymUnr, false, EwaldVjpPair>
            <<<p.L.G, kVjpGenNT, VjpGenK::SMEM, ctx->stream>>>(
                static_cast<const float *>(ctx->adj.pkw), static_cast<float4 *>(ctx->part), ctx->flags, p.L,
                (float)(ctx->eps * ctx->eps), 1.f, ctx->ew);
    else if (ctx->periodic)
        ewald_vjp_f32_kernel<kEwVjpNT, kEwVjpIPT, kEwVjpJT, kStages, kEwVjpMinB>
            <<<p.L.G, kEwVjpNT, EwVjpK::SMEM, ctx->stream>>>(
                static_cast<const float *>(ctx->adj.pkw), static_cast<float4 *>(ctx->part), ctx->flags,
                p.L, (float)(ctx->eps * ctx->eps), ctx->ew);
    else if (eqm && p.L.sym)
        vjp_sym_eqm_f32_kernel<kVjpSymNT, kVjpSymUnr><<<p.L.G, kVjpSymNT, VjpSymK::SMEM, ctx->stream>>>(
            static_cast<const float *>(ctx->adj.pkw), static_cast<float4 *>(ctx->part), ctx->flags, p.L,
            (float)(ctx->eps * ctx->eps), ctx->mass_eq);
    else if (eqm)
        vjp_eqm_f32_kernel<kVjpNT, kVjpJT, kStages, kVjpMINB, kVjpUnr>
            <<<p.L.G, kVjpNT, VjpK::SMEM, ctx->stream>>>(
                static_cast<const float *>(ctx->adj.pkw), static_cast<float4 *>(ctx->part),
                ctx->flags, p.L, (float)(ctx->eps * ctx->eps));
    else if (p.L.sym && ctx->eq_mass && p.n_pad == ctx->N)
        vjp_sym_f32_kernel<kVjpGenNT, kVjpGenUnr, true><<<p.L.G, kVjpGenNT, VjpGenK::SMEM, ctx->stream>>>(
            static_cast<const float *>(ctx->adj.pkw), static_cast<float4 *>(ctx->part), ctx->flags, p.L,
            (float)(ctx->eps * ctx->eps), ctx->mass_eq, PlummerVjpPair::Args{});
    else if (p.L.sym)
        vjp_sym_f32_kernel<kVjpGenNT, kVjpGenUnr, false><<<p.L.G, kVjpGenNT, VjpGenK::SMEM, ctx->stream>>>(
            static_cast<const float *>(ctx->adj.pkw), static_cast<float4 *>(ctx->part), ctx->flags, p.L,
            (float)(ctx->eps * ctx->eps), 1.f, PlummerVjpPair::Args{});
    else if (f64)
        vjp_f64_kernel<kV64NT, kV64JT, kStages><<<p.L.G, kV64NT, Vjp64K::SMEM, ctx->stream>>>(
            static_cast<const double4 *>(ctx->adj.pkw), static_cast<double4 *>(ctx->part),
            ctx->flags, p.L, ctx->eps * ctx->eps);
    else
        vjp_f32_kernel<kVjpNT, kVjpIPT, kVjpJT, kStages, kVjpMINB, kVjpUnr>
            <<<p.L.G, kVjpNT, VjpK::SMEM, ctx->stream>>>(
                static_cast<const float *>(ctx->adj.pkw), static_cast<float4 *>(ctx->part),
                ctx->flags, p.L, (float)(ctx->eps * ctx->eps));
    TRY(launched(ctx));
    ctx->interactions += (double)ctx->N * (double)ctx->N;
    TRY(prof_end(ctx, 1));
    if (!ctx->periodic) return COLATUS_OK;
    return f64 ? run_ewald_kspace_vjp<double, double4>(ctx) : run_ewald_kspace_vjp<float, float4>(ctx);
}

// N x 3 vectors (dtype, device) -> float4 / double4 per body.
template <typename T4, typename T>
__global__ void vec3_to4_kernel(const void *src, int f64, long long N, T4 *dst) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N) return;
    dst[i] = load3<T4, T>(src, f64, i);
}


// ------------------------------------------------------------------ tangent
TangentState tan_state(colatus_t ctx) {
    auto &t = ctx->tan;
    TangentState T;
    T.dx = t.dx;
    T.dv = t.dv;
    T.dvh = t.dvh;
    T.dxp = ctx->periodic ? t.dxp : nullptr;
    T.pkt = t.pkt;
    T.seeds = t.seeds;
    T.growth = t.growth;
    T.cap = t.cap;
    T.base = t.base;
    T.B = t.B;
    T.nchunk = t.nchunk;
    return T;
}

// Reciprocal-space JVP of every tangent at the positions in pk, into
// tan.lrt[b]: phase tables and the mass structure factors once, then per
// chunk of kTB tangents one pass for the structure factors weighted by
// m_j dx_j (3 kTB channels), their per-k weights (a plane per tangent), and
// one pass per body for the chunk (m_i -> 1, w_i -> dx_i).
colatus_status run_ewald_kspace_jvp(colatus_t ctx, const float *pk) {
    auto &t = ctx->tan;
    if (!t.lrt) CU(cudaMalloc(&t.lrt, (size_t)t.B * t.n_pad * sizeof(float4)));
    TRY(kweight_bufs(ctx));
    ChanSrc C{};
    C.src = masses_of(pk, nullptr);
    C.mode = 0;
    C.widx[0] = 6;
    C.tdx = t.dxp;   // the tangent positions of this JVP (tan_pack_kernel)
    C.n_pad = t.n_pad;
    C.B = t.B;
    float2 *ph = static_cast<float2 *>(ctx->ph);
    ewald_phase_kernel<float><<<blocks_for(3 * ctx->N, 128), 128, 0, ctx->stream>>>(C.src, ctx->N, ctx->ew,
                                                                                   ph, nullptr);
    TRY(launched(ctx));
    const int splits = ew_splits<float>(ctx);
    const size_t plane = (size_t)splits * ctx->nkv;
    TRY(grow(ctx, &ctx->rho_part, &ctx->rho_part_bytes, (1 + 3 * kTB) * plane * sizeof(double2)));
    double2 *rp = static_cast<double2 *>(ctx->rho_part);
    const dim3 grid(ctx->nrchunk, splits);
    ewald_rho_multi_kernel<float, 1><<<grid, kEwKThreads, ew_rho_multi_smem<float, 1>(ctx->ew.nk, ctx->rchunk_np),
                                       ctx->stream>>>(C, ctx->N, ph, ctx->pen, ctx->rchunk, ctx->rchunk_np,
                                                      ctx->nkv, ctx->ew, rp);
    TRY(launched(ctx));
    const double tpl = 2.0 * std::acos(-1.0) / ctx->ew.L;
    float2 *wr = static_cast<float2 *>(ctx->kwr), *wl = static_cast<float2 *>(ctx->kwl);
    C.mode = 1;
    for (int b0 = 0; b0 < t.B; b0 += kTB) {
        C.b0 = b0;
        ewald_rho_multi_kernel<float, 3 * kTB>
            <<<grid, kEwKThreads, ew_rho_multi_smem<float, 3 * kTB>(ctx->ew.nk, ctx->rchunk_np), ctx->stream>>>(
                C, ctx->N, ph, ctx->pen, ctx->rchunk, ctx->rchunk_np, ctx->nkv, ctx->ew, rp + plane);
        TRY(launched(ctx));
        const int ntan = std::min(kTB, t.B - b0);
        for (int q = 0; q < ntan; ++q) {
            ewald_vjp_weights_kernel<float><<<blocks_for(ctx->nkv, 128), 128, 0, ctx->stream>>>(
                rp, rp + (1 + 3 * q) * plane, splits, ctx->nkv, ctx->kw, ctx->pen, ctx->npen, tpl, wr,
                wl + (size_t)q * ctx->nkv);
            TRY(launched(ctx));
        }
        ewald_kvjp_kernel<float, float4, kTB><<<blocks_for(ctx->N, kEwFThreads), kEwFThreads * kEwFSlices,
                                                ew_kvjp_smem<float, kTB>(ctx->ew.nk), ctx->stream>>>(
            ctx->N, ph, ctx->pen, ctx->npen, ctx->nkv, wr, wl, C.src, t.dxp + (size_t)b0 * t.n_pad, t.n_pad,
            ntan, ctx->ew, t.lrt + (size_t)b0 * t.n_pad, t.n_pad);
        TRY(launched(ctx));
    }
    return COLATUS_OK;
}

// Pack positions (pair-interleaved pk) with the tangents and run the JVP.
// JVP of every tangent at the positions pk, the tangent positions formed
// from the tangent state as `mode` says (TanDrift, drift time t_drift).
colatus_status run_jvp(colatus_t ctx, const float *pk, int mode, float t_drift) {
    auto &t = ctx->tan;
    // periodic: the reciprocal-space JVP reads the tangent positions as float4
    if (ctx->periodic && !t.dxp) CU(cudaMalloc(&t.dxp, (size_t)t.B * t.n_pad * sizeof(float4)));
    const TangentState T = tan_state(ctx);
    dim3 grid(blocks_for(t.n_pad, 256), t.nchunk);
    tan_pack_kernel<<<grid, 256, 0, ctx->stream>>>(pk, T, ctx->N, t.n_pad, mode, t_drift);
    TRY(launched(ctx));
    TRY(ensure_part(ctx, t.plan.part_bytes));
    if (ctx->periodic)
        ewald_jvp_f32x2_kernel<kJvpNT, kJvpIPT, kJvpJT, kStages, kEwJvpMinB>
            <<<t.plan.L.G, kJvpNT, JvpK::SMEM, ctx->stream>>>(t.pkt, static_cast<float4 *>(ctx->part),
                                                              ctx->flags, t.plan.L, t.n_pad,
                                                              (float)(ctx->eps * ctx->eps), ctx->ew);
    else
        jvp_f32x2_kernel<kJvpNT, kJvpIPT, kJvpJT, kStages, kJvpMINB, kJvpUnr>
            <<<t.plan.L.G, kJvpNT, JvpK::SMEM, ctx->stream>>>(t.pkt, static_cast<float4 *>(ctx->part),
                                                              ctx->flags, t.plan.L, t.n_pad,
                                                              (float)(ctx->eps * ctx->eps));
    TRY(launched(ctx));
    ctx->interactions += (double)ctx->N * (double)ctx->N * t.B;
    return ctx->periodic ? run_ewald_kspace_jvp(ctx, pk) : COLATUS_OK;
}

// Per-body terms of the tangent epilogues: the deformation term and, with
// periodic boundaries, the reciprocal-space JVP of every tangent (lrt).
Extra tan_extra(colatus_t ctx) {
    Extra D = extra_args(ctx);
    D.lr32 = ctx->periodic ? ctx->tan.lrt : nullptr;
    D.lr64 = nullptr;
    return D;
}

}  // namespace

// ================================================================ C ABI
extern "C" {

colatus_status colatus_init(colatus_t *out, int64_t N, const double *masses, double eps,
                            double Omega_R, double Omega_M, double Omega_K, double Omega_L,
                            double H0, double a_start) {
    colatus_t ctx = nullptr;
    if (!out) return fail(nullptr, COLATUS_E_ARG, "out is NULL");
    *out = nullptr;
    if (N < 1) return fail(nullptr, COLATUS_E_ARG, "N must be >= 1 (got %lld)", (long long)N);
    if (!masses) return fail(nullptr, COLATUS_E_ARG, "masses is NULL");
    if (!(eps > 0.0) || !std::isfinite(eps))
        return fail(nullptr, COLATUS_E_ARG, "eps must be finite and > 0 (got %g)", eps);
    if (!(a_start > 0.0) || !std::isfinite(a_start))
        return fail(nullptr, COLATUS_E_ARG, "a_start must be finite and > 0");
    const double om[5] = {Omega_R, Omega_M, Omega_K, Omega_L, H0};
    for (double o : om)
        if (!std::isfinite(o)) return fail(nullptr, COLATUS_E_ARG, "cosmological parameters must be finite");
    const double e2 = Omega_R / std::pow(a_start, 4) + Omega_M / std::pow(a_start, 3) +
                      Omega_K / (a_start * a_start) + Omega_L;
    if (!(e2 >= 0.0)) return fail(nullptr, COLATUS_E_ARG, "H^2(a_start) < 0");
    for (int64_t i = 0; i < N; ++i)
        if (!std::isfinite(masses[i]) || masses[i] < 0.0)
            return fail(nullptr, COLATUS_E_ARG, "mass %lld is negative or not finite", (long long)i);

    ctx = new (std::nothrow) colatus_ctx();
    if (!ctx) return fail(nullptr, COLATUS_E_OOM, "host allocation failed");
    auto bail = [&](colatus_status st) {
        snprintf(g_init_err, sizeof(g_init_err), "%s", ctx->err);
        free_all(ctx);
        delete ctx;
        return st;
    };
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e != cudaSuccess) {
        fail(ctx, COLATUS_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
        return bail(COLATUS_E_CUDA);
    }
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, ctx->device);
    if (e != cudaSuccess) {
        fail(ctx, COLATUS_E_CUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
        return bail(COLATUS_E_CUDA);
    }
    ctx->num_sms = prop.multiProcessorCount;
    ctx->sym_max_bytes = prop.totalGlobalMem / kSymMemShare;
    ctx->tab_smem = (int)prop.sharedMemPerBlockOptin;
    if ((e = cudaFuncSetAttribute(friedmann_table_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  ctx->tab_smem)) != cudaSuccess) {
        fail(ctx, COLATUS_E_CUDA, "schedule kernel attributes: %s", cudaGetErrorString(e));
        return bail(COLATUS_E_CUDA);
    }
    ctx->N = N;
    ctx->n_alloc = round_up(N, kPadAlloc);
    colatus_status st = build_plans(ctx);
    if (st != COLATUS_OK) return bail(st);
    // every buffer holds the largest padded size any launch plan uses
    for (const ForcePlan &p : ctx->plan32) ctx->n_alloc = std::max(ctx->n_alloc, p.n_pad);
    for (const ForcePlan *p : {&ctx->plan64, &ctx->plan_vjp32, &ctx->plan_vjp64, &ctx->plan_ewvjp32,
                               &ctx->plan_ewvjp64, &ctx->plan_ew32[0],
                               &ctx->plan_ew32[1], &ctx->plan_ew64, &ctx->plan_vjp_sym, &ctx->plan_vjp_gen,
                               &ctx->plan_ew_sym[0], &ctx->plan_ew_sym[1], &ctx->plan_ewvjp_sym})
        ctx->n_alloc = std::max(ctx->n_alloc, p->n_pad);
    ctx->eps = eps;
    ctx->cosmo = Cosmo{Omega_R, Omega_M, Omega_K, Omega_L, H0};

    auto alloc = [&](void **p, size_t bytes) -> colatus_status {
        cudaError_t r = cudaMalloc(p, bytes);
        if (r != cudaSuccess)
            return fail(ctx, r == cudaErrorMemoryAllocation ? COLATUS_E_OOM : COLATUS_E_CUDA,
                        "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(r));
        return COLATUS_OK;
    };
    const size_t na = (size_t)ctx->n_alloc;
    void **f4[] = {(void **)&ctx->xs, (void **)&ctx->vs, (void **)&ctx->vh, (void **)&ctx->acc};
    for (void **p : f4)
        if (st == COLATUS_OK) st = alloc(p, na * sizeof(float4));
    for (int b = 0; b < 3 && st == COLATUS_OK; ++b) st = alloc((void **)&ctx->pk[b], na * 16);
    void **d4[] = {(void **)&ctx->xs64, (void **)&ctx->vs64, (void **)&ctx->vh64,
                   (void **)&ctx->acc64, (void **)&ctx->pos64[0], (void **)&ctx->pos64[1],
                   (void **)&ctx->pos64[2]};
    for (void **p : d4)
        if (st == COLATUS_OK) st = alloc(p, na * sizeof(double4));
    if (st == COLATUS_OK) st = alloc((void **)&ctx->m64, na * sizeof(double));
    if (st == COLATUS_OK) st = alloc((void **)&ctx->flags, NUM_FLAGS * sizeof(int));
    if (st == COLATUS_OK) st = alloc((void **)&ctx->mstat, 2 * sizeof(int));
    if (st == COLATUS_OK) st = alloc((void **)&ctx->clk, sizeof(DevClock));
    if (st == COLATUS_OK) st = alloc((void **)&ctx->tclk, sizeof(DevClock));
    if (st == COLATUS_OK) st = alloc((void **)&ctx->table, kTabCap * sizeof(StepCoef));
    if (st == COLATUS_OK) st = alloc((void **)&ctx->stage, na * 3 * sizeof(double));
    if (st == COLATUS_OK) st = alloc((void **)&ctx->stage2, na * 3 * sizeof(double));
    if (st == COLATUS_OK) st = alloc((void **)&ctx->diag, kDiagSlots * sizeof(double));
    if (st != COLATUS_OK) return bail(st);

    if ((e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking)) != cudaSuccess) {
        fail(ctx, COLATUS_E_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        return bail(COLATUS_E_CUDA);
    }
    ctx->own_stream = true;
    if ((e = cudaStreamCreateWithFlags(&ctx->tstream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&ctx->main_ev, cudaEventDisableTiming)) != cudaSuccess) {
        fail(ctx, COLATUS_E_CUDA, "stream/event creation: %s", cudaGetErrorString(e));
        return bail(COLATUS_E_CUDA);
    }
    for (int k = 0; k < kTabEvents; ++k) {
        if ((e = cudaEventCreateWithFlags(&ctx->tab_ev[k], cudaEventDisableTiming)) != cudaSuccess) {
            fail(ctx, COLATUS_E_CUDA, "event creation: %s", cudaGetErrorString(e));
            return bail(COLATUS_E_CUDA);
        }
        ctx->tab_ev_covers[k] = -1;
    }

    DevClock clk{0.0, a_start, 0, 0};
    cudaMemsetAsync(ctx->flags, 0, NUM_FLAGS * sizeof(int), ctx->stream);
    cudaMemcpyAsync(ctx->clk, &clk, sizeof(clk), cudaMemcpyHostToDevice, ctx->stream);
    // zero everything so that padding bodies are zero-mass at the origin
    for (void **p : f4) cudaMemsetAsync(*p, 0, na * sizeof(float4), ctx->stream);
    for (void **p : d4) cudaMemsetAsync(*p, 0, na * sizeof(double4), ctx->stream);
    for (int b = 0; b < 3; ++b) cudaMemsetAsync(ctx->pk[b], 0, na * 16, ctx->stream);
    cudaMemcpyAsync(ctx->stage, masses, N * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    if ((st = load_masses(ctx, ctx->stage, 1)) != COLATUS_OK) return bail(st);
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) {
        fail(ctx, COLATUS_E_CUDA, "init: %s", cudaGetErrorString(e));
        return bail(COLATUS_E_CUDA);
    }
    if ((st = read_flags(ctx, true)) != COLATUS_OK) return bail(COLATUS_E_ARG);
    *out = ctx;
    return COLATUS_OK;
}

colatus_status colatus_set_config(colatus_t ctx, colatus_prec prec, colatus_scheme scheme,
                                  double G, void *cuda_stream) {
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    if (prec != COLATUS_FP32 && prec != COLATUS_FP32_COMP && prec != COLATUS_FP64)
        return fail(ctx, COLATUS_E_ARG, "bad precision %d", (int)prec);
    if (scheme != COLATUS_DKD && scheme != COLATUS_KDK && scheme != COLATUS_KDK_CANONICAL)
        return fail(ctx, COLATUS_E_ARG, "bad scheme %d", (int)scheme);
    if (!std::isfinite(G)) return fail(ctx, COLATUS_E_ARG, "G must be finite");
    if (cuda_stream && (cudaStream_t)cuda_stream != ctx->stream) {
        CU(cudaStreamSynchronize(ctx->stream));
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        ctx->stream = (cudaStream_t)cuda_stream;
        ctx->own_stream = false;
    }
    const bool was64 = ctx->prec == COLATUS_FP64, is64 = prec == COLATUS_FP64;
    if (ctx->have_state && was64 != is64) {
        convert_state_kernel<<<blocks_for(ctx->N, 256), 256, 0, ctx->stream>>>(
            ctx->xs, ctx->vs, ctx->xs64, ctx->vs64, is64 ? 1 : 0, ctx->N);
        TRY(launched(ctx));
    }
    if (prec != ctx->prec || (scheme == COLATUS_DKD) != (ctx->scheme == COLATUS_DKD))
        ctx->acc_valid = false;
    if (scheme != ctx->scheme) ctx->tab_valid = false;   // the schedule's coefficients change
    ctx->spec_valid = false;
    ctx->tan.open = false;   // the tangent's half kick too
    ctx->prec = prec;
    ctx->scheme = scheme;
    ctx->G = G;
    if (ctx->periodic && was64 != is64) TRY(ewald_setup(ctx));   // tolerance follows the precision
    return COLATUS_OK;
}

colatus_status colatus_set_masses(colatus_t ctx, const void *m, int dtype, int on_device) {
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    TRY(check_dtype(ctx, dtype));
    if (!m) return fail(ctx, COLATUS_E_ARG, "masses is NULL");
    const void *src = m;
    if (!on_device) {
        CU(cudaMemcpyAsync(ctx->stage, m, ctx->N * elem_size(dtype), cudaMemcpyHostToDevice,
                           ctx->stream));
        src = ctx->stage;
    }
    CU(cudaStreamSynchronize(ctx->stream));
    TRY(read_flags(ctx, true));
    TRY(load_masses(ctx, src, dtype == COLATUS_F64));
    colatus_status st = sync_and_check(ctx);
    if (st == COLATUS_E_NONFINITE) return fail(ctx, COLATUS_E_ARG, "masses must be finite and >= 0");
    TRY(st);
    ctx->acc_valid = false;
    ctx->spec_valid = false;
    ctx->tan.open = false;   // the tangent's half kick too
    return COLATUS_OK;
}

colatus_status colatus_set_state(colatus_t ctx, const void *x, const void *v, int dtype,
                                 int on_device) {
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    TRY(check_dtype(ctx, dtype));
    if (!x) return fail(ctx, COLATUS_E_ARG, "x is NULL");
    const size_t bytes = (size_t)ctx->N * 3 * elem_size(dtype);
    const void *px = x, *pv = v;
    if (!on_device) {
        CU(cudaMemcpyAsync(ctx->stage, x, bytes, cudaMemcpyHostToDevice, ctx->stream));
        px = ctx->stage;
        if (v) {
            CU(cudaMemcpyAsync(ctx->stage2, v, bytes, cudaMemcpyHostToDevice, ctx->stream));
            pv = ctx->stage2;
        }
    }
    CU(cudaStreamSynchronize(ctx->stream));
    TRY(read_flags(ctx, true));
    load_state_kernel<<<blocks_for(ctx->N, 256), 256, 0, ctx->stream>>>(
        px, pv, dtype == COLATUS_F64, ctx->m64, ctx->N, ctx->xs, ctx->vs, ctx->xs64, ctx->vs64,
        ctx->flags);
    TRY(launched(ctx));
    TRY(sync_and_check(ctx));
    ctx->have_state = true;
    ctx->acc_valid = false;
    ctx->spec_valid = false;
    ctx->tan.open = false;   // the tangent's half kick too
    return COLATUS_OK;
}

colatus_status wait_reads(colatus_t ctx) {
    for (auto &r : ctx->rslot)
        if (r.busy) {
            CU(cudaEventSynchronize(r.done));
            r.busy = false;
        }
    return COLATUS_OK;
}

colatus_status colatus_get_state(colatus_t ctx, void *x, void *v, int dtype, int on_device,
                                 double *t, double *a) {
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    TRY(check_dtype(ctx, dtype));
    TRY(wait_reads(ctx));
    TRY(sync_and_check(ctx));
    if (x || v) {
        if (!ctx->have_state) return fail(ctx, COLATUS_E_STATE, "no state has been set");
        const size_t bytes = (size_t)ctx->N * 3 * elem_size(dtype);
        void *dx = on_device ? x : (x ? (void *)ctx->stage : nullptr);
        void *dv = on_device ? v : (v ? (void *)ctx->stage2 : nullptr);
        store_state_kernel<<<blocks_for(ctx->N, 256), 256, 0, ctx->stream>>>(
            ctx->xs, ctx->vs, ctx->xs64, ctx->vs64, ctx->prec == COLATUS_FP64, ctx->N, dx, dv,
            dtype == COLATUS_F64);
        TRY(launched(ctx));
        if (!on_device) {
            if (x) CU(cudaMemcpyAsync(x, ctx->stage, bytes, cudaMemcpyDeviceToHost, ctx->stream));
            if (v) CU(cudaMemcpyAsync(v, ctx->stage2, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        }
        CU(cudaStreamSynchronize(ctx->stream));
    }
    if (t || a) {
        DevClock c;
        CU(cudaMemcpy(&c, ctx->clk, sizeof(c), cudaMemcpyDeviceToHost));
        if (t) *t = c.t;
        if (a) *a = c.a;
    }
    return COLATUS_OK;
}

colatus_status colatus_get_state_async(colatus_t ctx, void *x, void *v, int dtype) {
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    TRY(check_dtype(ctx, dtype));
    if (!x && !v) return fail(ctx, COLATUS_E_ARG, "x and v are both NULL");
    if (!ctx->have_state) return fail(ctx, COLATUS_E_STATE, "no state has been set");
    if (!ctx->cstream) {
        CU(cudaStreamCreateWithFlags(&ctx->cstream, cudaStreamNonBlocking));
        for (auto &r : ctx->rslot) {
            CU(cudaMalloc(&r.x, (size_t)ctx->N * 3 * sizeof(double)));
            CU(cudaMalloc(&r.v, (size_t)ctx->N * 3 * sizeof(double)));
            CU(cudaEventCreateWithFlags(&r.snap, cudaEventDisableTiming));
            CU(cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming));
        }
    }
    auto &r = ctx->rslot[ctx->rnext];
    ctx->rnext = (ctx->rnext + 1) % kReadSlots;
    if (r.busy) CU(cudaEventSynchronize(r.done));   // its previous copy still reads the slot
    r.busy = false;
    // snapshot, ordered after the steps enqueued so far
    store_state_kernel<<<blocks_for(ctx->N, 256), 256, 0, ctx->stream>>>(
        ctx->xs, ctx->vs, ctx->xs64, ctx->vs64, ctx->prec == COLATUS_FP64, ctx->N, x ? r.x : nullptr,
        v ? r.v : nullptr, dtype == COLATUS_F64);
    TRY(launched(ctx));
    CU(cudaEventRecord(r.snap, ctx->stream));
    CU(cudaStreamWaitEvent(ctx->cstream, r.snap, 0));
    const size_t bytes = (size_t)ctx->N * 3 * elem_size(dtype);
    if (x) CU(cudaMemcpyAsync(x, r.x, bytes, cudaMemcpyDeviceToHost, ctx->cstream));
    if (v) CU(cudaMemcpyAsync(v, r.v, bytes, cudaMemcpyDeviceToHost, ctx->cstream));
    CU(cudaEventRecord(r.done, ctx->cstream));
    r.busy = true;
    return COLATUS_OK;
}

colatus_status colatus_wait_state(colatus_t ctx) {
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    TRY(wait_reads(ctx));
    return sync_and_check(ctx);
}

colatus_status colatus_forces(colatus_t ctx, void *acc_out, int dtype, int on_device) {
    NvtxRange nvtx_("colatus_forces");
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    TRY(check_dtype(ctx, dtype));
    if (!acc_out) return fail(ctx, COLATUS_E_ARG, "acc_out is NULL");
    if (!ctx->have_state) return fail(ctx, COLATUS_E_STATE, "no state has been set");
    TRY(force_at_state(ctx));
    void *dst = on_device ? acc_out : (void *)ctx->stage;
    TRY(force_output(ctx, dst, dtype == COLATUS_F64, true));
    ctx->acc_valid = true;
    if (!on_device) {
        CU(cudaMemcpyAsync(acc_out, ctx->stage, (size_t)ctx->N * 3 * elem_size(dtype),
                           cudaMemcpyDeviceToHost, ctx->stream));
        TRY(sync_and_check(ctx));
    }
    return COLATUS_OK;
}

colatus_status colatus_step(colatus_t ctx, double dt, int64_t nsteps) {
    NvtxRange nvtx_("colatus_step");
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, COLATUS_E_ARG, "dt must be finite and > 0");
    if (nsteps < 0) return fail(ctx, COLATUS_E_ARG, "nsteps must be >= 0");
    if (!ctx->have_state) return fail(ctx, COLATUS_E_STATE, "no state has been set");
    if (nsteps == 0) return COLATUS_OK;
    if (ctx->spec_valid && ctx->spec_tau != dt) ctx->spec_valid = false;
    for (int64_t done = 0; done < nsteps;) {
        const int n = (int)std::min<int64_t>(kChunk, nsteps - done);
        TRY(need_table(ctx, dt, n, kTabPiece));
        if (!ctx->spec_valid) {
            TRY(open_step(ctx, dt));
            ctx->spec_valid = true;
            ctx->spec_tau = dt;
        }
        for (int j = 0; j < n; ++j) {
            TRY(wait_table_at(ctx, j, n));
            TRY(one_step(ctx, j, dt));
        }
        done += n;
        ctx->host_step += n;
        TRY(refill_table(ctx));
    }
    ctx->acc_valid = is_kdk(ctx);
    return COLATUS_OK;
}

colatus_status colatus_synchronize(colatus_t ctx) {
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    TRY(wait_reads(ctx));
    return sync_and_check(ctx);
}

colatus_status colatus_record_tracers(colatus_t ctx, const int64_t *idx, int ntr,
                                      int64_t capacity_steps) {
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    if (ntr < 0) return fail(ctx, COLATUS_E_ARG, "ntr must be >= 0");
    if (ntr > 0 && (!idx || capacity_steps < 1))
        return fail(ctx, COLATUS_E_ARG, "need indices and capacity_steps >= 1");
    std::vector<int> slot;
    if (ntr > 0) {
        slot.assign(ctx->N, -1);
        for (int k = 0; k < ntr; ++k) {
            if (idx[k] < 0 || idx[k] >= ctx->N)
                return fail(ctx, COLATUS_E_ARG, "tracer index %lld out of range", (long long)idx[k]);
            if (slot[idx[k]] >= 0) return fail(ctx, COLATUS_E_ARG, "duplicate tracer index");
            slot[idx[k]] = k;
        }
    }
    CU(cudaStreamSynchronize(ctx->stream));
    if (ctx->tslot) cudaFree(ctx->tslot);
    if (ctx->rec) cudaFree(ctx->rec);
    ctx->tslot = nullptr;
    ctx->rec = nullptr;
    ctx->ntr = 0;
    ctx->rec_cap = 0;
    ctx->tidx.clear();
    if (ntr == 0) return COLATUS_OK;
    CU(cudaMalloc(&ctx->tslot, ctx->N * sizeof(int)));
    CU(cudaMalloc(&ctx->rec, (size_t)capacity_steps * ntr * 6 * sizeof(float)));
    CU(cudaMemcpy(ctx->tslot, slot.data(), ctx->N * sizeof(int), cudaMemcpyHostToDevice));
    ctx->ntr = ntr;
    ctx->rec_cap = capacity_steps;
    ctx->rec_base = ctx->host_step;
    ctx->tidx.assign(idx, idx + ntr);
    return COLATUS_OK;
}

colatus_status colatus_read_tracers(colatus_t ctx, float *xv_out, int64_t *nrec_out) {
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    if (!nrec_out) return fail(ctx, COLATUS_E_ARG, "nrec_out is NULL");
    TRY(sync_and_check(ctx));
    if (ctx->ntr == 0) {
        *nrec_out = 0;
        return COLATUS_OK;
    }
    const long long total = ctx->host_step - ctx->rec_base;
    const long long nrec = std::min(total, ctx->rec_cap);
    *nrec_out = nrec;
    if (!xv_out || nrec == 0) return COLATUS_OK;
    const size_t row = (size_t)ctx->ntr * 6;
    std::vector<float> ring((size_t)ctx->rec_cap * row);
    CU(cudaMemcpy(ring.data(), ctx->rec, ring.size() * sizeof(float), cudaMemcpyDeviceToHost));
    for (long long k = 0; k < nrec; ++k) {
        const long long s = total - nrec + k;   // steps since the recording started
        const long long r = s % ctx->rec_cap;
        std::memcpy(xv_out + k * row, ring.data() + r * row, row * sizeof(float));
    }
    return COLATUS_OK;
}

colatus_status colatus_diagnostics(colatus_t ctx, double out[COLATUS_NDIAG]) {
    NvtxRange nvtx_("colatus_diagnostics");
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    if (!out) return fail(ctx, COLATUS_E_ARG, "out is NULL");
    if (!ctx->have_state) return fail(ctx, COLATUS_E_STATE, "no state has been set");
    TRY(sync_and_check(ctx));
    const bool f64 = ctx->prec == COLATUS_FP64;
    CU(cudaMemsetAsync(ctx->diag, 0, kDiagSlots * sizeof(double), ctx->stream));
    const unsigned nb = (unsigned)std::min<long long>(
        {(long long)blocks_for(ctx->N, kDiagThreads), 4LL * ctx->num_sms, (long long)kDiagMaxBlocks});
    // potential pair sums: i-tiles x source splits.  Blocks are equal work
    // (tps source tiles), so the time goes as ceil(blocks / SMs) x tps; take
    // the split with the least (fewer blocks on ties), at most 64 splits and
    // at most 64 MB of per-split sums.
    const long long n_ib = (ctx->N + kPotITILE - 1) / kPotITILE;
    const long long n_jt = (ctx->N + kPotJT - 1) / kPotJT;
    const long long max_sp = std::max(1LL, std::min({n_jt, 64LL, (8LL << 20) / ctx->N}));
    long long tps = n_jt, best = -1;
    for (long long sp = 1; sp <= max_sp; ++sp) {
        const long long t = (n_jt + sp - 1) / sp, blocks = n_ib * ((n_jt + t - 1) / t);
        const long long cost = (blocks + ctx->num_sms - 1) / ctx->num_sms * t;
        if (best < 0 || cost < best) {
            best = cost;
            tps = t;
        }
    }
    const int splits = (int)((n_jt + tps - 1) / tps);
    TRY(grow(ctx, &ctx->pot_part, &ctx->pot_part_bytes, (size_t)splits * ctx->N * sizeof(double)));
    double *pot_part = static_cast<double *>(ctx->pot_part);
    const dim3 pgrid((unsigned)n_ib, (unsigned)splits);
    if (f64)
        potential_f64_kernel<<<pgrid, kDiagThreads, 0, ctx->stream>>>(
            ctx->xs64, ctx->N, ctx->eps * ctx->eps, (int)tps, pot_part);
    else
        potential_f32_kernel<<<pgrid, kDiagThreads, 0, ctx->stream>>>(
            ctx->xs, ctx->N, (float)(ctx->eps * ctx->eps), (int)tps, pot_part);
    TRY(launched(ctx));
    potential_sum_kernel<<<nb, kDiagThreads, 0, ctx->stream>>>(pot_part, splits, ctx->xs, ctx->xs64,
                                                               f64 ? 1 : 0, ctx->N, ctx->diag);
    TRY(launched(ctx));
    moments_kernel<<<nb, kDiagThreads, 0, ctx->stream>>>(ctx->xs, ctx->vs, ctx->xs64, ctx->vs64,
                                                        f64 ? 1 : 0, ctx->N, ctx->diag);
    TRY(launched(ctx));
    finish_diagnostics_kernel<<<1, kDiagQ * 32, 0, ctx->stream>>>(ctx->diag, (int)nb, ctx->clk, ctx->cosmo,
                                                                ctx->G);
    TRY(launched(ctx));
    CU(cudaMemcpyAsync(out, ctx->diag + kDiagOut, COLATUS_NDIAG * sizeof(double),
                       cudaMemcpyDeviceToHost, ctx->stream));
    TRY(sync_and_check(ctx));
    out[15] = (double)ctx->host_step;
    return COLATUS_OK;
}

colatus_status colatus_profile_forces(colatus_t ctx, int on) {
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->profiling = on != 0;
    ctx->ev_used = 0;
    return COLATUS_OK;
}

colatus_status colatus_profile_read_kinds(colatus_t ctx, double out[6]) {
    if (!ctx || !out) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    CU(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < 6; ++k) out[k] = 0.0;
    for (size_t k = 0; k + 1 < ctx->ev_used; k += 2) {
        float e = 0.f;
        CU(cudaEventElapsedTime(&e, ctx->ev_pool[k], ctx->ev_pool[k + 1]));
        const int c = 2 * std::min(ctx->ev_cat[k], 2);
        out[c] += e;
        out[c + 1] += 1.0;
    }
    ctx->ev_used = 0;
    return COLATUS_OK;
}

colatus_status colatus_profile_read(colatus_t ctx, double out[4]) {
    if (!ctx || !out) return COLATUS_E_ARG;
    double all[6];
    TRY(colatus_profile_read_kinds(ctx, all));
    for (int k = 0; k < 4; ++k) out[k] = all[k];
    return COLATUS_OK;
}


colatus_status colatus_force_vjp(colatus_t ctx, const void *w, void *gx, void *gm, int dtype,
                                 int on_device) {
    NvtxRange nvtx_("colatus_force_vjp");
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    TRY(check_dtype(ctx, dtype));
    if (!w || (!gx && !gm)) return fail(ctx, COLATUS_E_ARG, "need w and at least one output");
    if (!ctx->have_state) return fail(ctx, COLATUS_E_STATE, "no state has been set");
    TRY(adj_alloc(ctx));
    const int f64in = dtype == COLATUS_F64;
    const size_t vbytes = (size_t)ctx->N * 3 * elem_size(dtype);
    const void *src = w;
    if (!on_device) {
        CU(cudaMemcpyAsync(ctx->stage, w, vbytes, cudaMemcpyHostToDevice, ctx->stream));
        src = ctx->stage;
    }
    const unsigned nb = blocks_for(ctx->N, 256);
    void *dgx = on_device ? gx : (gx ? (void *)ctx->stage : nullptr);
    void *dgm = on_device ? gm : (gm ? (void *)ctx->stage2 : nullptr);
    if (ctx->prec == COLATUS_FP64) {
        const ForcePlan &p = vjp_plan(ctx);
        vec3_to4_kernel<double4, double><<<nb, 256, 0, ctx->stream>>>(
            src, f64in, ctx->N, static_cast<double4 *>(ctx->adj.lx));
        TRY(launched(ctx));
        vjp_pack_f64_kernel<<<blocks_for(p.n_pad, 256), 256, 0, ctx->stream>>>(
            ctx->xs64, static_cast<const double4 *>(ctx->adj.lx), ctx->clk, ctx->G, 1,
            static_cast<double4 *>(ctx->adj.pkw), ctx->N, p.n_pad);
        TRY(launched(ctx));
        TRY(run_vjp(ctx));
        vjp_out_f64_kernel<<<nb, 256, 0, ctx->stream>>>(static_cast<const double4 *>(ctx->part), p.L,
                                                        p.itile, ctx->N, dgx, dgm, f64in,
                                                        static_cast<const double4 *>(ctx->adj.pkw),
                                                        vjp_extra(ctx));
    } else {
        const ForcePlan &p = vjp_plan(ctx);
        vec3_to4_kernel<float4, float><<<nb, 256, 0, ctx->stream>>>(
            src, f64in, ctx->N, static_cast<float4 *>(ctx->adj.lx));
        TRY(launched(ctx));
        vjp_pack_f32_kernel<<<blocks_for(p.n_pad, 256), 256, 0, ctx->stream>>>(
            ctx->xs, static_cast<const float4 *>(ctx->adj.lx), ctx->clk, ctx->G, 1,
            static_cast<float *>(ctx->adj.pkw), ctx->N, p.n_pad);
        TRY(launched(ctx));
        TRY(run_vjp(ctx));
        vjp_out_f32_kernel<<<nb, 256, 0, ctx->stream>>>(static_cast<const float4 *>(ctx->part), p.L,
                                                        p.itile, ctx->N, dgx, dgm, f64in,
                                                        static_cast<const float *>(ctx->adj.pkw),
                                                        vjp_extra(ctx));
    }
    TRY(launched(ctx));
    if (!on_device) {
        if (gx) CU(cudaMemcpyAsync(gx, ctx->stage, vbytes, cudaMemcpyDeviceToHost, ctx->stream));
        if (gm)
            CU(cudaMemcpyAsync(gm, ctx->stage2, (size_t)ctx->N * elem_size(dtype),
                               cudaMemcpyDeviceToHost, ctx->stream));
        TRY(sync_and_check(ctx));
    }
    return COLATUS_OK;
}

colatus_status colatus_adjoint_forward(colatus_t ctx, double dt, int64_t nsteps,
                                       int64_t checkpoint_every) {
    NvtxRange nvtx_("colatus_adjoint_forward");
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, COLATUS_E_ARG, "dt must be finite and > 0");
    if (nsteps < 1 || checkpoint_every < 1)
        return fail(ctx, COLATUS_E_ARG, "nsteps and checkpoint_every must be >= 1");
    if (!ctx->have_state) return fail(ctx, COLATUS_E_STATE, "no state has been set");
    auto &a = ctx->adj;
    a.ready = false;
    TRY(adj_alloc(ctx));
    const int k = (int)std::min<int64_t>(checkpoint_every, nsteps);
    const int nck = (int)((nsteps + k - 1) / k);
    const size_t body = ctx->prec == COLATUS_FP64 ? sizeof(double4) : sizeof(float4);
    const size_t plane = (size_t)ctx->n_alloc * body;
    if (a.ck_bytes < nck * plane) {
        if (a.ck_x) cudaFree(a.ck_x);
        if (a.ck_v) cudaFree(a.ck_v);
        a.ck_x = a.ck_v = nullptr;
        a.ck_bytes = 0;
        CU(cudaMalloc(&a.ck_x, nck * plane));
        CU(cudaMalloc(&a.ck_v, nck * plane));
        a.ck_bytes = nck * plane;
    }
    TRY(grow(ctx, &a.seg_x, &a.seg_bytes, (size_t)k * plane));
    TRY(grow(ctx, reinterpret_cast<void **>(&a.table), &a.tab_bytes, (size_t)nsteps * sizeof(StepCoef)));
    // the forward's schedule, computed from the current clock exactly as the
    // look-ahead schedule is (same kernel, same start): bitwise the same values
    clock_copy_kernel<<<1, 1, 0, ctx->stream>>>(ctx->clk, a.rclk);
    TRY(launched(ctx));
    // index the forward's schedule by step within the pass (0 .. nsteps-1)
    CU(cudaMemsetAsync(&a.rclk->step, 0, sizeof(a.rclk->step), ctx->stream));
    // only the backward pass reads it: computed on the side stream, off the
    // forward steps' critical path (which then use the smaller grids)
    CU(cudaEventRecord(ctx->main_ev, ctx->stream));
    CU(cudaStreamWaitEvent(ctx->tstream, ctx->main_ev, 0));
    friedmann_table_kernel<<<1, 1, ctx->tab_smem, ctx->tstream>>>(
        ctx->cosmo, a.rclk, a.table, (int)nsteps, (int)nsteps, dt, ctx->G, kFriedmannSub,
        canonical(ctx));
    TRY(launched(ctx));
    CU(cudaEventRecord(a.tab_ev, ctx->tstream));
    const long long step0 = ctx->host_step;
    const bool f64 = ctx->prec == COLATUS_FP64;
    for (int c = 0; c < nck; ++c) {
        char *cx = static_cast<char *>(a.ck_x) + c * plane;
        char *cv = static_cast<char *>(a.ck_v) + c * plane;
        CU(cudaMemcpyAsync(cx, f64 ? (void *)ctx->xs64 : (void *)ctx->xs, (size_t)ctx->N * body,
                           cudaMemcpyDeviceToDevice, ctx->stream));
        CU(cudaMemcpyAsync(cv, f64 ? (void *)ctx->vs64 : (void *)ctx->vs, (size_t)ctx->N * body,
                           cudaMemcpyDeviceToDevice, ctx->stream));
        TRY(colatus_step(ctx, dt, std::min<int64_t>(k, nsteps - (int64_t)c * k)));
    }
    a.ready = true;
    a.nsteps = nsteps;
    a.step0 = step0;
    a.k = k;
    a.nck = nck;
    a.tau = dt;
    a.prec = ctx->prec;
    a.scheme = ctx->scheme;
    a.G = ctx->G;
    return COLATUS_OK;
}

colatus_status colatus_adjoint_backward(colatus_t ctx, const void *gx_T, const void *gv_T,
                                        const void *gm_T, void *gx_0, void *gv_0, void *gm,
                                        int dtype, int on_device) {
    NvtxRange nvtx_("colatus_adjoint_backward");
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    TRY(check_dtype(ctx, dtype));
    auto &a = ctx->adj;
    if (!a.ready) return fail(ctx, COLATUS_E_STATE, "no adjoint forward pass recorded");
    if (ctx->host_step != a.step0 + a.nsteps || ctx->prec != a.prec || ctx->scheme != a.scheme ||
        ctx->G != a.G)
        return fail(ctx, COLATUS_E_STATE, "the state or the configuration changed since the adjoint forward pass");
    CU(cudaStreamWaitEvent(ctx->stream, a.tab_ev, 0));   // the forward's schedule
    const bool f64 = ctx->prec == COLATUS_FP64;
    const int in64 = dtype == COLATUS_F64;
    const size_t vbytes = (size_t)ctx->N * 3 * elem_size(dtype);
    const size_t sbytes = (size_t)ctx->N * elem_size(dtype);
    const void *sx = gx_T, *sv = gv_T, *sm = gm_T;
    if (!on_device) {
        if (gx_T) {
            CU(cudaMemcpyAsync(ctx->stage, gx_T, vbytes, cudaMemcpyHostToDevice, ctx->stream));
            sx = ctx->stage;
        }
        if (gv_T) {
            CU(cudaMemcpyAsync(ctx->stage2, gv_T, vbytes, cudaMemcpyHostToDevice, ctx->stream));
            sv = ctx->stage2;
        }
        if (gm_T) {
            CU(cudaMemcpyAsync(a.rvs, gm_T, sbytes, cudaMemcpyHostToDevice, ctx->stream));
            sm = a.rvs;
        }
    }
    const size_t body = f64 ? sizeof(double4) : sizeof(float4);
    const size_t plane = (size_t)ctx->n_alloc * body;
    const ForcePlan &pv0 = vjp_plan(ctx);
    const long long NS = a.nsteps;
    const unsigned nbv = blocks_for(pv0.n_pad, 256);
    // Equal masses, isolated boundaries, no deformation term and no padding in
    // the VJP's tiles: the equal-mass VJP, whose mass gradient takes the force
    // at each position; the recompute keeps them (seg_f, slot n - s0 for x_n).
    // DKD (Eqs. 3-5): one VJP per step at the half-drift position xh_n, formed
    // from the segment's positions and velocities (seg_v keeps the latter).
    const bool dkd = a.scheme == COLATUS_DKD;
    const bool eqm = !dkd && !f64 && ctx->eq_mass && !ctx->periodic && ctx->defo_C == 0.0 &&
                     pv0.n_pad == ctx->N;
    // the consumers' segment layout: the kernel run_vjp(ctx, eqm) launches
    // (the pair-once one has the same padding, so pv0.n_pad stands for both)
    const ForcePlan &pv = vjp_plan(ctx, eqm);
    if (eqm) TRY(grow(ctx, &a.seg_f, &a.segf_bytes, (size_t)(a.k + 1) * plane));
    if (dkd) TRY(grow(ctx, &a.seg_v, &a.segv_bytes, (size_t)a.k * plane));
    auto fslot = [&](long long j) {
        return static_cast<float4 *>(a.seg_f) + (size_t)j * ctx->n_alloc;
    };
    auto vjp_args = [&](const float4 *f) {
        Extra D = vjp_extra(ctx);
        if (eqm) {
            D.eqf = f;
            D.eqminv = 1.f / ctx->mass_eq;
        }
        return D;
    };
    if (f64)
        adj_init_f64_kernel<<<nbv, 256, 0, ctx->stream>>>(
            sx, sv, sm, in64, ctx->xs64, static_cast<double4 *>(a.lx), static_cast<double4 *>(a.lv),
            static_cast<double *>(a.lm), a.table, NS - 1, static_cast<double4 *>(a.pkw), ctx->N, pv.n_pad);
    else
        adj_init_f32_kernel<<<nbv, 256, 0, ctx->stream>>>(
            sx, sv, sm, in64, ctx->xs, static_cast<float4 *>(a.lx), static_cast<float4 *>(a.lv),
            static_cast<float *>(a.lm), a.table, NS - 1, static_cast<float *>(a.pkw), ctx->N, pv.n_pad);
    TRY(launched(ctx));

    for (int c = a.nck - 1; c >= 0; --c) {
        const long long s0 = (long long)c * a.k, s1 = std::min<long long>(s0 + a.k, NS);
        char *ckx = static_cast<char *>(a.ck_x) + c * plane;
        char *ckv = static_cast<char *>(a.ck_v) + c * plane;
        auto pos = [&](long long n) -> void * {
            return n == s0 ? (void *)ckx : (void *)(static_cast<char *>(a.seg_x) + (n - s0) * plane);
        };
        auto vel = [&](long long n) -> void * {
            return n == s0 ? (void *)ckv : (void *)(static_cast<char *>(a.seg_v) + (n - s0) * plane);
        };
        if (eqm) {
            // F(x_{s1}): the forward's last force, or the checkpoint force of
            // the segment swept before this one (its slot 0)
            const void *src = c == a.nck - 1 ? (const void *)ctx->acc : (const void *)fslot(0);
            CU(cudaMemcpyAsync(fslot(s1 - s0), src, (size_t)ctx->N * sizeof(float4),
                               cudaMemcpyDeviceToDevice, ctx->stream));
        }
        if (s1 - s0 > 1 || eqm) {
            // recompute x_{s0+1} .. x_{s1-1} with the forward's own kernels
            StepBufs b;
            b.xs = reinterpret_cast<float4 *>(ckx);
            b.vs = reinterpret_cast<float4 *>(ckv);
            b.vh = static_cast<float4 *>(a.rvh);
            b.acc = eqm ? fslot(0) : static_cast<float4 *>(a.racc);
            b.pk[0] = static_cast<float *>(a.rpk[0]);
            b.pk[1] = static_cast<float *>(a.rpk[1]);
            b.xs64 = reinterpret_cast<double4 *>(ckx);
            b.vs64 = reinterpret_cast<double4 *>(ckv);
            b.vh64 = static_cast<double4 *>(a.rvh);
            b.acc64 = static_cast<double4 *>(a.racc);
            b.pos64[0] = static_cast<double4 *>(a.rpk[0]);
            b.pos64[1] = static_cast<double4 *>(a.rpk[1]);
            b.table = a.table;
            b.tcap = (int)NS;
            b.clk = a.rclk;
            b.tr = Tracers{nullptr, nullptr, 1, 0, 0};
            if (dkd) {
                // the DKD steps update the velocity in place: start from a copy
                // of the checkpoint's, then the half drift into the force input
                CU(cudaMemcpyAsync(a.rvs, ckv, (size_t)ctx->N * body, cudaMemcpyDeviceToDevice,
                                   ctx->stream));
                b.vs = static_cast<float4 *>(a.rvs);
                b.vs64 = static_cast<double4 *>(a.rvs);
                if (f64) {
                    const ForcePlan &p = plan_f64(ctx);
                    dkd_open_f64_kernel<<<blocks_for(p.n_pad, 256), 256, 0, ctx->stream>>>(
                        b.xs64, b.vs64, b.pos64[1], a.tau, ctx->N, p.n_pad);
                } else {
                    const ForcePlan &p = plan_f32(ctx);
                    dkd_open_f32_kernel<<<blocks_for(p.n_pad, 256), 256, 0, ctx->stream>>>(
                        b.xs, b.vs, b.pk[1], a.tau, ctx->N, p.n_pad);
                }
                TRY(launched(ctx));
            } else {
                // F at the checkpoint
                if (f64) {
                    const ForcePlan &p = plan_f64(ctx);
                    pack_f64_kernel<<<blocks_for(p.n_pad, 256), 256, 0, ctx->stream>>>(
                        b.xs64, b.pos64[0], ctx->N, p.n_pad);
                    TRY(launched(ctx));
                    TRY(run_force_f64(ctx, b.pos64[0]));
                    forces_out_f64_kernel<<<blocks_for(ctx->N, 256), 256, 0, ctx->stream>>>(
                        static_cast<const double4 *>(ctx->part), p.L, p.itile, ctx->N, ctx->clk, ctx->G,
                        nullptr, 0, b.acc64, b.pos64[0], extra_args(ctx));
                } else {
                    const ForcePlan &p = plan_f32(ctx);
                    pack_f32_kernel<<<blocks_for(p.n_pad, 256), 256, 0, ctx->stream>>>(
                        b.xs, b.pk[0], ctx->N, p.n_pad);
                    TRY(launched(ctx));
                    TRY(run_force_f32(ctx, p, b.pk[0]));
                    if (ctx->prec == COLATUS_FP32_COMP)
                        launch_forces_out_f32<true>(ctx, p, nullptr, 0, b.acc, b.pk[0]);
                    else
                        launch_forces_out_f32<false>(ctx, p, nullptr, 0, b.acc, b.pk[0]);
                }
                TRY(launched(ctx));
                TRY(launch_kdk_open(ctx, b, 1, s0, a.tau));
                b.vs = static_cast<float4 *>(a.rvs);
                b.vs64 = static_cast<double4 *>(a.rvs);
            }
            int cur = 1;
            for (long long n = s0; n < s1 - 1; ++n) {
                b.xs = static_cast<float4 *>(pos(n + 1));
                b.xs64 = static_cast<double4 *>(pos(n + 1));
                if (eqm) b.acc = fslot(n + 1 - s0);
                TRY(launch_step(ctx, b, cur, n, a.tau));
                if (dkd)
                    CU(cudaMemcpyAsync(vel(n + 1), a.rvs, (size_t)ctx->N * body, cudaMemcpyDeviceToDevice,
                                       ctx->stream));
                cur ^= 1;
            }
        }
        for (long long n = s1 - 1; n >= s0 && dkd; --n) {
            // DKD step n: pack (xh_n, W_n), the VJP at xh_n, the update
            if (f64)
                dkd_adj_pack_f64_kernel<<<nbv, 256, 0, ctx->stream>>>(
                    static_cast<const double4 *>(pos(n)), static_cast<const double4 *>(vel(n)),
                    static_cast<const double4 *>(a.lx), static_cast<const double4 *>(a.lv), a.table, n,
                    a.tau, static_cast<double4 *>(a.pkw), ctx->N, pv.n_pad);
            else
                dkd_adj_pack_f32_kernel<<<nbv, 256, 0, ctx->stream>>>(
                    static_cast<const float4 *>(pos(n)), static_cast<const float4 *>(vel(n)),
                    static_cast<const float4 *>(a.lx), static_cast<const float4 *>(a.lv), a.table, n,
                    a.tau, static_cast<float *>(a.pkw), ctx->N, pv.n_pad);
            TRY(launched(ctx));
            TRY(run_vjp(ctx));
            TRY(prof_begin(ctx));
            const unsigned nbn = blocks_for(ctx->N, 256);
            if (f64)
                dkd_adj_update_f64_kernel<<<nbn, 256, 0, ctx->stream>>>(
                    static_cast<const double4 *>(ctx->part), pv.L, pv.itile, static_cast<double4 *>(a.lx),
                    static_cast<double4 *>(a.lv), static_cast<double *>(a.lm), a.table, n, a.tau,
                    static_cast<const double4 *>(a.pkw), ctx->N, vjp_extra(ctx));
            else
                dkd_adj_update_f32_kernel<<<nbn, 256, 0, ctx->stream>>>(
                    static_cast<const float4 *>(ctx->part), pv.L, pv.itile, static_cast<float4 *>(a.lx),
                    static_cast<float4 *>(a.lv), static_cast<float *>(a.lm), a.table, n, a.tau,
                    static_cast<const float *>(a.pkw), ctx->N, vjp_extra(ctx));
            TRY(launched(ctx));
            TRY(prof_end(ctx, 2));
        }
        for (long long n = s1 - 1; n >= s0 && !dkd; --n) {
            TRY(run_vjp(ctx, eqm));
            TRY(prof_begin(ctx));
            if (f64)
                adj_step_f64_kernel<<<nbv, 256, 0, ctx->stream>>>(
                    static_cast<const double4 *>(ctx->part), pv.L, pv.itile,
                    static_cast<const double4 *>(pos(n)), static_cast<double4 *>(a.lx),
                    static_cast<double4 *>(a.lv), static_cast<double4 *>(a.lvh),
                    static_cast<double *>(a.lm), a.table, n, a.tau, static_cast<double4 *>(a.pkw),
                    ctx->N, pv.n_pad, vjp_extra(ctx));
            else
                adj_step_f32_kernel<<<nbv, 256, 0, ctx->stream>>>(
                    static_cast<const float4 *>(ctx->part), pv.L, pv.itile,
                    static_cast<const float4 *>(pos(n)), static_cast<float4 *>(a.lx),
                    static_cast<float4 *>(a.lv), static_cast<float4 *>(a.lvh),
                    static_cast<float *>(a.lm), a.table, n, a.tau, static_cast<float *>(a.pkw),
                    ctx->N, pv.n_pad, vjp_args(eqm ? fslot(n + 1 - s0) : nullptr));
            TRY(launched(ctx));
            TRY(prof_end(ctx, 2));
        }
    }
    // KDK: F(x_0) enters the first half kick, so one more VJP at x_0 (F(x_0):
    // slot 0 of the first segment for the equal-mass form).  DKD: the sweep
    // already ended at step 0.
    if (!dkd) TRY(run_vjp(ctx, eqm));
    const unsigned nb = blocks_for(ctx->N, 256);
    void *dgx = on_device ? gx_0 : (gx_0 ? (void *)ctx->stage : nullptr);
    void *dgv = on_device ? gv_0 : (gv_0 ? (void *)ctx->stage2 : nullptr);
    void *dgm = on_device ? gm : (gm ? a.rvh : nullptr);
    if (f64) {
        if (!dkd) {
            adj_final_f64_kernel<<<nb, 256, 0, ctx->stream>>>(
                static_cast<const double4 *>(ctx->part), pv.L, pv.itile, static_cast<double4 *>(a.lx),
                static_cast<double *>(a.lm), ctx->N, static_cast<const double4 *>(a.pkw), vjp_extra(ctx));
            TRY(launched(ctx));
        }
        adj_store_kernel<double4, double><<<nb, 256, 0, ctx->stream>>>(
            static_cast<const double4 *>(a.lx), static_cast<const double4 *>(a.lv),
            static_cast<const double *>(a.lm), ctx->N, dgx, dgv, dgm, in64);
    } else {
        if (!dkd) {
            adj_final_f32_kernel<<<nb, 256, 0, ctx->stream>>>(
                static_cast<const float4 *>(ctx->part), pv.L, pv.itile, static_cast<float4 *>(a.lx),
                static_cast<float *>(a.lm), ctx->N, static_cast<const float *>(a.pkw),
                vjp_args(eqm ? fslot(0) : nullptr));
            TRY(launched(ctx));
        }
        adj_store_kernel<float4, float><<<nb, 256, 0, ctx->stream>>>(
            static_cast<const float4 *>(a.lx), static_cast<const float4 *>(a.lv),
            static_cast<const float *>(a.lm), ctx->N, dgx, dgv, dgm, in64);
    }
    TRY(launched(ctx));
    if (!on_device) {
        if (gx_0) CU(cudaMemcpyAsync(gx_0, ctx->stage, vbytes, cudaMemcpyDeviceToHost, ctx->stream));
        if (gv_0) CU(cudaMemcpyAsync(gv_0, ctx->stage2, vbytes, cudaMemcpyDeviceToHost, ctx->stream));
        if (gm) CU(cudaMemcpyAsync(gm, a.rvh, sbytes, cudaMemcpyDeviceToHost, ctx->stream));
        TRY(sync_and_check(ctx));
    }
    return COLATUS_OK;
}

colatus_status colatus_tangent_init(colatus_t ctx, const int64_t *seeds, int B, const double *dir,
                                    int64_t capacity_steps) {
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    auto &t = ctx->tan;
    if (B < 1 || !seeds || capacity_steps < 1) return fail(ctx, COLATUS_E_ARG, "need B >= 1 seeds and capacity");
    for (int b = 0; b < B; ++b)
        if (seeds[b] < 0 || seeds[b] >= ctx->N) return fail(ctx, COLATUS_E_ARG, "seed out of range");
    double d[3] = {1.0, 0.0, 0.0};
    if (dir) {
        const double nrm = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
        if (!(nrm > 0.0) || !std::isfinite(nrm)) return fail(ctx, COLATUS_E_ARG, "bad direction");
        for (int c = 0; c < 3; ++c) d[c] = dir[c] / nrm;
    }
    if (!ctx->have_state) return fail(ctx, COLATUS_E_STATE, "no state has been set");
    CU(cudaStreamSynchronize(ctx->stream));
    void *old[] = {t.dx, t.dv, t.dvh, t.dxp, t.pkt, t.seeds, t.growth, t.lrt};
    for (void *p : old)
        if (p) cudaFree(p);
    t = colatus_ctx::Tangent();
    int occ = 0;
    if (JvpK::SMEM > 48 * 1024)
        CU(cudaFuncSetAttribute(jvp_f32x2_kernel<kJvpNT, kJvpIPT, kJvpJT, kStages, kJvpMINB, kJvpUnr>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, JvpK::SMEM));
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, jvp_f32x2_kernel<kJvpNT, kJvpIPT, kJvpJT, kStages, kJvpMINB, kJvpUnr>, kJvpNT, JvpK::SMEM));
    if (JvpK::SMEM > 48 * 1024)
        CU(cudaFuncSetAttribute(ewald_jvp_f32x2_kernel<kJvpNT, kJvpIPT, kJvpJT, kStages, kEwJvpMinB>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, JvpK::SMEM));
    int occ_e = 0;   // the periodic JVP shares the plan: the smaller residency of the two
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ_e, ewald_jvp_f32x2_kernel<kJvpNT, kJvpIPT, kJvpJT, kStages, kEwJvpMinB>, kJvpNT, JvpK::SMEM));
    occ = std::min(occ, occ_e);
    if (occ < 1) return fail(ctx, COLATUS_E_CUDA, "JVP kernel cannot be resident");
    t.B = B;
    t.nchunk = (B + kTB - 1) / kTB;
    t.n_pad = round_up(ctx->N, std::max(JvpK::ITILE, kJvpJT));
    // units over all chunks' (i-tile x j-tile) pairs
    auto jvp_launch = [&](int sms) {
        ForceLaunch L{};
        L.n_it = (int)(t.n_pad / JvpK::ITILE);
        L.n_jt = (int)(t.n_pad / kJvpJT);
        L.W = (long long)t.nchunk * L.n_it * L.n_jt;
        L.G = (int)std::max(1LL, std::min<long long>((long long)occ * sms, L.W));
        long long smax = 1;
        for (long long ct = 0; ct < (long long)t.nchunk * L.n_it; ++ct)
            smax = std::max(smax, sk_owner((ct + 1) * L.n_jt - 1, L.W, L.G) -
                                      sk_owner(ct * L.n_jt, L.W, L.G) + 1);
        L.S_max = (int)smax;
        return L;
    };
    t.plan.L = jvp_launch(std::max(1, ctx->num_sms - 1));   // one SM for the schedule kernel
    t.plan.itile = JvpK::ITILE;
    t.plan.jt = kJvpJT;
    t.plan.n_pad = t.n_pad;
    t.plan.part_bytes = (size_t)t.nchunk * t.plan.L.n_it * t.plan.L.S_max * kTPlanes * JvpK::ITILE *
                        sizeof(float4);
    const size_t tb = (size_t)B * t.n_pad * sizeof(float4);
    CU(cudaMalloc(&t.dx, tb));
    CU(cudaMalloc(&t.dv, tb));
    CU(cudaMalloc(&t.dvh, tb));
    CU(cudaMalloc(&t.pkt, (size_t)t.nchunk * t.n_pad * kPktSlots * sizeof(float)));
    CU(cudaMalloc(&t.seeds, B * sizeof(long long)));
    CU(cudaMalloc(&t.growth, (size_t)capacity_steps * B * sizeof(float)));
    CU(cudaMemset(t.dx, 0, tb));
    CU(cudaMemset(t.dv, 0, tb));
    CU(cudaMemset(t.dvh, 0, tb));
    std::vector<long long> sd(seeds, seeds + B);
    CU(cudaMemcpy(t.seeds, sd.data(), B * sizeof(long long), cudaMemcpyHostToDevice));
    const float4 unit = make_float4((float)d[0], (float)d[1], (float)d[2], 0.f);
    for (int b = 0; b < B; ++b)
        CU(cudaMemcpy(t.dx + (size_t)b * t.n_pad + seeds[b], &unit, sizeof(unit), cudaMemcpyHostToDevice));
    for (int c = 0; c < 3; ++c) t.dir[c] = d[c];
    t.cap = capacity_steps;
    t.base = ctx->host_step;
    t.last_step = ctx->host_step;
    t.ready = true;
    t.open = false;
    return COLATUS_OK;
}

colatus_status colatus_tangent_step(colatus_t ctx, double dt, int64_t nsteps) {
    NvtxRange nvtx_("colatus_tangent_step");
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    auto &t = ctx->tan;
    if (!t.ready) return fail(ctx, COLATUS_E_STATE, "colatus_tangent_init first");
    if (ctx->prec == COLATUS_FP64)
        return fail(ctx, COLATUS_E_ARG, "the tangent model runs with FP32 precision");
    if (t.last_step != ctx->host_step)
        return fail(ctx, COLATUS_E_STATE, "the state moved without its tangents; re-initialise");
    if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) return fail(ctx, COLATUS_E_ARG, "bad dt/nsteps");
    if (nsteps == 0) return COLATUS_OK;
    // KDK: the half kick dvh belongs to one step size; a new one re-opens
    // from the tangent at the state's step (dx, dv), as the state does
    const bool kdk = is_kdk(ctx);
    if (t.open && (t.tau != dt || !kdk)) t.open = false;
    if (ctx->spec_valid && ctx->spec_tau != dt) ctx->spec_valid = false;
    const TangentState T = tan_state(ctx);
    dim3 grid(blocks_for(ctx->N, 256), t.nchunk);
    for (int64_t done = 0; done < nsteps;) {
        const int n = (int)std::min<int64_t>(kChunk, nsteps - done);
        TRY(need_table(ctx, dt, n, kTabPiece));
        if (kdk && !t.open) {
            // KDK tangent opening at x^n: JVP on the packed state positions
            const ForcePlan &p = plan_f32(ctx);
            pack_f32_kernel<<<blocks_for(p.n_pad, 256), 256, 0, ctx->stream>>>(ctx->xs, ctx->pk[2],
                                                                               ctx->N, p.n_pad);
            TRY(launched(ctx));
            TRY(run_jvp(ctx, ctx->pk[2], TAN_AT_STATE, 0.f));
            tan_open_kernel<<<grid, 256, 0, ctx->stream>>>(static_cast<const float4 *>(ctx->part),
                                                           t.plan.L, t.plan.itile, T, ctx->table,
                                                           kTabCap, ctx->host_step, ctx->N, t.n_pad,
                                                           tan_extra(ctx));
            TRY(launched(ctx));
            t.open = true;
            t.tau = dt;
        }
        if (!ctx->spec_valid) {
            TRY(open_step(ctx, dt));
            ctx->spec_valid = true;
            ctx->spec_tau = dt;
        }
        for (int j = 0; j < n; ++j) {
            // the step's force input pk[c] (x^{n+1} for KDK, x^{n+1/2} for
            // DKD) is also the JVP's; one_step writes the next into pk[c ^ 1]
            const int c = ctx->cur;
            TRY(wait_table_at(ctx, j, n));
            TRY(one_step(ctx, j, dt));
            if (kdk) {
                TRY(run_jvp(ctx, ctx->pk[c], TAN_KDK_DRIFT, (float)dt));
                tan_step_kernel<<<grid, 256, 0, ctx->stream>>>(
                    static_cast<const float4 *>(ctx->part), t.plan.L, t.plan.itile, T, ctx->table, kTabCap,
                    ctx->host_step + j, dt, ctx->N, t.n_pad, tan_extra(ctx));
            } else {
                TRY(run_jvp(ctx, ctx->pk[c], TAN_DKD_HALF, (float)(0.5 * dt)));
                tan_dkd_step_kernel<<<grid, 256, 0, ctx->stream>>>(
                    static_cast<const float4 *>(ctx->part), t.plan.L, t.plan.itile, T, ctx->table, kTabCap,
                    ctx->host_step + j, dt, ctx->N, t.n_pad, tan_extra(ctx));
            }
            TRY(launched(ctx));
        }
        done += n;
        ctx->host_step += n;
        TRY(refill_table(ctx));
    }
    ctx->acc_valid = true;
    t.last_step = ctx->host_step;
    return COLATUS_OK;
}

colatus_status colatus_tangent_read(colatus_t ctx, float *growth, int64_t *nrec_out) {
    if (!ctx || !nrec_out) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    auto &t = ctx->tan;
    TRY(sync_and_check(ctx));
    if (!t.ready) {
        *nrec_out = 0;
        return COLATUS_OK;
    }
    const long long total = t.last_step - t.base;
    const long long nrec = std::min(total, t.cap);
    *nrec_out = nrec;
    if (!growth || nrec == 0) return COLATUS_OK;
    std::vector<float> ring((size_t)t.cap * t.B);
    CU(cudaMemcpy(ring.data(), t.growth, ring.size() * sizeof(float), cudaMemcpyDeviceToHost));
    for (long long k = 0; k < nrec; ++k) {
        const long long s = total - nrec + k;
        std::memcpy(growth + k * t.B, ring.data() + (s % t.cap) * t.B, t.B * sizeof(float));
    }
    return COLATUS_OK;
}

colatus_status colatus_set_tuning(colatus_t ctx, int shape) {
    if (!ctx) return COLATUS_E_ARG;
    if (shape < -1 || shape >= kShapes) return fail(ctx, COLATUS_E_ARG, "shape must be -1 .. %d", kShapes - 1);
    if (shape >= 0) {
        const ForcePlan &p = ctx->plan32[4 * shape];
        if (!p.fits) return fail(ctx, COLATUS_E_ARG, "shape %d does not fit N", shape);
    }
    ctx->tuned_shape = shape;
    return COLATUS_OK;
}

colatus_status colatus_autotune(colatus_t ctx, int reps, double out_ms[4], int *chosen) {
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    if (ctx->periodic) return fail(ctx, COLATUS_E_STATE, "%s is not built for periodic boundaries", "autotuning");
    if (reps < 1) return fail(ctx, COLATUS_E_ARG, "reps must be >= 1");
    if (!ctx->have_state) return fail(ctx, COLATUS_E_STATE, "no state has been set");
    if (ctx->prec == COLATUS_FP64) return fail(ctx, COLATUS_E_ARG, "the tuned kernels are FP32");
    TRY(sync_and_check(ctx));
    const int keep = ctx->tuned_shape;
    const bool prof = ctx->profiling;
    const size_t used = ctx->ev_used;
    double best = 0.0;
    int best_sh = -1;
    for (int sh = 0; sh < kShapes; ++sh) {
        if (out_ms) out_ms[sh] = 0.0;
        if (!ctx->plan32[4 * sh].fits) continue;   // does not fit
        ctx->tuned_shape = sh;
        TRY(force_at_state(ctx));                   // warm-up launch
        ctx->profiling = true;
        ctx->ev_used = used;
        for (int r = 0; r < reps; ++r) TRY(force_at_state(ctx));
        CU(cudaStreamSynchronize(ctx->stream));
        double ms = 0.0;
        for (size_t k = used; k + 1 < ctx->ev_used; k += 2) {
            float e = 0.f;
            CU(cudaEventElapsedTime(&e, ctx->ev_pool[k], ctx->ev_pool[k + 1]));
            ms += e;
        }
        ms /= reps;
        ctx->profiling = prof;
        ctx->ev_used = used;
        if (out_ms) out_ms[sh] = ms;
        if (best_sh < 0 || ms < best) {
            best = ms;
            best_sh = sh;
        }
    }
    ctx->profiling = prof;
    ctx->ev_used = used;
    ctx->tuned_shape = best_sh >= 0 ? best_sh : keep;
    ctx->spec_valid = false;   // the next step re-opens with the chosen kernel
    ctx->tan.open = false;   // the tangent's half kick too
    if (chosen) *chosen = ctx->tuned_shape;
    return sync_and_check(ctx);
}

colatus_status colatus_probe_pipes(double out[6]) {
    colatus_t ctx = nullptr;
    if (!out) return fail(nullptr, COLATUS_E_ARG, "out is NULL");
    int dev = 0, nsm = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256, per_sm = 4, iters = 4096;
    const int blocks = nsm * per_sm;
    float *sink = nullptr;
    long long *cyc = nullptr;
    CU(cudaMalloc(&sink, threads * sizeof(float)));
    CU(cudaMalloc(&cyc, blocks * sizeof(long long)));
    std::vector<long long> h(blocks);
    colatus_status st = COLATUS_OK;
    for (int kind = 0; kind < 3 && st == COLATUS_OK; ++kind) {
        cudaMemset(cyc, 0, blocks * sizeof(long long));
        for (int rep = 0; rep < 2; ++rep) {   // the second run is timed (warm)
            cudaMemset(cyc, 0, blocks * sizeof(long long));
            if (kind == 0) probe_pipe_kernel<0><<<blocks, threads>>>(iters, 0.5f, sink, cyc);
            if (kind == 1) probe_pipe_kernel<1><<<blocks, threads>>>(iters, 0.5f, sink, cyc);
            if (kind == 2) probe_pipe_kernel<2><<<blocks, threads>>>(iters, 0.5f, sink, cyc);
        }
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(h.data(), cyc, blocks * sizeof(long long), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            st = fail(nullptr, COLATUS_E_CUDA, "probe: %s", cudaGetErrorString(e));
            break;
        }
        long long mx = 1;
        for (long long c : h) mx = std::max(mx, c);
        const double lanes = (double)per_sm * threads * iters * kProbeChains * (kind == 1 ? 2.0 : 1.0);
        out[kind] = lanes / (double)mx;
    }
    cudaFree(sink);
    cudaFree(cyc);
    out[3] = nsm;
    out[4] = per_sm;
    out[5] = 0.0;
    return st;
}

colatus_status colatus_selftest_wait(colatus_t ctx, int64_t limit_cycles) {
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    if (limit_cycles < 1 || limit_cycles > kWaitCycles)
        return fail(ctx, COLATUS_E_ARG, "limit_cycles must be in [1, %lld]", kWaitCycles);
    TRY(sync_and_check(ctx));
    wait_selftest_kernel<<<1, 32, 0, ctx->stream>>>(ctx->flags, limit_cycles);
    TRY(launched(ctx));
    return sync_and_check(ctx);
}

colatus_status colatus_set_periodic(colatus_t ctx, double L, double alpha, int nk) {
    if (!ctx) return COLATUS_E_ARG;
    DeviceGuard dg(ctx->device);
    if (L == 0.0) {
        if (ctx->periodic) {
            ctx->periodic = false;
            ctx->acc_valid = ctx->spec_valid = false;
            ctx->tan.open = false;   // the tangent's half kick too
        }
        return COLATUS_OK;
    }
    if (!(L > 0.0) || !std::isfinite(L)) return fail(ctx, COLATUS_E_ARG, "L must be finite and > 0");
    if (!std::isfinite(alpha)) return fail(ctx, COLATUS_E_ARG, "alpha must be finite");
    if (nk > kEwMaxNk) return fail(ctx, COLATUS_E_ARG, "nk must be <= %d", kEwMaxNk);
    if (ctx->defo_C != 0.0)
        return fail(ctx, COLATUS_E_ARG, "periodic boundaries do not combine with the deformation term");
    ctx->box = L;
    ctx->ew_alpha_req = alpha;
    ctx->ew_nk_req = nk;
    ctx->periodic = true;
    colatus_status st = ewald_setup(ctx);
    if (st != COLATUS_OK) ctx->periodic = false;
    ctx->acc_valid = ctx->spec_valid = false;
    ctx->tan.open = false;
    ctx->adj.ready = false;
    return st;
}

colatus_status colatus_periodic_params(colatus_t ctx, double *alpha_out, int *nk_out, int *nkv_out) {
    if (!ctx) return COLATUS_E_ARG;
    if (!ctx->periodic) return fail(ctx, COLATUS_E_STATE, "boundaries are not periodic");
    if (alpha_out) *alpha_out = ctx->ew.alpha;
    if (nk_out) *nk_out = ctx->ew.nk;
    if (nkv_out) *nkv_out = ctx->nkv;
    return COLATUS_OK;
}

colatus_status colatus_set_deformation(colatus_t ctx, double Cpsi, const double *x_psi) {
    if (!ctx) return COLATUS_E_ARG;
    if (!std::isfinite(Cpsi)) return fail(ctx, COLATUS_E_ARG, "C psi must be finite");
    if (Cpsi != 0.0) {
        if (!x_psi) return fail(ctx, COLATUS_E_ARG, "x_psi is NULL");
        for (int c = 0; c < 3; ++c)
            if (!std::isfinite(x_psi[c])) return fail(ctx, COLATUS_E_ARG, "x_psi must be finite");
        if (ctx->G == 0.0) return fail(ctx, COLATUS_E_ARG, "the deformation term needs G != 0");
        if (ctx->periodic)
            return fail(ctx, COLATUS_E_ARG, "the deformation term does not combine with periodic boundaries");
        for (int c = 0; c < 3; ++c) ctx->defo_x[c] = x_psi[c];
    }
    ctx->defo_C = Cpsi;
    ctx->acc_valid = false;
    ctx->spec_valid = false;
    ctx->tan.open = false;
    return COLATUS_OK;
}

const char *colatus_last_error(colatus_t ctx) { return ctx ? ctx->err : g_init_err; }

void colatus_destroy(colatus_t ctx) {
    if (!ctx) return;
    {
        DeviceGuard dg(ctx->device);
        // the schedule and read-back streams may still run work that uses the buffers
        if (ctx->stream) cudaStreamSynchronize(ctx->stream);
        if (ctx->tstream) cudaStreamSynchronize(ctx->tstream);
        if (ctx->cstream) cudaStreamSynchronize(ctx->cstream);
        free_all(ctx);
    }
    delete ctx;
}

colatus_status colatus_force_plan(colatus_t ctx, int64_t out[9]) {
    if (!ctx || !out) return COLATUS_E_ARG;
    const bool f64 = ctx->prec == COLATUS_FP64;
    const ForcePlan &p = f64 ? plan_f64(ctx) : plan_f32(ctx);
    out[0] = (ctx->periodic ? 2 : 0) + (f64 ? 1 : 0);
    if (!f64 && !ctx->periodic && f32_variant(p.variant).sym) out[0] = 4;
    if (!f64 && ctx->periodic && p.L.sym) out[0] = 5;
    if (f64) {
        out[1] = ctx->periodic ? kEw64NT : kF64NT;
        out[2] = ctx->periodic ? 1 : kF64IPT;
        out[4] = 0;
        out[5] = 0;
    } else if (ctx->periodic) {
        out[1] = p.L.sym ? kEwSymNT : kEwNT;
        out[2] = p.L.sym ? kEwSymIPT : kEwIPT;
        out[4] = ctx->prec == COLATUS_FP32_COMP ? 1 : 0;
        out[5] = ctx->eq_mass && p.n_pad == ctx->N ? 1 : 0;
    } else {
        const F32Variant &fv = f32_variant(p.variant);
        out[1] = fv.nt;
        out[2] = fv.ipt;
        out[4] = fv.comp ? 1 : 0;
        out[5] = fv.eqm ? 1 : 0;
    }
    out[3] = p.jt;
    out[6] = p.L.G;
    out[7] = p.L.W;
    out[8] = f64 || ctx->periodic ? 0 : f32_variant(p.variant).nrcp;
    return COLATUS_OK;
}

colatus_status colatus_vjp_plan(colatus_t ctx, int64_t out[6]) {
    if (!ctx || !out) return COLATUS_E_ARG;
    const bool f64 = ctx->prec == COLATUS_FP64;
    const ForcePlan &p0 = vjp_plan(ctx);
    const bool eqm = ctx->scheme != COLATUS_DKD && !f64 && ctx->eq_mass && !ctx->periodic &&
                     ctx->defo_C == 0.0 && p0.n_pad == ctx->N;
    const ForcePlan &p = vjp_plan(ctx, eqm);
    if (ctx->periodic && !f64 && p.L.sym) {
        out[0] = 7;
        out[1] = kVjpGenNT;
        out[2] = VjpGenK::IPT;
    } else if (ctx->periodic) {
        out[0] = f64 ? 3 : 2;
        out[1] = f64 ? kEwV64NT : kEwVjpNT;
        out[2] = f64 ? 1 : kEwVjpIPT;
    } else if (f64) {
        out[0] = 1;
        out[1] = kV64NT;
        out[2] = 1;
    } else if (eqm && p.L.sym) {
        out[0] = 5;
        out[1] = kVjpSymNT;
        out[2] = VjpSymK::IPT;
    } else if (p.L.sym) {
        out[0] = 6;
        out[1] = kVjpGenNT;
        out[2] = VjpGenK::IPT;
    } else {
        out[0] = eqm ? 4 : 0;
        out[1] = kVjpNT;
        out[2] = kVjpIPT;
    }
    out[3] = p.jt;
    out[4] = p.L.G;
    out[5] = p.L.W;
    return COLATUS_OK;
}

colatus_status colatus_stats(colatus_t ctx, double out[4]) {
    if (!ctx || !out) return COLATUS_E_ARG;
    out[0] = (double)ctx->launches;
    out[1] = ctx->interactions;
    out[2] = (double)ctx->host_step;
    out[3] = (double)ctx->N;
    return COLATUS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- ensembles
#include "ensemble_api.cuh"
#include "spectrum_api.cuh"
#include "selftest_api.cuh"
