// ensemble.cuh -- many independent realisations of Eqs. 1-5 (uneven N) in one
// persistent launch per step.
//
// Realisation r holds N_r bodies, padded with zero-mass bodies to a multiple
// of the tile size and stored contiguously (pair-interleaved FP32, as in
// force.cuh).  Its interaction matrix is cut into i-tile x j-tile units; the
// units of all realisations are concatenated into one work list, which a
// persistent grid splits into equal contiguous ranges (stream-K), so the load
// is balanced whatever the mix of N_r.  Softening is per realisation.  The
// j-tiles of a unit never cross a realisation boundary, so realisations never
// interact.
//
// Padding bodies have zero mass and sit at (2^100, 2^100, 2^100): the squared
// distance from any body at moderate coordinates overflows to +inf, rsqrt
// gives 0 and the pair term is exactly 0 in either form of the pair sum,
// including the equal-mass form that never reads the mass.  When every
// realisation has equal masses, the kernel takes that form (one FP32 lane-op
// fewer per interaction) and the epilogues multiply the sums by m_r.
#pragma once

#include "common.cuh"
#include "force.cuh"
#include "force_sym.cuh"
#include "sym_reduce.cuh"
#include "integrate.cuh"

namespace colatus {

struct EnsLaunch {
    long long W;                    // total units
    int R;                          // realisations
    int G;                          // CTAs
    int S_max;                      // max segments of any i-tile
    int T;                          // total i-tiles
    const long long *unit_off;      // [R+1] first unit of realisation r
    const long long *body_off;      // [R+1] first (padded) body of realisation r
    const long long *nbody;         // [R]   real bodies of realisation r
    const int *n_jt;                // [R]   j-tiles per i-tile of realisation r
    const float *eps2;              // [R]   softening^2
    const int *tile_r;              // [T]   realisation of global i-tile t
    const long long *tile_u0;       // [T]   first unit of global i-tile t
    const float *meq;               // [R]   equal mass of realisation r (equal-mass kernel), or null
    // the pair-once plan (ens_sym.cuh) only, else null / 0: its tables and
    // the float4 offset of its column slots in the segment buffer
    const int *sym;
    long long sym_col_off;
};

constexpr int kEnsSymT = 512;   // bodies per tile of the pair-once plan


constexpr float kEnsFar = 0x1p100f;   // coordinate of the padding bodies

// Realisation containing unit u (binary search over unit_off).
__device__ __forceinline__ int ens_find(const long long *off, int R, long long u) {
    int lo = 0, hi = R;   // off[lo] <= u < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= u)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Body index of the first j-body of unit u in realisation r.
__device__ __forceinline__ long long ens_jbody(const EnsLaunch &E, int r, long long u, int JT) {
    const long long local = u - E.unit_off[r];
    return E.body_off[r] + (local % E.n_jt[r]) * JT;
}

template <int NT, int IPT, int JT, int STAGES, int FOLD, int MINB, bool EQM, int NRCP = 0>
__global__ void __launch_bounds__(NT, MINB)
    ens_force_kernel(const float *__restrict__ pk, float4 *__restrict__ part, int *__restrict__ flags,
                     EnsLaunch E) {
    using K = F32Kernel<NT, IPT, JT, STAGES, FOLD, false, EQM>;
    extern __shared__ __align__(128) unsigned char smem[];
    float4 *tiles = reinterpret_cast<float4 *>(smem);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * K::TILE_BYTES);

    const int tid = threadIdx.x;
    const long long G = gridDim.x, g = blockIdx.x;
    const long long u0 = sk_begin(g, E.W, G), u1 = sk_begin(g + 1, E.W, G);

    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
    }
    __syncthreads();
    // producer cursor (thread 0): realisation of the next unit to fetch
    int rp = 0;
    if (tid == 0) {
        rp = ens_find(E.unit_off, E.R, u0);
        for (int s = 0; s < STAGES && u0 + s < u1; ++s) {
            while (u0 + s >= E.unit_off[rp + 1]) ++rp;
            mbar_arrive_expect_tx(&full[s], K::TILE_BYTES);
            bulk_load(tiles + s * JT, pk + ens_jbody(E, rp, u0 + s, JT) * 4, K::TILE_BYTES, &full[s]);
        }
    }
    int r = ens_find(E.unit_off, E.R, u0);
    long long u = u0;
    bool bad = false;
    int stage = 0;
    uint32_t parity = 0;
    while (u < u1) {
        while (u >= E.unit_off[r + 1]) ++r;
        const int njt = E.n_jt[r];
        const long long local = u - E.unit_off[r];
        const long long it = local / njt;
        const long long uend = min(u1, E.unit_off[r] + (it + 1) * (long long)njt);
        const long long ibase = E.body_off[r] + it * K::ITILE;
        const float eps2 = E.eps2[r];
        const float2 e2 = make_float2(eps2, eps2);
        float2 nx[IPT], ny[IPT], nz[IPT];
        float hx[IPT], hy[IPT], hz[IPT], lx[IPT], ly[IPT], lz[IPT];
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const long long i = ibase + tid + k * NT;
            const float *p = pk + (i >> 1) * 8 + (i & 1);
            const float x = __ldg(p), y = __ldg(p + 2), z = __ldg(p + 4);
            nx[k] = make_float2(-x, -x);
            ny[k] = make_float2(-y, -y);
            nz[k] = make_float2(-z, -z);
            hx[k] = hy[k] = hz[k] = 0.f;
            lx[k] = ly[k] = lz[k] = 0.f;
        }
        for (; u < uend; ++u) {
            const bool ok = mbar_wait_bounded(&full[stage], parity);
            if (ok)
                f32_tile<IPT, JT, FOLD, false, EQM, 2, NRCP>(tiles + stage * JT, nx, ny, nz, e2, hx, hy,
                                                          hz, lx, ly, lz);
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
            if (tid == 0 && u + STAGES < u1) {
                const long long un = u + STAGES;
                while (un >= E.unit_off[rp + 1]) ++rp;
                mbar_arrive_expect_tx(&full[stage], K::TILE_BYTES);
                bulk_load(tiles + stage * JT, pk + ens_jbody(E, rp, un, JT) * 4, K::TILE_BYTES,
                          &full[stage]);
            }
            if (++stage == STAGES) {
                stage = 0;
                parity ^= 1u;
            }
        }
        if (bad) break;
        const long long t = ibase / K::ITILE;   // global i-tile
        const long long sidx = g - sk_owner(E.tile_u0[t], E.W, G);
        float4 *dst = part + (t * E.S_max + sidx) * (long long)K::ITILE;
#pragma unroll
        for (int k = 0; k < IPT; ++k) dst[tid + k * NT] = make_float4(hx[k], hy[k], hz[k], 0.f);
    }
    if (bad && tid == 0) {
        atomicOr(&flags[FLAG_TIMEOUT], 1);
        for (long long v = u; v < u1 && v < u + STAGES; ++v) {
            mbar_wait_bounded(&full[stage], parity);
            if (++stage == STAGES) {
                stage = 0;
                parity ^= 1u;
            }
        }
    }
}

// Int tables of the ensemble's pair-once plan (EnsLaunch::sym):
//   [0] R, [1] NW, [2] U tile pairs in all, [3] G CTAs, [4] TT tiles in all,
//   [kSymHdr ...] ub[R + 1] (first tile pair of realisation r),
//                 tb[R + 1] (first tile of realisation r),
//                 row_g0[TT], row_ns[TT], col_start[TT + 1], unit_g0[U],
//                 unit_ko[U], unit_nk[U], cta_pu[G + 1]
// with the meanings of force_sym.cuh, tiles and tile pairs numbered over all
// realisations (the column slots on the bodies of global tile t are the run
// [col_start[t], col_start[t + 1])).
struct EnsSymTab {
    const int *ub, *tb, *row_g0, *row_ns, *col_start, *unit_g0, *unit_ko, *unit_nk, *cta_pu;
    int R, NW, U, G, TT;
    __host__ __device__ explicit EnsSymTab(const int *t) {
        R = t[0];
        NW = t[1];
        U = t[2];
        G = t[3];
        TT = t[4];
        ub = t + kSymHdr;
        tb = ub + R + 1;
        row_g0 = tb + R + 1;
        row_ns = row_g0 + TT;
        col_start = row_ns + TT;
        unit_g0 = col_start + TT + 1;
        unit_ko = unit_g0 + U;
        unit_nk = unit_ko + U;
        cta_pu = unit_nk + U;
    }
};

// Epilogue side: the (G-less, mass-free for EQM) force sum of body i (global
// padded index, realisation r) of the pair-once plan with tiles of T bodies:
// the row segments of its tile, then the column slots on its tile, in that
// fixed order.
__device__ __forceinline__ float3 ens_reduce_sym(const float4 *__restrict__ part, const EnsLaunch &E, int r,
                                                 long long i, int T) {
    const EnsSymTab S(E.sym);
    const long long l = i - E.body_off[r];
    const int t = (int)(l / T), il = (int)(l - (long long)t * T);
    const int gt = S.tb[r] + t;
    float fx = 0.f, fy = 0.f, fz = 0.f, lx = 0.f, ly = 0.f, lz = 0.f;
    sym_sum_run<false>(part + (long long)gt * E.S_max * T + il, T, S.row_ns[gt], 0, fx, fy, fz, lx, ly, lz);
    const int k0 = S.col_start[gt];
    sym_sum_run<false>(part + E.sym_col_off + (long long)k0 * T + il, T, S.col_start[gt + 1] - k0, 0, fx, fy,
                       fz, lx, ly, lz);
    return make_float3(fx, fy, fz);
}

// Segment sum of body i (global padded index) in CTA order.
__device__ __forceinline__ float3 ens_reduce(const float4 *__restrict__ part, const EnsLaunch &E,
                                             int itile, long long i) {
    const long long t = i / itile, il = i - t * itile;
    const int r = E.tile_r[t];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    if (E.sym) {
        const float3 f = ens_reduce_sym(part, E, r, i, kEnsSymT);   // each pair evaluated once
        fx = f.x;
        fy = f.y;
        fz = f.z;
    } else {
        const long long g0 = sk_owner(E.tile_u0[t], E.W, E.G);
        const long long g1 = sk_owner(E.tile_u0[t] + E.n_jt[r] - 1, E.W, E.G);
        const float4 *p = part + t * E.S_max * (long long)itile + il;
        for (long long s = 0; s <= g1 - g0; ++s) {
            const float4 v = __ldg(p + s * itile);
            fx += v.x;
            fy += v.y;
            fz += v.z;
        }
    }
    if (E.meq) {
        const float m = E.meq[r];
        fx *= m;
        fy *= m;
        fz *= m;
    }
    return make_float3(fx, fy, fz);
}

// Is padded body i a real body of its realisation?
__device__ __forceinline__ bool ens_real(const EnsLaunch &E, int itile, long long i) {
    const int r = E.tile_r[i / itile];
    return i - E.body_off[r] < E.nbody[r];
}

// Schedule of n steps from the clock (not advanced here; the step epilogue
// advances it): entry j of `table` is step j of the chunk.  The same
// sequence as the single-system schedule (friedmann_table_kernel): DKD's
// (c, d) at t^{n+1/2}, KDK's half kicks at t^n and t^{n+1}, or with
// canonical != 0 the canonical leapfrog's (c1, d1, c2, d2) from the
// integrals of dt/a and dt/a^2.
__global__ void ens_table_kernel(Cosmo cosmo, const DevClock *clk, StepCoef *table, int n,
                                 double tau, double G, int nsub, int canonical) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double a = clk->a, t = clk->t;
    const long long step0 = clk->step;
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
        table[j] = s;
        a = s.a1;
    }
}

// Packing of the (real) state into the force input; padding is zero-mass and far away.
__global__ void ens_pack_kernel(const float4 *__restrict__ xs, float *__restrict__ pk, EnsLaunch E,
                                int itile, long long Npad) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= Npad) return;
    if (ens_real(E, itile, i)) {
        const float4 b = xs[i];
        pk_store(pk, i, b.x, b.y, b.z, b.w);
    } else {
        pk_store(pk, i, kEnsFar, kEnsFar, kEnsFar, 0.f);
    }
}

// F (G-less) of every body into acc; out (optional, real bodies only, in the
// user's concatenated order via `user`) = G a^-3 F.
__global__ void ens_forces_out_kernel(const float4 *__restrict__ part, EnsLaunch E, int itile,
                                      long long Npad, float4 *__restrict__ acc) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= Npad) return;
    const float3 f = ens_reduce(part, E, itile, i);
    acc[i] = make_float4(f.x, f.y, f.z, 0.f);
}

// KDK opening for every body: vh = c1 v + d1 F;  x' = x + tau vh (packed).
__global__ void ens_open_kernel(const float4 *__restrict__ xs, const float4 *__restrict__ vs,
                                const float4 *__restrict__ acc, float4 *__restrict__ vh,
                                float *__restrict__ pk_out, const StepCoef *__restrict__ table,
                                double tau, EnsLaunch E, int itile, long long Npad, int dkd) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= Npad) return;
    if (!ens_real(E, itile, i)) {
        pk_store(pk_out, i, kEnsFar, kEnsFar, kEnsFar, 0.f);
        return;
    }
    const float4 x = xs[i], v = vs[i];
    if (dkd) {   // DKD opening: the half drift, no force
        const float h = (float)(0.5 * tau);
        pk_store(pk_out, i, drift1(x.x, h, v.x), drift1(x.y, h, v.y), drift1(x.z, h, v.z), x.w);
        return;
    }
    const float c1 = (float)table[0].c1, d1 = (float)table[0].d1, t = (float)tau;
    const float4 F = acc[i];
    const float hx = kick2(c1, v.x, d1, F.x), hy = kick2(c1, v.y, d1, F.y), hz = kick2(c1, v.z, d1, F.z);
    vh[i] = make_float4(hx, hy, hz, 0.f);
    pk_store(pk_out, i, drift1(x.x, t, hx), drift1(x.y, t, hy), drift1(x.z, t, hz), x.w);
}

// KDK step j of a chunk after the force at x^{n+1} (pk_in): close the step
// with (c2, d2), open the next one with (c1, d1) of entry j + 1 when
// `next_entry` (the canonical scheme; the chunk's schedule then holds one
// entry more) or else (c2, d2) again, which for the drag scheme are the same
// numbers: both are the half kick at t^{n+1}.
__global__ void ens_step_kernel(const float4 *__restrict__ part, EnsLaunch E, int itile,
                                const float *__restrict__ pk_in, float4 *__restrict__ xs,
                                float4 *__restrict__ vs, float4 *__restrict__ vh,
                                float4 *__restrict__ acc, float *__restrict__ pk_out,
                                const StepCoef *__restrict__ table, int j, double tau,
                                long long Npad, int *flags, DevClock *clk, Tracers tr, int next_entry) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= Npad) return;
    const StepCoef &sc = table[j];
    if (i == 0) advance_clock(clk, sc, flags);
    if (!ens_real(E, itile, i)) {
        pk_store(pk_out, i, kEnsFar, kEnsFar, kEnsFar, 0.f);
        return;
    }
    const float c2 = (float)sc.c2, d2 = (float)sc.d2, t = (float)tau;
    const float c1n = next_entry ? (float)table[j + 1].c1 : c2, d1n = next_entry ? (float)table[j + 1].d1 : d2;
    const float3 F = ens_reduce(part, E, itile, i);
    const float4 x = pk_load(pk_in, i);
    const float4 h = vh[i];
    const float vx = kick2(c2, h.x, d2, F.x), vy = kick2(c2, h.y, d2, F.y), vz = kick2(c2, h.z, d2, F.z);
    acc[i] = make_float4(F.x, F.y, F.z, 0.f);
    xs[i] = x;
    vs[i] = make_float4(vx, vy, vz, 0.f);
    record(tr, i, sc.step, x.x, x.y, x.z, vx, vy, vz);   // tr.slot is indexed by padded body
    const float nx = kick2(c1n, vx, d1n, F.x), ny = kick2(c1n, vy, d1n, F.y), nz = kick2(c1n, vz, d1n, F.z);
    vh[i] = make_float4(nx, ny, nz, 0.f);
    pk_store(pk_out, i, drift1(x.x, t, nx), drift1(x.y, t, ny), drift1(x.z, t, nz), x.w);
    if (!finite3(x.x, x.y, x.z) || !finite3(vx, vy, vz)) atomicOr(&flags[FLAG_NONFINITE], 1);
}

// DKD step j of a chunk (Eqs. 3-5; c, d at t^{n+1/2}) after the force at
// the half-drift positions x^{n+1/2} (pk_in): kick, second half drift,
// record, and the next step's half drift into pk_out.
__global__ void ens_dkd_step_kernel(const float4 *__restrict__ part, EnsLaunch E, int itile,
                                    const float *__restrict__ pk_in, float4 *__restrict__ xs,
                                    float4 *__restrict__ vs, float4 *__restrict__ acc,
                                    float *__restrict__ pk_out, const StepCoef *__restrict__ table, int j,
                                    double tau, long long Npad, int *flags, DevClock *clk, Tracers tr) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= Npad) return;
    const StepCoef &sc = table[j];
    if (i == 0) advance_clock(clk, sc, flags);
    if (!ens_real(E, itile, i)) {
        pk_store(pk_out, i, kEnsFar, kEnsFar, kEnsFar, 0.f);
        return;
    }
    const float c = (float)sc.c, d = (float)sc.d, h = (float)(0.5 * tau);
    const float3 F = ens_reduce(part, E, itile, i);
    const float4 xh = pk_load(pk_in, i);
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

}  // namespace colatus
