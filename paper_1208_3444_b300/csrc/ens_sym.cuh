// ens_sym.cuh -- the ensemble's force with every pair evaluated once.
//
// Each realisation is cut into tiles of T = IPT NT bodies and its tile pairs
// (it, jt), it <= jt, are evaluated as in force_sym.cuh: symmetrically off the
// diagonal (one evaluation serves both bodies), for every ordered pair on the
// i side within a diagonal tile.  The tile pairs of all realisations are
// concatenated realisation by realisation into one work list of NW phases
// per pair, which a persistent grid splits by cost, so the load is balanced
// whatever the mix of N_r; softening is per realisation.
//
// Storage keeps the ensemble's 256-body padding, so a realisation's last tile
// may hold fewer valid (padded) bodies than T.  The bodies beyond are taken as
// the padding bodies are: at (2^100, 2^100, 2^100) with zero mass, in shared
// memory for the j side and in registers for the i side.  A pair with such a
// body has a squared distance that overflows to +inf, so rsqrt gives 0 and the
// term is exactly 0 in either form of the pair sum (two such bodies coincide
// and contribute 0 too).  Their partial sums are written but never read.
#pragma once

#include <algorithm>
#include <vector>

#include "ensemble.cuh"
#include "force_sym.cuh"

namespace colatus {

template <int NT>
struct EnsSymKernel {
    static constexpr int IPT = 4;
    static constexpr int NW = NT / 32;
    static constexpr int T = NT * IPT;        // bodies per tile
    static constexpr int TP = T / 2;          // j-pairs per tile
    static constexpr int SLICE = TP / NW;     // j-pairs per warp slice
    static constexpr int ROT = SLICE / 32;    // 32-round rotations per phase
    static constexpr uint32_t TILE_BYTES = T * 16;
    // staging tile, the two doubled halves, the column sums [x y z][TP] float2,
    // one mbarrier
    static constexpr int SMEM = TILE_BYTES + 2 * TILE_BYTES + 3 * TP * 8 + 16;
    static_assert(SLICE % 32 == 0 && T % 256 == 0, "whole rotations, whole 256-body padding tiles");
    static_assert(T == kEnsSymT, "the epilogues sum segments of kEnsSymT-body tiles");
};

// Realisation of a tile pair / tile (binary search over a first-index table).
__host__ __device__ __forceinline__ int ens_find_int(const int *off, int R, int u) {
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

// Persistent pair-once ensemble force kernel (FP32, plain sums).  pk: the
// ensemble's pair-interleaved bodies.  part: row segments [TT][S_max][T]
// float4, then from float4 offset E.sym_col_off the column slots [slot][T]
// float4 (negated when written, so both are forces on the bodies they index).
// EQM: every realisation has equal masses; the sums leave out m_r (the
// epilogues multiply by it).
template <int NT, int MINB, bool EQM, int UNR>
__global__ void __launch_bounds__(NT, MINB)
    ens_sym_force_kernel(const float *__restrict__ pk, float4 *__restrict__ part, int *__restrict__ flags,
                         EnsLaunch E) {
    using K = EnsSymKernel<NT>;
    constexpr int NW = K::NW, T = K::T, TP = K::TP, IPT = K::IPT;
    extern __shared__ __align__(128) unsigned char smem[];
    float4 *raw = reinterpret_cast<float4 *>(smem);   // staging: T float4 (pair-interleaved)
    float4 *sA = raw + T;                             // 2 TP float4: x0 x1 y0 y1, blocks doubled
    float4 *sB = sA + 2 * TP;                         // 2 TP float4: z0 z1 m0 m1, blocks doubled
    float2 *acc = reinterpret_cast<float2 *>(sB + 2 * TP);   // [3][TP]
    uint64_t *bar = reinterpret_cast<uint64_t *>(acc + 3 * TP);

    const EnsSymTab S(E.sym);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = blockIdx.x;
    int pu = S.cta_pu[g];
    const int pu_end = S.cta_pu[g + 1];
    if (pu >= pu_end) return;
    int u = pu / NW;
    int r = ens_find_int(S.ub, S.R, u);
    int nr = S.tb[r + 1] - S.tb[r];
    int it, jt;
    sym_decode(u - S.ub[r], nr, it, jt);
    // valid (stored) bodies of tile t of realisation rr
    auto valid = [&](int rr, int t) {
        const long long np = E.body_off[rr + 1] - E.body_off[rr];
        return (int)min((long long)T, np - (long long)t * T);
    };

    for (int q = tid; q < 3 * TP; q += NT) acc[q] = make_float2(0.f, 0.f);
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        const uint32_t bytes = (uint32_t)valid(r, jt) * 16u;
        mbar_arrive_expect_tx(bar, bytes);
        bulk_load(raw, pk + (E.body_off[r] + (long long)jt * T) * 4, bytes, bar);
    }
    bool inflight = true;

    float2 e2 = make_float2(E.eps2[r], E.eps2[r]);
    float2 nx[IPT], ny[IPT], nz[IPT], mi[IPT];
    float hx[IPT], hy[IPT], hz[IPT];
    auto load_i = [&](int rr, int row) {
        const long long np = E.body_off[rr + 1] - E.body_off[rr];
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const long long l = (long long)row * T + tid + k * NT;
            float x = kEnsFar, y = kEnsFar, z = kEnsFar, m = 0.f;
            if (l < np) {
                const long long i = E.body_off[rr] + l;
                const float *p = pk + (i >> 1) * 8 + (i & 1);
                x = __ldg(p);
                y = __ldg(p + 2);
                z = __ldg(p + 4);
                m = __ldg(p + 6);
            }
            nx[k] = make_float2(-x, -x);
            ny[k] = make_float2(-y, -y);
            nz[k] = make_float2(-z, -z);
            mi[k] = make_float2(m, m);
            hx[k] = hy[k] = hz[k] = 0.f;
        }
    };
    load_i(r, it);

    uint32_t parity = 0;
    bool bad = false;
    const PlummerPair::Args pa{};
    while (pu < pu_end) {
        const int uend = min(pu_end, (u + 1) * NW);
        const int p0 = pu - u * NW, p1 = uend - u * NW;
        const bool ok = mbar_wait_bounded(bar, parity);
        if (__syncthreads_or(!ok)) {
            bad = true;
            break;
        }
        inflight = false;
        parity ^= 1u;
        const int vq = valid(r, jt) / 2;   // j-pairs with stored bodies
        for (int q = tid; q < TP; q += NT) {
            const int e = 2 * q - (q & 31);   // entry of pair q in its doubled block
            float4 A = make_float4(kEnsFar, kEnsFar, kEnsFar, kEnsFar), B = make_float4(kEnsFar, kEnsFar, 0.f, 0.f);
            if (q < vq) {
                A = raw[2 * q];
                B = raw[2 * q + 1];
            }
            sA[e] = A;
            sA[e + 32] = A;
            sB[e] = B;
            sB[e + 32] = B;
        }
        __syncthreads();
        // the next tile pair: within the realisation's triangle, then the next realisation
        int r_n = r, it_n = it, jt_n = jt + 1;
        if (jt_n == nr) {
            ++it_n;
            jt_n = it_n;
            if (it_n == nr) {
                ++r_n;
                it_n = jt_n = 0;
            }
        }
        if (uend < pu_end) {
            if (tid == 0) {
                const uint32_t bytes = (uint32_t)valid(r_n, jt_n) * 16u;
                mbar_arrive_expect_tx(bar, bytes);
                bulk_load(raw, pk + (E.body_off[r_n] + (long long)jt_n * T) * 4, bytes, bar);
            }
            inflight = true;
        }
        const bool sym = jt != it;
        for (int p = p0; p < p1; ++p) {
            const int slice = (warp + p) % NW;
            float2 px[IPT], py[IPT], pz[IPT];
#pragma unroll
            for (int k = 0; k < IPT; ++k) px[k] = py[k] = pz[k] = make_float2(0.f, 0.f);
#pragma unroll 1
            for (int s = 0; s < K::ROT; ++s) {
                const int base = slice * K::SLICE + s * 32;
                const float4 *bA = sA + 2 * base, *bB = sB + 2 * base;
                float2 jx = make_float2(0.f, 0.f), jy = jx, jz = jx;
                if (sym) {
                    sym_rotation<PlummerPair, IPT, true, EQM, UNR>(bA, bB, lane, nx, ny, nz, mi, e2, pa, px, py,
                                                                   pz, jx, jy, jz);
                    const int q = base + lane;
                    acc[q] = __fadd2_rn(acc[q], jx);
                    acc[TP + q] = __fadd2_rn(acc[TP + q], jy);
                    acc[2 * TP + q] = __fadd2_rn(acc[2 * TP + q], jz);
                } else {
                    sym_rotation<PlummerPair, IPT, false, EQM, UNR>(bA, bB, lane, nx, ny, nz, mi, e2, pa, px,
                                                                    py, pz, jx, jy, jz);
                }
            }
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                hx[k] += px[k].x + px[k].y;
                hy[k] += py[k].x + py[k].y;
                hz[k] += pz[k].x + pz[k].y;
            }
            __syncthreads();   // the slices change hands
        }
        if (sym) {
            const int slot = S.unit_ko[u] + (g - S.unit_g0[u]);
            float4 *dst = part + E.sym_col_off + (long long)slot * T;
            for (int q = tid; q < TP; q += NT) {
                const float2 a = acc[q], b = acc[TP + q], c = acc[2 * TP + q];
                dst[2 * q] = make_float4(-a.x, -b.x, -c.x, 0.f);
                dst[2 * q + 1] = make_float4(-a.y, -b.y, -c.y, 0.f);
                acc[q] = acc[TP + q] = acc[2 * TP + q] = make_float2(0.f, 0.f);
            }
            __syncthreads();
        }
        pu = uend;
        ++u;
        if (r_n != r || it_n != it || pu == pu_end) {
            // the row segment of tile it of realisation r
            const int gt = S.tb[r] + it;
            const int sidx = g - S.row_g0[gt];
            float4 *dst = part + ((long long)gt * E.S_max + sidx) * T;
#pragma unroll
            for (int k = 0; k < IPT; ++k) dst[tid + k * NT] = make_float4(hx[k], hy[k], hz[k], 0.f);
            if (pu < pu_end) {
                if (r_n != r) {
                    nr = S.tb[r_n + 1] - S.tb[r_n];
                    e2 = make_float2(E.eps2[r_n], E.eps2[r_n]);
                }
                load_i(r_n, it_n);
            }
        }
        r = r_n;
        it = it_n;
        jt = jt_n;
    }
    if (bad && tid == 0) {
        atomicOr(&flags[FLAG_TIMEOUT], 1);
        if (inflight) mbar_wait_bounded(bar, parity);   // drain the copy in flight, bounded
    }
}

// Host side: the tables for realisations of n_r[r] tiles over at most
// G_target CTAs, phases split by cost (cost_diag / cost_sym per phase of a
// diagonal / symmetric tile pair), each CTA at least one phase.
struct EnsSymTables {
    std::vector<int> tab;
    int U = 0, G = 0, TT = 0, S_row = 0;
    long long slots = 0;
};

inline EnsSymTables build_ens_sym_tables(const std::vector<int> &n_r, int NW, long long G_target, int cost_diag,
                                         int cost_sym) {
    EnsSymTables s;
    const int R = (int)n_r.size();
    std::vector<int> ub(R + 1, 0), tb(R + 1, 0);
    for (int r = 0; r < R; ++r) {
        ub[r + 1] = ub[r] + n_r[r] * (n_r[r] + 1) / 2;
        tb[r + 1] = tb[r] + n_r[r];
    }
    const long long U = ub[R], P = U * NW;
    const int TT = tb[R];
    const int G = (int)std::max(1LL, std::min(G_target, P));
    long long total = 0;
    for (int r = 0; r < R; ++r)
        total += ((long long)n_r[r] * cost_diag + (long long)n_r[r] * (n_r[r] - 1) / 2 * cost_sym) * NW;
    std::vector<long long> start(G + 1, 0);
    long long pu = 0, prefix = 0;
    int g = 1;
    for (int r = 0; r < R; ++r)
        for (int it = 0; it < n_r[r]; ++it)
            for (int jt = it; jt < n_r[r]; ++jt) {
                const int c = it == jt ? cost_diag : cost_sym;
                for (int p = 0; p < NW; ++p, ++pu) {
                    while (g < G && prefix * G >= total * g) start[g++] = pu;
                    prefix += c;
                }
            }
    while (g < G) start[g++] = P;
    start[G] = P;
    for (int k = 1; k < G; ++k)
        start[k] = std::min(std::max(start[k], start[k - 1] + 1), P - (G - k));
    auto owner = [&](long long q) {
        return (int)(std::upper_bound(start.begin(), start.end() - 1, q) - start.begin()) - 1;
    };
    std::vector<int> row_g0(TT), row_ns(TT), col_start(TT + 1), unit_g0(U), unit_ko(U, 0), unit_nk(U);
    int S_row = 1;
    for (int r = 0; r < R; ++r) {
        const int n = n_r[r];
        for (int it = 0; it < n; ++it) {
            const long long u0 = ub[r] + sym_row_u0(it, n);
            const int gt = tb[r] + it;
            row_g0[gt] = owner(u0 * NW);
            row_ns[gt] = owner((u0 + (n - it)) * NW - 1) - row_g0[gt] + 1;
            S_row = std::max(S_row, row_ns[gt]);
            for (int jt = it; jt < n; ++jt) {
                const long long u = u0 + (jt - it);
                unit_g0[u] = owner(u * NW);
                unit_nk[u] = it == jt ? 0 : owner(u * NW + NW - 1) - unit_g0[u] + 1;
            }
        }
    }
    // column slots numbered column by column within each realisation
    long long ko = 0;
    for (int r = 0; r < R; ++r) {
        const int n = n_r[r];
        for (int jt = 0; jt < n; ++jt) {
            col_start[tb[r] + jt] = (int)ko;
            for (int it = 0; it < jt; ++it) {
                const long long u = ub[r] + sym_row_u0(it, n) + (jt - it);
                unit_ko[u] = (int)ko;
                ko += unit_nk[u];
            }
        }
    }
    col_start[TT] = (int)ko;
    s.tab.assign(kSymHdr, 0);
    s.tab[0] = R;
    s.tab[1] = NW;
    s.tab[2] = (int)U;
    s.tab[3] = G;
    s.tab[4] = TT;
    s.tab.insert(s.tab.end(), ub.begin(), ub.end());
    s.tab.insert(s.tab.end(), tb.begin(), tb.end());
    s.tab.insert(s.tab.end(), row_g0.begin(), row_g0.end());
    s.tab.insert(s.tab.end(), row_ns.begin(), row_ns.end());
    s.tab.insert(s.tab.end(), col_start.begin(), col_start.end());
    s.tab.insert(s.tab.end(), unit_g0.begin(), unit_g0.end());
    s.tab.insert(s.tab.end(), unit_ko.begin(), unit_ko.end());
    s.tab.insert(s.tab.end(), unit_nk.begin(), unit_nk.end());
    for (int k = 0; k <= G; ++k) s.tab.push_back((int)start[k]);
    s.U = (int)U;
    s.G = G;
    s.TT = TT;
    s.S_row = S_row;
    s.slots = ko;
    return s;
}

}  // namespace colatus
