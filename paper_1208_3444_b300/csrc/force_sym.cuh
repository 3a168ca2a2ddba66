// force_sym.cuh -- the all-pairs force of Eq. 1 with every pair evaluated
// once: the pair term that j exerts on k is minus the one k exerts on j
// (Newton's third law), so one evaluation of
//
//   w_kj = (|x_j - x_k|^2 + eps^2)^{-3/2},  d = x_j - x_k
//
// adds m_j w d to F_k and m_k w (-d) to F_j.  Per unordered pair that is 14
// FP32 lane-ops with equal masses (16 in general) and one MUFU.RSQ, against
// 2 x 11 (2 x 12) when each ordered pair is evaluated separately.
//
// The pair term is a policy (PlummerPair here; EwaldPair in ewald.cuh for the
// real-space part under periodic boundaries, whose term is as antisymmetric).
//
// Decomposition.  Bodies are cut into tiles of T = IPT NT.  The units are the
// tile pairs (it, jt) with it <= jt, ordered i-major:
//   u(it, jt) = row_u0(it) + jt - it,  row_u0(it) = it n - it (it - 1) / 2.
// A unit with it < jt is evaluated symmetrically: the i-tile's bodies sit in
// registers (IPT per thread, as duplicated float2 pairs), the j-tile in shared
// memory.  A diagonal unit (it == jt) is evaluated for every ordered pair on
// the i side only, which needs no mask (the self pair is exactly 0 for
// eps > 0).  Each unit is cut into NW phases (NW = warps per CTA); in phase p
// warp w takes the j-slice (w + p) mod NW, so after NW phases every j-pair has
// met every i-body of the tile and no two warps ever touch one slice at once.
// A slice holds ROT blocks of 32 j-pairs.  The tables' unit of scheduling is
// either a whole phase (NW per unit) or, where a CTA would get few phases,
// one block of every warp's slice, a sub-phase (PH = NW ROT per unit), so a
// CTA's share can end inside a phase.  The slices change hands (a barrier)
// only after a phase's last block, and the i-side sums are folded into the
// row's once per phase either way.
// Inside a slice the 32 lanes rotate the j-pairs: in round r lane l takes
// j-pair (l + r) mod 32, and the j-pair's running sum moves one lane down by
// a warp shuffle after each round, so it stays with its j-pair.  At the end
// of a 32-round rotation each lane folds the sum it holds into the slice's
// shared-memory accumulator.  A persistent grid splits the phases of all
// units evenly by cost (a diagonal phase costs 11/14 or 12/16 of a symmetric
// one); a CTA keeps the i-side sums of a row in registers across its units
// and writes one row segment per row, and one column slot per symmetric unit
// it worked on.  The step epilogue adds, for a body of tile t, the row
// segments of t and the column slots of the units (t', t), t' < t, in a fixed
// order, so the result does not depend on timing.
//
// Bodies come pair-interleaved ([x0 x1 y0 y1 z0 z1 m0 m1] per pair); a unit's
// j-tile is bulk-copied into a staging buffer (bounded mbarrier wait) and then
// split into the (x0 x1 y0 y1) and (z0 z1 m0 m1) halves, so that the 32
// lanes' different j-pairs load without bank conflicts, with every 32-pair
// block stored twice, so that a lane's rounds read consecutive entries.  The copy for the
// next unit runs while the current one is evaluated.
#pragma once

#include <algorithm>
#include <vector>

#include "force.cuh"

namespace colatus {

// Layout of the int tables of a symmetric plan (ForceLaunch::sym):
//   [0] n tiles, [1] scheduling units per tile pair (NW or PH), [2] U units, [3] G CTAs,
//   [kSymHdr ...]  row_g0[n], row_ns[n], col_start[n + 1], unit_g0[U],
//                  unit_ko[U], unit_nk[U], cta_pu[G + 1]
// row_g0 / row_ns: first CTA and number of row segments of i-tile t;
// unit_g0 / unit_ko / unit_nk: first CTA, first column slot and number of
// column slots of unit u (0 for a diagonal unit); the slots are numbered
// column by column (tile jt, then it < jt, then CTA), so the slots on the
// bodies of tile t are the one run [col_start[t], col_start[t + 1]);
// cta_pu: first scheduling unit (u [1] + unit) of CTA g.
constexpr int kSymHdr = 8;

__host__ __device__ inline long long sym_row_u0(long long it, long long n) {
    return it * n - it * (it - 1) / 2;
}

struct SymTab {
    const int *row_g0, *row_ns, *col_start, *unit_g0, *unit_ko, *unit_nk, *cta_pu;
    int n, NW, U, G;   // NW: the tables' scheduling units per tile pair
    __host__ __device__ explicit SymTab(const int *t) {
        n = t[0];
        NW = t[1];
        U = t[2];
        G = t[3];
        row_g0 = t + kSymHdr;
        row_ns = row_g0 + n;
        col_start = row_ns + n;
        unit_g0 = col_start + n + 1;
        unit_ko = unit_g0 + U;
        unit_nk = unit_ko + U;
        cta_pu = unit_nk + U;
    }
};

template <int NT, int IPT_, bool COMP>
struct SymKernel {
    static constexpr int IPT = IPT_;
    static constexpr int NW = NT / 32;
    static constexpr int T = NT * IPT;        // bodies per tile
    static constexpr int TP = T / 2;          // j-pairs per tile
    static constexpr int SLICE = TP / NW;     // j-pairs per warp slice
    static constexpr int ROT = SLICE / 32;    // 32-round rotations per phase
    static constexpr int PH = NW * ROT;       // sub-phases per unit (one 32-pair block each)
    static constexpr uint32_t TILE_BYTES = T * 16;
    static constexpr int PLANES = COMP ? 2 : 1;
    // staging tile, the two halves (each 32-pair block stored twice, so that
    // lane l's 32 rounds read 32 consecutive entries from its own start), the
    // column accumulators [plane][x y z][TP] float2, one mbarrier
    static constexpr int SMEM = TILE_BYTES + 2 * TILE_BYTES + PLANES * 3 * TP * 8 + 16;
    static_assert(SLICE % 32 == 0, "a warp slice is whole rotations");
};

// Unit u -> (it, jt).
__host__ __device__ __forceinline__ void sym_decode(long long u, int n, int &it, int &jt) {
    const double b = 2.0 * n + 1.0;
    long long t = (long long)((b - sqrt(b * b - 8.0 * (double)u)) * 0.5);
    if (t < 0) t = 0;
    if (t > n - 1) t = n - 1;
    while (t > 0 && sym_row_u0(t, n) > u) --t;
    while (t + 1 < n && sym_row_u0(t + 1, n) <= u) ++t;
    it = (int)t;
    jt = (int)(t + (u - sym_row_u0(t, n)));
}

// A float2 moved between lanes as one 64-bit value (the two halves stay a
// register pair).
__device__ __forceinline__ float2 shfl_float2(float2 v, int src) {
    unsigned long long b = (unsigned long long)__float_as_uint(v.x) |
                           ((unsigned long long)__float_as_uint(v.y) << 32);
    b = __shfl_sync(0xffffffffu, b, src);
    return make_float2(__uint_as_float((unsigned)b), __uint_as_float((unsigned)(b >> 32)));
}

// Pair terms.  A pair policy P gives, for the separation (dx, dy, dz) = x_j -
// x_i of two j-bodies at once, the mass-free weight w with which the pair adds
// m_j w d to body i and -m_i w d to body j; it may replace d by the
// separation it uses (the minimum image under periodic boundaries).
// PlummerPair: w = (|d|^2 + eps^2)^{-3/2} (Eq. 1), 8 FP32 lane-ops and one
// MUFU.RSQ.
struct PlummerPair {
    struct Args {};
    __device__ __forceinline__ static float2 weight(float2 &dx, float2 &dy, float2 &dz, const float2 e2,
                                                    const Args &) {
        float2 r2 = __ffma2_rn(dx, dx, e2);
        r2 = __ffma2_rn(dy, dy, r2);
        r2 = __ffma2_rn(dz, dz, r2);
        const float2 inv = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
        const float2 inv2 = __fmul2_rn(inv, inv);
        return __fmul2_rn(inv, inv2);
    }
};

// One 32-round rotation of a warp over the 32 j-pairs of one doubled block
// (entries 32..63 repeat 0..31; the block's entries start at sA, sB + 64 blk):
// every lane's IPT i-bodies against every j-pair, lane l taking entry l + r
// in round r.  SYM: also
// the j-side sums, which travel with their j-pairs (one lane down after every
// round) and so end, in lane l, as the sum of j-pair base + l (returned in
// jx, jy, jz; they hold sum_k m_k w d, minus the force on j; without m_k for
// EQM).
template <class P, int IPT, bool SYM, bool EQM, int UNR>
__device__ __forceinline__ void sym_rotation(const float4 *__restrict__ sA, const float4 *__restrict__ sB,
                                             int lane, const float2 (&nx)[IPT],
                                             const float2 (&ny)[IPT], const float2 (&nz)[IPT],
                                             const float2 (&mi)[IPT], const float2 e2, const typename P::Args &pa,
                                             float2 (&px)[IPT], float2 (&py)[IPT], float2 (&pz)[IPT],
                                             float2 &jx, float2 &jy, float2 &jz) {
    const int src = (lane + 1) & 31;
    const float4 *a = sA + lane, *b = sB + lane;
#pragma unroll(UNR)
    for (int r = 0; r < 32; ++r) {
        const float4 A = a[r];   // x0 x1 y0 y1
        const float4 B = b[r];   // z0 z1 m0 m1
        const float2 xj = make_float2(A.x, A.y), yj = make_float2(A.z, A.w);
        const float2 zj = make_float2(B.x, B.y), mj = make_float2(B.z, B.w);
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            float2 dx = __fadd2_rn(xj, nx[k]);
            float2 dy = __fadd2_rn(yj, ny[k]);
            float2 dz = __fadd2_rn(zj, nz[k]);
            const float2 w = P::weight(dx, dy, dz, e2, pa);
            const float2 wi = EQM ? w : __fmul2_rn(mj, w);
            px[k] = __ffma2_rn(dx, wi, px[k]);
            py[k] = __ffma2_rn(dy, wi, py[k]);
            pz[k] = __ffma2_rn(dz, wi, pz[k]);
            if (SYM) {
                const float2 wj = EQM ? w : __fmul2_rn(mi[k], w);
                jx = __ffma2_rn(dx, wj, jx);
                jy = __ffma2_rn(dy, wj, jy);
                jz = __ffma2_rn(dz, wj, jz);
            }
        }
        if (SYM) {
            jx = shfl_float2(jx, src);
            jy = shfl_float2(jy, src);
            jz = shfl_float2(jz, src);
        }
    }
}

// Persistent symmetric force kernel, FP32, for the pair term P (pa: its
// parameters).  pk: pair-interleaved bodies
// (N_pad a multiple of T).  part: row segments [n][S_max][PLANES][T] float4,
// then from float4 offset L.col_off the column slots [slot][PLANES][T]
// float4 (for COMP the second plane holds the low words).  EQM: every body
// has mass mass_eq and no zero-mass padding enters; segments are scaled by
// mass_eq.  Both the row and column sums are forces on the bodies they index
// (the column slots are negated when written).
// FINE: the tables are in sub-phases (NW ROT per tile pair), else in whole
// phases (NW); the host builds them and sets ForceLaunch::fine together.
template <int NT, int IPT, bool COMP, bool EQM, int UNR, class P = PlummerPair, bool FINE = false>
__global__ void __launch_bounds__(NT, 1)
    force_sym_f32_kernel(const float *__restrict__ pk, float4 *__restrict__ part, int *__restrict__ flags,
                         ForceLaunch L, float eps2, float mass_eq, typename P::Args pa) {
    using K = SymKernel<NT, IPT, COMP>;
    constexpr int NW = K::NW, T = K::T, TP = K::TP, PL = K::PLANES, ROT = K::ROT;
    extern __shared__ __align__(128) unsigned char smem[];
    float4 *raw = reinterpret_cast<float4 *>(smem);   // staging: T float4 (pair-interleaved)
    float4 *sA = raw + T;                             // 2 TP float4: x0 x1 y0 y1, blocks doubled
    float4 *sB = sA + 2 * TP;                         // 2 TP float4: z0 z1 m0 m1, blocks doubled
    float2 *acc = reinterpret_cast<float2 *>(sB + 2 * TP);   // [PL][3][TP]
    uint64_t *bar = reinterpret_cast<uint64_t *>(acc + PL * 3 * TP);

    const SymTab S(L.sym);
    const int n = S.n;
    const int *row_g0 = S.row_g0, *unit_g0 = S.unit_g0, *unit_ko = S.unit_ko, *cta_pu = S.cta_pu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = blockIdx.x;
    // scheduling units per tile pair: whole phases (NW) or sub-phases (NW ROT)
    constexpr bool fine = FINE && ROT > 1;
    constexpr int PH = fine ? K::PH : NW;
    constexpr int BPU = fine ? 1 : ROT;   // 32-pair blocks per scheduling unit
    int pu = cta_pu[g];
    const int pu_end = cta_pu[g + 1];
    if (pu >= pu_end) return;
    long long u = pu / PH;
    int it, jt;
    sym_decode(u, n, it, jt);

    for (int q = tid; q < PL * 3 * TP; q += NT) acc[q] = make_float2(0.f, 0.f);
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(bar, K::TILE_BYTES);
        bulk_load(raw, pk + (long long)jt * T * 4, K::TILE_BYTES, bar);
    }
    bool inflight = true;

    const float2 e2 = make_float2(eps2, eps2);
    const float ms = EQM ? mass_eq : 1.f;
    float2 nx[IPT], ny[IPT], nz[IPT], mi[IPT];
    float hx[IPT], hy[IPT], hz[IPT], lx[IPT], ly[IPT], lz[IPT];
    auto load_i = [&](int row) {
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const long long i = (long long)row * T + tid + k * NT;
            const float *p = pk + (i >> 1) * 8 + (i & 1);
            const float x = __ldg(p), y = __ldg(p + 2), z = __ldg(p + 4), m = __ldg(p + 6);
            nx[k] = make_float2(-x, -x);
            ny[k] = make_float2(-y, -y);
            nz[k] = make_float2(-z, -z);
            mi[k] = make_float2(m, m);
            hx[k] = hy[k] = hz[k] = 0.f;
            lx[k] = ly[k] = lz[k] = 0.f;
        }
    };
    load_i(it);

    uint32_t parity = 0;
    bool bad = false;
    while (pu < pu_end) {
        const int uend = (int)min((long long)pu_end, (u + 1) * PH);
        const int p0 = pu - (int)(u * PH), p1 = uend - (int)(u * PH);
        const bool ok = mbar_wait_bounded(bar, parity);
        if (__syncthreads_or(!ok)) {
            bad = true;
            break;
        }
        inflight = false;
        parity ^= 1u;
        for (int q = tid; q < TP; q += NT) {
            const int e = 2 * q - (q & 31);   // entry of pair q in its doubled block
            const float4 A = raw[2 * q], B = raw[2 * q + 1];
            sA[e] = A;
            sA[e + 32] = A;
            sB[e] = B;
            sB[e + 32] = B;
        }
        __syncthreads();
        // the next unit's j-tile into the staging buffer while this one runs
        int it_n = it, jt_n = jt + 1;
        if (jt_n == n) {
            ++it_n;
            jt_n = it_n;
        }
        if (uend < pu_end) {
            if (tid == 0) {
                mbar_arrive_expect_tx(bar, K::TILE_BYTES);
                bulk_load(raw, pk + (long long)jt_n * T * 4, K::TILE_BYTES, bar);
            }
            inflight = true;
        }
        const bool sym = jt != it;
        // the i-side sums of a phase: folded into the row's sums once per
        // phase (or at the end of the CTA's range), as many folds as with
        // whole phases, so the plain FP32 row sums round no more
        float2 px[IPT], py[IPT], pz[IPT];
#pragma unroll 1
        for (int ps = p0; ps < p1; ++ps) {
            const int p = fine ? ps / ROT : ps;           // phase
            const int sb = fine ? ps - p * ROT : 0;       // first block of the slice
            const int slice = (warp + p) % NW;
            const bool last = sb + BPU == ROT || ps == p1 - 1;
            if (sb == 0 || ps == p0) {
#pragma unroll
                for (int k = 0; k < IPT; ++k) px[k] = py[k] = pz[k] = make_float2(0.f, 0.f);
            }
#pragma unroll 1
            for (int s = sb; s < sb + BPU; ++s) {
                const int base = slice * K::SLICE + s * 32;
                const float4 *bA = sA + 2 * base, *bB = sB + 2 * base;   // the block's doubled entries
                float2 jx = make_float2(0.f, 0.f), jy = jx, jz = jx;
                if (sym) {
                    sym_rotation<P, IPT, true, EQM, UNR>(bA, bB, lane, nx, ny, nz, mi, e2, pa, px, py, pz,
                                                         jx, jy, jz);
                    const int q = base + lane;
                    float2 *h = acc + q;
                    if (COMP) {
                        float2 *l = acc + 3 * TP + q;
                        float2 a = h[0], b = h[TP], c = h[2 * TP];
                        float2 d = l[0], e = l[TP], f = l[2 * TP];
                        acc2_add(a.x, d.x, jx.x);
                        acc2_add(a.y, d.y, jx.y);
                        acc2_add(b.x, e.x, jy.x);
                        acc2_add(b.y, e.y, jy.y);
                        acc2_add(c.x, f.x, jz.x);
                        acc2_add(c.y, f.y, jz.y);
                        h[0] = a;
                        h[TP] = b;
                        h[2 * TP] = c;
                        l[0] = d;
                        l[TP] = e;
                        l[2 * TP] = f;
                    } else {
                        h[0] = __fadd2_rn(h[0], jx);
                        h[TP] = __fadd2_rn(h[TP], jy);
                        h[2 * TP] = __fadd2_rn(h[2 * TP], jz);
                    }
                } else {
                    sym_rotation<P, IPT, false, EQM, UNR>(bA, bB, lane, nx, ny, nz, mi, e2, pa, px, py, pz,
                                                          jx, jy, jz);
                }
            }
            if (last) {
#pragma unroll
                for (int k = 0; k < IPT; ++k) {
                    if (COMP) {
                        acc2_add(hx[k], lx[k], px[k].x + px[k].y);
                        acc2_add(hy[k], ly[k], py[k].x + py[k].y);
                        acc2_add(hz[k], lz[k], pz[k].x + pz[k].y);
                    } else {
                        hx[k] += px[k].x + px[k].y;
                        hy[k] += py[k].x + py[k].y;
                        hz[k] += pz[k].x + pz[k].y;
                    }
                }
                // the slices change hands after a phase's last block; the range's
                // end is a barrier too (the column slot and the next staging follow)
                __syncthreads();
            }
        }
        if (sym) {
            // this CTA's share of unit u on the j-tile's bodies: the column slot
            const int slot = unit_ko[u] + (g - unit_g0[u]);
            float4 *dst = part + L.col_off + (long long)slot * PL * T;
            for (int q = tid; q < TP; q += NT) {
                const float2 a = acc[q], b = acc[TP + q], c = acc[2 * TP + q];
                dst[2 * q] = make_float4(-ms * a.x, -ms * b.x, -ms * c.x, 0.f);
                dst[2 * q + 1] = make_float4(-ms * a.y, -ms * b.y, -ms * c.y, 0.f);
                acc[q] = acc[TP + q] = acc[2 * TP + q] = make_float2(0.f, 0.f);
                if (COMP) {
                    float2 *l = acc + 3 * TP;
                    const float2 d = l[q], e = l[TP + q], f = l[2 * TP + q];
                    dst[T + 2 * q] = make_float4(-ms * d.x, -ms * e.x, -ms * f.x, 0.f);
                    dst[T + 2 * q + 1] = make_float4(-ms * d.y, -ms * e.y, -ms * f.y, 0.f);
                    l[q] = l[TP + q] = l[2 * TP + q] = make_float2(0.f, 0.f);
                }
            }
            __syncthreads();
        }
        pu = uend;
        ++u;
        if (it_n != it || pu == pu_end) {
            // the row segment of i-tile it
            const int sidx = g - row_g0[it];
            float4 *dst = part + ((long long)it * L.S_max + sidx) * PL * T;
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                dst[tid + k * NT] = make_float4(ms * hx[k], ms * hy[k], ms * hz[k], 0.f);
                if (COMP) dst[T + tid + k * NT] = make_float4(ms * lx[k], ms * ly[k], ms * lz[k], 0.f);
            }
            if (it_n != it && pu < pu_end) load_i(it_n);
        }
        it = it_n;
        jt = jt_n;
    }
    if (bad && tid == 0) {
        atomicOr(&flags[FLAG_TIMEOUT], 1);
        if (inflight) mbar_wait_bounded(bar, parity);   // drain the copy in flight, bounded
    }
}

// Host side: the tables of a symmetric plan for n_pad bodies (a multiple of
// T) over at most G_target CTAs.  The phases of all units are split so that
// every CTA gets the same cost (cost_diag / cost_sym per phase of a diagonal
// / symmetric unit), each CTA at least one phase.
struct SymTables {
    std::vector<int> tab;
    int n = 0, U = 0, G = 0, S_row = 0;
    long long slots = 0;   // column slots in all
};

inline SymTables build_sym_tables(long long n_pad, int T, int NW, long long G_target, int cost_diag,
                                  int cost_sym) {
    SymTables s;
    const int n = (int)(n_pad / T);
    const long long U = (long long)n * (n + 1) / 2, P = U * NW;
    const int G = (int)std::max(1LL, std::min(G_target, P));
    const long long total = ((long long)n * cost_diag + (U - n) * cost_sym) * NW;
    std::vector<long long> start(G + 1, 0);
    long long pu = 0, prefix = 0;
    int g = 1;
    for (int it = 0; it < n; ++it)
        for (int jt = it; jt < n; ++jt) {
            const int c = it == jt ? cost_diag : cost_sym;
            for (int p = 0; p < NW; ++p, ++pu) {
                while (g < G && prefix * G >= total * g) start[g++] = pu;
                prefix += c;
            }
        }
    while (g < G) start[g++] = P;
    start[G] = P;
    for (int k = 1; k < G; ++k)   // no empty CTA: strictly increasing starts
        start[k] = std::min(std::max(start[k], start[k - 1] + 1), P - (G - k));
    auto owner = [&](long long q) {
        return (int)(std::upper_bound(start.begin(), start.end() - 1, q) - start.begin()) - 1;
    };
    std::vector<int> row_g0(n), row_ns(n), col_start(n + 1), unit_g0(U), unit_ko(U, 0), unit_nk(U);
    int S_row = 1;
    for (int it = 0; it < n; ++it) {
        const long long a = sym_row_u0(it, n) * NW, b = sym_row_u0(it + 1, n) * NW - 1;
        row_g0[it] = owner(a);
        row_ns[it] = owner(b) - row_g0[it] + 1;
        S_row = std::max(S_row, row_ns[it]);
        for (int jt = it; jt < n; ++jt) {
            const long long u = sym_row_u0(it, n) + (jt - it);
            unit_g0[u] = owner(u * NW);
            unit_nk[u] = it == jt ? 0 : owner(u * NW + NW - 1) - unit_g0[u] + 1;
        }
    }
    // column slots numbered column by column
    long long ko = 0;
    for (int jt = 0; jt < n; ++jt) {
        col_start[jt] = (int)ko;
        for (int it = 0; it < jt; ++it) {
            const long long u = sym_row_u0(it, n) + (jt - it);
            unit_ko[u] = (int)ko;
            ko += unit_nk[u];
        }
    }
    col_start[n] = (int)ko;
    s.tab.assign(kSymHdr, 0);
    s.tab[0] = n;
    s.tab[1] = NW;
    s.tab[2] = (int)U;
    s.tab[3] = G;
    s.tab.insert(s.tab.end(), row_g0.begin(), row_g0.end());
    s.tab.insert(s.tab.end(), row_ns.begin(), row_ns.end());
    s.tab.insert(s.tab.end(), col_start.begin(), col_start.end());
    s.tab.insert(s.tab.end(), unit_g0.begin(), unit_g0.end());
    s.tab.insert(s.tab.end(), unit_ko.begin(), unit_ko.end());
    s.tab.insert(s.tab.end(), unit_nk.begin(), unit_nk.end());
    for (int k = 0; k <= G; ++k) s.tab.push_back((int)start[k]);
    s.n = n;
    s.U = (int)U;
    s.G = G;
    s.S_row = S_row;
    s.slots = ko;
    return s;
}

}  // namespace colatus
