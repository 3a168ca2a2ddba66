// sym_check.cuh -- host replay of the pair-once kernels' walk over their
// scheduling tables (force_sym.cuh for the force, the VJPs and the periodic
// real space; ens_sym.cuh for the ensemble), behind the self-test entry points.
//
// Each CTA g takes the phases cta_pu[g] .. cta_pu[g+1]-1 of the tile pairs
// in order.  It decodes its first tile pair with the kernels' own sym_decode
// (and ens_find_int), steps to the next pair as the kernels do, writes one
// column slot unit_ko[u] + (g - unit_g0[u]) per symmetric pair it worked on,
// and one row segment g - row_g0[it] whenever it leaves a row or ends.  The
// replay checks that every phase of every tile pair is taken exactly once,
// that every row segment and column slot is written exactly once and lies in
// its table's bounds, and that each tile's column run
// col_start[t] .. col_start[t+1] holds exactly the slots of the pairs
// (t', t), t' < t, in order: the sums the consumers add.
#pragma once

#include <string>
#include <vector>

#include "ens_sym.cuh"
#include "force_sym.cuh"

namespace colatus {

// "" when the single-system tables hold, else the first failure.
inline std::string check_sym_tables(const SymTables &s) {
    const SymTab S(s.tab.data());
    const int n = s.n, U = s.U, NW = S.NW;
    if (S.n != n || S.U != U || S.G != s.G) return "header";
    if ((long long)s.tab.size() != kSymHdr + 3LL * n + 1 + 3LL * U + s.G + 1) return "table size";
    if (U != (long long)n * (n + 1) / 2) return "tile pair count";
    for (int t = 0; t < n; ++t) {
        int k = S.col_start[t];
        for (int tp = 0; tp < t; ++tp) {
            const long long u = sym_row_u0(tp, n) + (t - tp);
            for (int c = 0; c < S.unit_nk[u]; ++c, ++k)
                if (S.unit_ko[u] + c != k) return "column run of tile " + std::to_string(t);
        }
        if (k != S.col_start[t + 1]) return "column run end of tile " + std::to_string(t);
    }
    if (S.col_start[n] != s.slots) return "column slot total";
    for (int it = 0; it < n; ++it)
        for (int jt = it; jt < n; ++jt) {
            const long long u = sym_row_u0(it, n) + (jt - it);
            if ((it == jt) != (S.unit_nk[u] == 0)) return "slots of tile pair " + std::to_string(u);
        }
    std::vector<int> phase((size_t)U * NW, 0), rows((size_t)n * s.S_row, 0), cols((size_t)s.slots, 0);
    for (int g = 0; g < s.G; ++g) {
        int pu = S.cta_pu[g];
        const int pe = S.cta_pu[g + 1];
        if (pu >= pe) return "empty CTA " + std::to_string(g);
        long long u = pu / NW;
        int it, jt;
        sym_decode(u, n, it, jt);
        if (it < 0 || jt < it || jt >= n || sym_row_u0(it, n) + (jt - it) != u) return "decode";
        while (pu < pe) {
            const int uend = (int)std::min((long long)pe, (u + 1) * NW);
            for (int p = pu; p < uend; ++p) ++phase[(size_t)p];
            int it_n = it, jt_n = jt + 1;
            if (jt_n == n) {
                ++it_n;
                jt_n = it_n;
            }
            if (uend < pe && (it_n >= n || sym_row_u0(it_n, n) + (jt_n - it_n) != u + 1)) return "step";
            if (jt != it) {
                const int k = g - S.unit_g0[u];
                if (k < 0 || k >= S.unit_nk[u]) return "column slot of CTA " + std::to_string(g);
                ++cols[(size_t)(S.unit_ko[u] + k)];
            }
            pu = uend;
            ++u;
            if (it_n != it || pu == pe) {
                const int k = g - S.row_g0[it];
                if (k < 0 || k >= S.row_ns[it] || S.row_ns[it] > s.S_row) return "row segment of CTA " + std::to_string(g);
                ++rows[(size_t)it * s.S_row + k];
            }
            it = it_n;
            jt = jt_n;
        }
    }
    for (size_t p = 0; p < phase.size(); ++p)
        if (phase[p] != 1) return "phase " + std::to_string(p) + " taken " + std::to_string(phase[p]) + " times";
    for (size_t k = 0; k < cols.size(); ++k)
        if (cols[k] != 1) return "column slot " + std::to_string(k) + " written " + std::to_string(cols[k]) + " times";
    for (int it = 0; it < n; ++it)
        for (int k = 0; k < S.row_ns[it]; ++k)
            if (rows[(size_t)it * s.S_row + k] != 1) return "row segment " + std::to_string(k) + " of tile " + std::to_string(it);
    return "";
}

// The ensemble's tables: realisations of np[r] stored bodies (a multiple of
// the storage padding) in tiles of T; tiles[r] = ceil(np[r] / T).
inline std::string check_ens_sym_tables(const EnsSymTables &s, const std::vector<long long> &np, int T) {
    const EnsSymTab S(s.tab.data());
    const int R = S.R, NW = S.NW;
    if (R != (int)np.size() || S.U != s.U || S.G != s.G || S.TT != s.TT) return "header";
    for (int r = 0; r < R; ++r) {
        const int nr = S.tb[r + 1] - S.tb[r];
        if (nr != (int)((np[r] + T - 1) / T)) return "tiles of realisation " + std::to_string(r);
        if (S.ub[r + 1] - S.ub[r] != nr * (nr + 1) / 2) return "tile pairs of realisation " + std::to_string(r);
        for (int t = 0; t < nr; ++t) {
            int k = S.col_start[S.tb[r] + t];
            for (int tp = 0; tp < t; ++tp) {
                const int u = S.ub[r] + (int)sym_row_u0(tp, nr) + (t - tp);
                for (int c = 0; c < S.unit_nk[u]; ++c, ++k)
                    if (S.unit_ko[u] + c != k) return "column run of realisation " + std::to_string(r);
            }
            if (k != S.col_start[S.tb[r] + t + 1]) return "column run end of realisation " + std::to_string(r);
        }
    }
    if (S.col_start[S.TT] != s.slots) return "column slot total";
    auto valid = [&](int r, int t) { return (long long)std::min<long long>(T, np[r] - (long long)t * T); };
    std::vector<int> phase((size_t)S.U * NW, 0), rows((size_t)S.TT * s.S_row, 0), cols((size_t)s.slots, 0);
    for (int g = 0; g < S.G; ++g) {
        int pu = S.cta_pu[g];
        const int pe = S.cta_pu[g + 1];
        if (pu >= pe) return "empty CTA " + std::to_string(g);
        int u = pu / NW;
        int r = ens_find_int(S.ub, R, u);
        int nr = S.tb[r + 1] - S.tb[r];
        int it, jt;
        sym_decode(u - S.ub[r], nr, it, jt);
        while (pu < pe) {
            const int uend = std::min(pe, (u + 1) * NW);
            for (int p = pu; p < uend; ++p) ++phase[(size_t)p];
            const long long vb = valid(r, jt);
            if (vb <= 0 || vb % 2) return "stored bodies of a j-tile";
            int r_n = r, it_n = it, jt_n = jt + 1;
            if (jt_n == nr) {
                ++it_n;
                jt_n = it_n;
                if (it_n == nr) {
                    ++r_n;
                    it_n = jt_n = 0;
                }
            }
            if (uend < pe) {
                if (r_n >= R) return "step past the last realisation";
                const int nn = S.tb[r_n + 1] - S.tb[r_n];
                if (S.ub[r_n] + sym_row_u0(it_n, nn) + (jt_n - it_n) != u + 1) return "step";
            }
            if (jt != it) {
                const int k = g - S.unit_g0[u];
                if (k < 0 || k >= S.unit_nk[u]) return "column slot of CTA " + std::to_string(g);
                ++cols[(size_t)(S.unit_ko[u] + k)];
            }
            pu = uend;
            ++u;
            if (r_n != r || it_n != it || pu == pe) {
                const int gt = S.tb[r] + it, k = g - S.row_g0[gt];
                if (k < 0 || k >= S.row_ns[gt] || S.row_ns[gt] > s.S_row) return "row segment of CTA " + std::to_string(g);
                ++rows[(size_t)gt * s.S_row + k];
                if (pu < pe && r_n != r) nr = S.tb[r_n + 1] - S.tb[r_n];
            }
            r = r_n;
            it = it_n;
            jt = jt_n;
        }
    }
    for (size_t p = 0; p < phase.size(); ++p)
        if (phase[p] != 1) return "phase " + std::to_string(p) + " taken " + std::to_string(phase[p]) + " times";
    for (size_t k = 0; k < cols.size(); ++k)
        if (cols[k] != 1) return "column slot " + std::to_string(k) + " written " + std::to_string(cols[k]) + " times";
    for (int t = 0; t < S.TT; ++t)
        for (int k = 0; k < S.row_ns[t]; ++k)
            if (rows[(size_t)t * s.S_row + k] != 1) return "row segment " + std::to_string(k) + " of tile " + std::to_string(t);
    return "";
}

}  // namespace colatus
