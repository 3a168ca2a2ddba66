// selftest_api.cuh -- host-only self-tests of the pair-once scheduling
// tables (colatus_selftest_sym_tables, colatus_selftest_ens_sym_tables):
// they build the tables exactly as a context or ensemble does and replay the
// kernels' walk over them on the host (sym_check.cuh).  No GPU is touched.
// Included at the end of colatus.cu, after ensemble_api.cuh.
#pragma once

#include "sym_check.cuh"

extern "C" {

colatus_status colatus_selftest_sym_tables(int64_t n_pad, int T, int NW, int G, int cost_diag, int cost_sym,
                                           int64_t out[5]) {
    if (T < 64 || NW < 1 || (T / 2) % (NW * 32) != 0 || n_pad < T || n_pad % T != 0 || n_pad / T > 2048 ||
        G < 1 || cost_diag < 1 || cost_sym < 1)
        return fail(nullptr, COLATUS_E_ARG,
                    "selftest_sym_tables: need T/2 a multiple of 32 NW, n_pad a multiple of T (at most "
                    "2048 tiles), G >= 1 and positive costs");
    const colatus::SymTables s = colatus::build_sym_tables(n_pad, T, NW, G, cost_diag, cost_sym);
    const std::string e = colatus::check_sym_tables(s);
    if (out) {
        out[0] = s.n;
        out[1] = s.U;
        out[2] = s.G;
        out[3] = s.S_row;
        out[4] = s.slots;
    }
    if (!e.empty()) return fail(nullptr, COLATUS_E_STATE, "pair-once tables: %s", e.c_str());
    return COLATUS_OK;
}

colatus_status colatus_selftest_ens_sym_tables(int R, const int64_t *n_bodies, int G, int cost_diag,
                                               int cost_sym, int64_t out[5]) {
    if (R < 1 || !n_bodies || G < 1 || cost_diag < 1 || cost_sym < 1)
        return fail(nullptr, COLATUS_E_ARG, "selftest_ens_sym_tables: need R >= 1, sizes, G >= 1, positive costs");
    std::vector<long long> np(R);
    std::vector<int> nt(R);
    long long tiles = 0;
    for (int r = 0; r < R; ++r) {
        if (n_bodies[r] < 1 || n_bodies[r] > (1LL << 26))
            return fail(nullptr, COLATUS_E_ARG, "selftest_ens_sym_tables: realisation sizes 1 .. 2^26");
        np[r] = (n_bodies[r] + kEnsTile - 1) / kEnsTile * kEnsTile;   // the ensemble's storage padding
        nt[r] = (int)((np[r] + colatus::kEnsSymT - 1) / colatus::kEnsSymT);
        tiles += nt[r];
    }
    if (tiles > 2048) return fail(nullptr, COLATUS_E_ARG, "selftest_ens_sym_tables: at most 2048 tiles");
    const colatus::EnsSymTables s = colatus::build_ens_sym_tables(nt, EnsSymK::NW, G, cost_diag, cost_sym);
    const std::string e = colatus::check_ens_sym_tables(s, np, colatus::kEnsSymT);
    if (out) {
        out[0] = s.TT;
        out[1] = s.U;
        out[2] = s.G;
        out[3] = s.S_row;
        out[4] = s.slots;
    }
    if (!e.empty()) return fail(nullptr, COLATUS_E_STATE, "ensemble pair-once tables: %s", e.c_str());
    return COLATUS_OK;
}

}  // extern "C"
