"""Host logic of the pair-once kernels: their scheduling tables (no GPU).

Every pair is evaluated once (Eq. 1 summed over unordered pairs, Newton's
third law): the kernels walk the tile pairs it <= jt, each cut into phases
that a persistent grid of CTAs shares by cost, and leave per-body partial sums
in row segments and column slots that the consumers add in a fixed order.
colatus_selftest_sym_tables / colatus_selftest_ens_sym_tables build the tables
exactly as a context or an ensemble does and replay every CTA's walk on the
host.  They fail unless every phase is taken once, every row segment and
column slot is written once and lies in bounds, and every tile's column run
holds exactly the slots of its tile pairs.  The geometries below are the
kernels': the force (2048-body tiles, 32 sub-phases: 16 warps' slices of two
32-pair blocks each), the equal-mass VJP and the VJP for any masses (1024, 8),
the periodic real space (1024, 16) and the periodic VJP (1024, 8), at the
phase costs each plan uses, and the ensemble's 512-body tiles per realisation.
"""
import numpy as np
import pytest

from paper_1208_3444_b300 import binding as B
from paper_1208_3444_b300 import inputs

# (T, NW, cost_diag, cost_sym) of each pair-once plan
GEOMETRIES = {
    "force_eqm": (2048, 32, 11, 14),
    "force": (2048, 32, 12, 16),
    "vjp_eqm": (1024, 8, 23, 27),
    "vjp_any_masses": (1024, 8, 36, 40),
    "ewald_force": (1024, 16, 35, 38),
    "ewald_vjp": (1024, 8, 68, 72),
}
GRIDS = [1, 7, 147, 148, 294, 1000]


def expect_shape(r, tiles, G, NW):
    pairs = tiles * (tiles + 1) // 2
    assert r["tiles"] == tiles
    assert r["tile_pairs"] == pairs
    assert r["ctas"] == min(G, pairs * NW)
    # every symmetric tile pair has at least one column slot, diagonal ones none
    assert r["column_slots"] >= pairs - tiles
    assert r["row_segments"] >= 1


@pytest.mark.parametrize("name", sorted(GEOMETRIES))
@pytest.mark.parametrize("tiles", [1, 2, 3, 8, 16, 17, 32, 33])
@pytest.mark.parametrize("G", GRIDS)
def test_tables_replay(name, tiles, G):
    T, NW, cd, cs = GEOMETRIES[name]
    r = B.colatus_selftest_sym_tables(tiles * T, T, NW, G, cd, cs)
    expect_shape(r, tiles, G, NW)


def test_tables_of_the_largest_workloads():
    # 128^3 = 2^21 bodies on 147 CTAs (the force), and 2^18 bodies with the VJP
    r = B.colatus_selftest_sym_tables(1 << 21, 2048, 32, 147, 11, 14)
    expect_shape(r, 1024, 147, 32)
    r = B.colatus_selftest_sym_tables(1 << 18, 1024, 8, 147, 36, 40)
    expect_shape(r, 256, 147, 8)


def test_row_segments_follow_the_phase_split():
    # a CTA's share of the work is about total / G: with 16 tiles and 147 CTAs
    # no tile row can need more segments than CTAs share its phases
    T, NW, cd, cs = GEOMETRIES["force_eqm"]
    r = B.colatus_selftest_sym_tables(16 * T, T, NW, 147, cd, cs)
    phases = 136 * NW
    assert r["row_segments"] <= -(-16 * NW * 147 // phases) + 2


@pytest.mark.parametrize("G", [7, 148, 592, 1000])
def test_ensemble_tables_of_the_64_realisation_workload(G):
    sizes = [c.N for c in inputs.ensemble(64, seed=5)]
    r = B.colatus_selftest_ens_sym_tables(sizes, G, 11, 14)
    tiles = [-(-(-(-n // 256) * 256) // 512) for n in sizes]
    assert r["tiles"] == sum(tiles)
    assert r["tile_pairs"] == sum(t * (t + 1) // 2 for t in tiles)
    assert r["ctas"] == min(G, r["tile_pairs"] * 4)


@pytest.mark.parametrize("sizes", [[1, 1, 1], [32768], [4096, 1, 4097, 256, 257, 511, 513],
                                   [5, 700, 1300, 2500], [512, 1000, 1729, 3000]])
@pytest.mark.parametrize("costs", [(11, 14), (12, 16)])
def test_ensemble_tables_edge_sizes(sizes, costs):
    r = B.colatus_selftest_ens_sym_tables(sizes, 592, *costs)
    assert r["tiles"] == sum(-(-(-(-n // 256) * 256) // 512) for n in sizes)


@pytest.mark.parametrize("args", [(1000, 2048, 16, 147, 11, 14),     # n_pad not a multiple of T
                                  (4096, 2048, 48, 147, 11, 14),     # T/2 not whole 32-pair slices
                                  (4096, 2048, 16, 0, 11, 14),       # no CTA
                                  (4096, 2048, 16, 147, 0, 14),      # zero cost
                                  (2049 * 2048, 2048, 16, 147, 11, 14)])   # beyond 2048 tiles
def test_bad_arguments(args):
    with pytest.raises(B.ColatusError) as e:
        B.colatus_selftest_sym_tables(*args)
    assert e.value.status == B.E_ARG


def test_ensemble_bad_arguments():
    for sizes, G in (([0, 10], 148), ([10], 0), ([1 << 27], 148)):
        with pytest.raises(B.ColatusError) as e:
            B.colatus_selftest_ens_sym_tables(np.array(sizes), G, 11, 14)
        assert e.value.status == B.E_ARG
