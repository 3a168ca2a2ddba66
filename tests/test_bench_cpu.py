"""Host-side accounting of bench.py that the reported roofline figures rest on
(no GPU): the FP32 lane-ops per counted interaction of the launched force
kernel, and the gate that reports the captured DRAM traffic only for the
captured kernel.

Lane-ops per pair, counted from the kernels: the pair-once force takes 14
(equal masses) or 16 FP32 lane-ops per symmetric pair and 11 or 12 per ordered
pair of a diagonal tile; the per-ordered-pair kernel 11 or 12 per ordered pair
over the padded bodies.  The expected values below are worked out by hand for
the benchmark's sizes.
"""
import bench

SYM_EQM = dict(kind="force_sym_f32", threads=512, ipt=4, jt=2048, comp=True, eqm=True, nrcp=0)


def test_lane_ops_pair_once_at_32_cubed():
    # 16 tiles of 2048: 120 symmetric tile pairs x 14 + 16 diagonal x 11 lane-ops,
    # each over 2048^2 pairs, per 32768^2 interactions: 1856 / 256 = 7.25
    assert abs(bench.pair_lane_ops(SYM_EQM, 32768) - 7.25) < 1e-12


def test_lane_ops_pair_once_at_128_cubed():
    # 1024 tiles: (523776 x 14 + 1024 x 11) / 1024^2 = 7344128 / 1048576
    assert abs(bench.pair_lane_ops(SYM_EQM, 1 << 21) - 7344128 / 1048576) < 1e-12


def test_lane_ops_pair_once_any_masses_and_padding():
    plan = dict(SYM_EQM, eqm=False)
    # 30000 bodies: 15 tiles of 2048 (30720 padded), 105 x 16 + 15 x 12 per tile pair
    want = (105 * 16 + 15 * 12) * 2048.0 ** 2 / 30000.0 ** 2
    assert abs(bench.pair_lane_ops(plan, 30000) - want) < 1e-12


def test_lane_ops_per_ordered_pair_kernel():
    plan = dict(kind="force_f32", threads=512, ipt=4, jt=512, comp=True, eqm=True, nrcp=0)
    assert bench.pair_lane_ops(plan, 32768) == 11.0
    plan = dict(plan, eqm=False)
    # 3000 bodies pad to 4096 (the 2048-body i-tile): 12 lane-ops over 4096^2
    assert abs(bench.pair_lane_ops(plan, 3000) - 12 * 4096.0 ** 2 / 3000.0 ** 2) < 1e-12


def test_traffic_reported_only_for_the_captured_kernel():
    nbytes, same_shape, same_source = bench.force_traffic(SYM_EQM)
    assert same_shape and same_source and nbytes == bench.FORCE_KERNEL_TRAFFIC["bytes"]
    # at least the positions read once (16 B per body at 32^3), and not far above
    assert 524288 <= nbytes < 1.2 * 524288
    for other in (dict(SYM_EQM, jt=1024), dict(SYM_EQM, comp=False), dict(SYM_EQM, kind="force_f32")):
        nbytes, same_shape, _ = bench.force_traffic(other)
        assert nbytes is None and not same_shape


def test_source_hash_tracks_the_kernel_sources():
    paths = bench.FORCE_KERNEL_TRAFFIC["sources"]
    assert bench.source_hash(paths) == bench.source_hash(list(paths))
    assert bench.source_hash(paths) != bench.source_hash(paths[:1])
