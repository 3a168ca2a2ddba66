"""CPU-side checks of the CUDA library: it builds for sm_103a, loads without a
GPU, and exports every entry point the C header declares; the binding fails
loudly (no fallback) when no device is present."""
import re
import subprocess

import numpy as np
import pytest

from paper_1208_3444_b300 import binding, build, inputs

HEADER = build.os.path.join(build.INCLUDE, "colatus.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(colatus_[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_header_symbols():
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r" T (colatus_\w+)", out))
    decl = declared_functions()
    assert decl, "no declarations parsed"
    missing = [d for d in decl if d not in exported]
    assert not missing, missing
    assert sorted(binding.EXPORTS) == decl


def test_build_targets_sm_103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_loads_and_reports_errors_without_gpu():
    L = binding.lib()
    for name in binding.EXPORTS:
        assert hasattr(L, name)
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present; covered by the gpu tests")
    except ImportError:
        pass
    with pytest.raises(binding.ColatusError) as e:
        binding.colatus_init(4, np.ones(4), 0.1, 0, 0.3, 0, 0.7, 1.0, 0.02)
    assert e.value.status == binding.E_CUDA


def test_argument_checks_happen_before_any_device_call():
    with pytest.raises(binding.ColatusError) as e:
        binding.colatus_init(4, np.ones(4), 0.0, 0, 0.3, 0, 0.7, 1.0, 0.02)
    assert e.value.status == binding.E_ARG and "eps" in str(e.value)
    with pytest.raises(binding.ColatusError) as e:
        binding.colatus_init(4, np.ones(4), 0.1, 0, 2.0, -1.0, 0.0, 1.0, 3.0)
    assert e.value.status == binding.E_ARG
    with pytest.raises(binding.ColatusError) as e:
        binding.colatus_init(2, np.array([1.0, np.nan]), 0.1, 0, 0.3, 0, 0.7, 1.0, 0.02)
    assert e.value.status == binding.E_ARG
    with pytest.raises(binding.ColatusError) as e:
        binding.colatus_init(0, np.ones(0), 0.1, 0, 0.3, 0, 0.7, 1.0, 0.02)
    assert e.value.status == binding.E_ARG


def test_input_recipes():
    g = inputs.grid16()
    assert g.N == 4096 and g.x.dtype == np.float64
    assert np.all(g.x == g.x.astype(np.float32))          # float32-representable
    assert np.allclose(g.m.sum(), 1.0) and np.all(g.v == 0)
    d = (g.x - g.q) * 16
    assert 0.03 < d.std() < 0.07                            # sigma = 0.05 spacing
    g2 = inputs.grid16()
    assert np.array_equal(g.x, g2.x)                        # seeded
    p = inputs.plummer_clusters(4000, 3)
    assert p.N == 4000 and abs(p.m.sum() - 1.0) < 1e-6
    e = inputs.ensemble(8, seed=5)
    assert all(1024 <= r.N <= 32768 for r in e)
    tr = inputs.tracers(4096, 64, 7)
    assert len(np.unique(tr)) == 64
    tau = inputs.lcdm_tau(2000)
    assert 4.7e-4 < tau < 4.9e-4


def test_tuning_cache_roundtrip(tmp_path):
    from paper_1208_3444_b300 import tuning
    p = str(tmp_path / "t.json")
    assert tuning.load(p) == {}
    k = tuning.key("B300", 32768, 1, True)
    tuning.save(p, {k: {"shape": 0, "ms": [0.3, 0.4, 0.9]}})
    assert tuning.load(p)[k]["shape"] == 0
    assert k == "B300|N=32768|prec=1|eqmass=1"
