"""Host-side checks of the CUDA library (no GPU needed).

The library builds for sm_103a, loads, exports every entry point declared in
include/hgks.h, computes footprints, and refuses to run without a device.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(hgks_[a-z0-9_]+)\s*\(", text))
    return names


def test_exports_every_declared_symbol():
    from paper_2207_01173_gb300 import hgks
    L = hgks.lib()
    decl = declared_symbols()
    assert "hgks_step" in decl and "hgks_create" in decl
    missing = [n for n in sorted(decl) if not hasattr(L, n)]
    assert not missing, missing
    assert set(hgks.EXPORTS) <= decl


def test_footprint_bytes_host_only():
    from paper_2207_01173_gb300 import hgks
    small = hgks.footprint_bytes((32, 32, 32))
    big = hgks.footprint_bytes((256, 256, 256))
    assert 0 < small < big
    # about 1.5 kB per cell at FP64 for the buffers the step keeps on the device
    assert 1000 < big / 256 ** 3 < 4000
    assert hgks.footprint_bytes((0, 4, 4)) == 0


def test_create_without_device_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2207_01173_gb300 import hgks
    with pytest.raises(hgks.HgksError) as e:
        hgks.Solver((8, 8, 8))
    assert e.value.status == hgks.HGKS_ERR_CUDA


def test_invalid_arguments_rejected_before_device():
    from paper_2207_01173_gb300 import hgks
    with pytest.raises(hgks.HgksError) as e:
        hgks.Solver((8, 8, 8), gamma=1.0)
    assert e.value.status == hgks.HGKS_ERR_INVALID_ARG
    with pytest.raises(hgks.HgksError) as e:
        hgks.Solver((8, 2, 8), bc_lo=(0, 1, 0), bc_hi=(0, 1, 0))
    assert e.value.status == hgks.HGKS_ERR_INVALID_ARG
    # an empty grid
    with pytest.raises(hgks.HgksError) as e:
        hgks.Solver((0, 8, 8))
    assert e.value.status == hgks.HGKS_ERR_INVALID_ARG
    # sub-domain sides: z only, and at least three planes
    with pytest.raises(hgks.HgksError) as e:
        hgks.Solver((8, 8, 8), bc_lo=(2, 0, 0), bc_hi=(2, 0, 0))
    assert e.value.status == hgks.HGKS_ERR_INVALID_ARG and "z only" in str(e.value)
    with pytest.raises(hgks.HgksError) as e:
        hgks.Solver((8, 8, 2), bc_lo=(0, 0, 2), bc_hi=(0, 0, 2))
    assert e.value.status == hgks.HGKS_ERR_INVALID_ARG
    with pytest.raises(hgks.HgksError) as e:
        hgks.Solver((8, 8, 8), bc_lo=(0, 0, 3), bc_hi=(0, 0, 0))
    assert e.value.status == hgks.HGKS_ERR_INVALID_ARG and "unknown" in str(e.value)


def test_batch_workload_is_seeded_and_in_range():
    from paper_2207_01173_gb300.workloads import batch_tgv_problems
    a, b = batch_tgv_problems(), batch_tgv_problems()
    assert a == b and len(a) == 64
    for n, Ma, Re in a:
        assert all(v in (24, 32, 48, 64, 96) for v in n)
        assert 0.1 <= Ma <= 0.5 and 400.0 <= Re <= 3200.0
    assert len({n for n, _, _ in a}) > 20  # uneven grids


def test_flop_model_counts_the_kernel_arithmetic():
    """The roofline's algorithmic flops come from running the kernels' own
    templated arithmetic on the host with a counting scalar; the counts are a
    property of the code (they change only when the arithmetic does)."""
    from paper_2207_01173_gb300 import hgks
    m = hgks.flop_model((256, 256, 256))
    assert m["flux_per_face"] == 13342 and m["div_per_face_flux"] == 82 and m["special_per_face_flux"] == 32
    assert m["normal_per_face"] == 1068 and m["tan1_per_pos"] == 2250
    # a step: two stages x three directions of each pass plus the cell passes
    faces = 257 * 256 * 256
    assert 2 * 3 * m["flux_per_face"] * faces < m["per_step"] < 1.2 * 2 * 3 * (
        m["flux_per_face"] * faces + m["tan1_per_pos"] * 257 * 256 * 260 + m["normal_per_face"] * 257 * 260 * 260)
