"""The state read that allocates no device memory (bm_read_state_noalloc).

Some callers must not allocate device memory while a simulation runs -- a
real-time control loop of an external rigid-body system reading state every
tick, where cudaMalloc/cudaFree would synchronise the device and stall, or a
process whose device memory a caching allocator already holds.  This test
calls that entry point through the C ABI and checks that it returns exactly
what the allocating bm_read_state returns, on two calls in a row, and that a
field larger than its 16 MiB staging array is refused.  The file is named so
that pytest collects it last.
"""
import numpy as np
import pytest

import bm_inputs as bi

pytestmark = pytest.mark.gpu

FIELDS = ("x", "v", "F", "D", "ut", "code", "mask1", "mask2", "X")


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2609_27342_gb300 as p
    from paper_2609_27342_gb300 import build
    build.build()
    p.load()
    return p


def test_noalloc_read_matches_read_state_twice(pkg):
    sc = bi.single_cut_cuboid(size=(0.04, 0.02, 0.02), edge_z0=0.0201, speed=1.0, n_down=100)
    g = pkg.Scene(sc)
    g.step(30)
    for call in range(2):
        ref = g.read(*FIELDS)
        got = g.read_noalloc(*FIELDS)
        for k in FIELDS:
            assert got[k].dtype == ref[k].dtype
            assert np.array_equal(got[k], ref[k]), (call, k)
        # the second call reads a changed state through the same array
        g.step(7)
    codes = g.read_noalloc("code")["code"]
    assert np.any(codes > 0), "the run must have assigned side labels"
    g.close()


def test_noalloc_read_rejects_fields_beyond_the_staging_array(pkg):
    from paper_2609_27342_gb300 import _abi as A
    X = bi.lattice_cuboid((0.32, 0.16, 0.16), 5e-3)  # 524,288 particles
    assert 9 * 4 * X.shape[0] > (16 << 20)
    sc = bi.Scene(X=X, dx=5e-3, V0=(5e-3) ** 3 / 8)
    g = pkg.Scene(sc)
    with pytest.raises(A.BMError) as e:
        g.read_noalloc("F")
    assert e.value.code == A.E_INVALID and "staging array" in str(e.value)
    # x (3 floats per particle) still fits and matches the allocating read
    assert np.array_equal(g.read_noalloc("x")["x"], g.read("x")["x"])
    g.close()
