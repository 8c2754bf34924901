"""Edge cases and failure detection through the C ABI (GPU).

Invalid arguments are refused before any work is enqueued; degenerate sizes
(zero substeps, an empty batch) are no-ops; failures made on the host -- a
NaN velocity, an inverted deformation gradient, more distinct codes at one
node than it has logical grids -- raise the sticky device error word of that
scene only, and the scenes beside it in a batch go on bit for bit.  No GPU
fault is involved: every one of these is a checked condition in a kernel.
"""
import copy

import numpy as np
import pytest

import bm_inputs as bi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2609_27342_gb300 as p
    from paper_2609_27342_gb300 import build
    build.build()
    p.load()
    return p


def test_invalid_arguments_are_refused(pkg):
    from paper_2609_27342_gb300 import _abi as A

    sc = bi.single_cut_cuboid()
    for field, bad in (("E", -1.0), ("dt", 0.0), ("dx", 0.0), ("nu", 0.5), ("rho", 0.0)):
        s2 = copy.copy(sc)
        setattr(s2, field, bad)
        with pytest.raises(pkg.BMError) as e:
            pkg.Scene(s2)
        assert e.value.code == A.E_INVALID, field
    s2 = copy.copy(sc)
    s2.X = np.zeros((0, 3))
    with pytest.raises(pkg.BMError) as e:
        pkg.Scene(s2)
    assert e.value.code == A.E_INVALID
    s2 = copy.deepcopy(sc)
    s2.blade.segments[0].cut_id = 32  # digits 0..31 only
    with pytest.raises(pkg.BMError) as e:
        pkg.Scene(s2)
    assert e.value.code == A.E_TOO_MANY_CUTS
    g = pkg.Scene(sc)
    with pytest.raises(pkg.BMError):
        g.step(-1)
    g.close()


def test_degenerate_sizes_are_no_ops(pkg):
    sc = bi.single_cut_cuboid()
    g = pkg.Scene(sc)
    g.step(3)
    before = g.read("x", "v", "F")
    g.step(0)
    after = g.read("x", "v", "F")
    for k in before:
        assert np.array_equal(before[k], after[k])
    b = pkg.Batch(max_particles=1000, max_nodes=1000, max_scenes=2)
    b.step(5)  # no members
    assert b.errors() == 0
    b.close()
    g.close()


def _batch_of(pkg, specs):
    fp = [pkg.footprint(s) for s in specs]
    members = [pkg.Scene(s) for s in specs]
    b = pkg.Batch(max_particles=sum(s.n for s in specs), max_nodes=sum(f[1] for f in fp),
                  max_scenes=len(specs), max_bricks=sum(f[2] for f in fp))
    for m in members:
        b.add(m)
    return b, members


def test_nonfinite_and_inverted_are_flagged_per_scene(pkg):
    from paper_2609_27342_gb300 import _abi as A

    specs = bi.batched_scenes(3, seed=11)
    alone = pkg.Scene(specs[2])
    b, m = _batch_of(pkg, specs)
    b.step(2)
    alone.step(2)
    v = m[0].read("v")["v"]
    v[5] = np.nan
    m[0].write(v=v)
    F = m[1].read("F")["F"]
    F[7] = np.array([-1.0, 0, 0, 0, 1.0, 0, 0, 0, 1.0], np.float32)  # det F < 0
    m[1].write(F=F)
    b.step(3)
    alone.step(3)
    assert m[0].info().error_bits & A.ERRBIT_NONFINITE
    assert m[1].info().error_bits & A.ERRBIT_INVERTED
    assert m[2].info().error_bits == 0
    assert b.errors() & (A.ERRBIT_NONFINITE | A.ERRBIT_INVERTED) == (A.ERRBIT_NONFINITE | A.ERRBIT_INVERTED)
    # the third scene is untouched by its neighbours' failures
    got, ref = m[2].read("x", "v", "F"), alone.read("x", "v", "F")
    for k in got:
        assert np.array_equal(got[k], ref[k]), k
    b.close()
    alone.close()


def test_slot_overflow_is_flagged(pkg):
    """Seventeen particles around one node carrying 17 distinct nonzero codes
    (18 with the unlabelled rest) exceed the 16 logical grids a node holds."""
    from paper_2609_27342_gb300 import _abi as A

    sc = bi.single_cut_cuboid()
    g = pkg.Scene(sc)
    X = np.asarray(sc.X, np.float64)
    base = np.floor((X - np.asarray(sc.origin)) / sc.dx - 0.5).astype(int)
    mid = np.array([8, 4, 4])
    node = mid + 1
    near = np.nonzero(np.all((base >= node - 2) & (base <= node), axis=1))[0]
    assert len(near) >= 17
    s1 = np.zeros(sc.n, np.uint32)
    s1[near[:17]] = (np.uint32(1) << np.arange(17, dtype=np.uint32))
    g.write(mask1=s1)
    assert g.info().error_bits & A.ERRBIT_SLOT_OVERFLOW
    g.close()
