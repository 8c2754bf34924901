"""Device memory owned by PyTorch's caching allocator (the bm_alloc callbacks).

The C ABI takes the caller's allocate/free callbacks; the Python binding
passes PyTorch's caching allocator (``TorchAllocator``), so a scene, a batch
and a server can live in memory that torch owns and accounts for.  Checked
here: the results are bit-identical to the cudaMalloc path (the kernels do
not depend on who allocated the pools), torch's allocated-bytes counter
grows by about the scene's footprint while it lives, and the memory goes back
to torch when the scene, batch or server closes.
"""
import numpy as np
import pytest

import bm_inputs as bi

pytestmark = pytest.mark.gpu

FIELDS = ("x", "v", "F", "D", "code")


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2609_27342_gb300 as p
    from paper_2609_27342_gb300 import build
    build.build()
    p.load()
    return p


def _scene():
    return bi.single_cut_cuboid(size=(0.04, 0.02, 0.02), edge_z0=0.0201, speed=1.0, n_down=120)


def test_scene_in_torch_memory_matches_cudamalloc(pkg):
    import torch
    sc = _scene()
    ref = pkg.Scene(sc, wrench_history=60)
    ref.step(60)
    want = ref.read(*FIELDS)
    w_ref = ref.wrench_history(0, 60)
    ref.close()

    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    al = pkg.TorchAllocator(torch.cuda.current_device())
    g = pkg.Scene(sc, allocator=al, wrench_history=60)
    grown = torch.cuda.memory_allocated() - before
    fp = pkg.footprint(sc)[3]
    # the pools come from torch: its counter grows by about the footprint
    assert 0.5 * fp <= grown <= 2.0 * fp, (grown, fp)
    g.step(60)
    got = g.read(*FIELDS)
    for k in FIELDS:
        assert np.array_equal(got[k], want[k]), k
    assert np.array_equal(g.wrench_history(0, 60), w_ref)
    g.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before


def test_batch_in_torch_memory_matches_cudamalloc(pkg):
    import torch
    scenes = bi.batched_scenes(n_scenes=3, seed=11, n_max=12000, n_substeps=200)
    fps = [pkg.footprint(s) for s in scenes]
    cap_p = sum(f[0] for f in fps)
    cap_n = sum(f[1] for f in fps)

    def run(allocator):
        b = pkg.Batch(max_particles=cap_p, max_nodes=cap_n, max_scenes=3, graph_chunk=8,
                      allocator=allocator)
        members = [pkg.Scene.in_batch(b, s) for s in scenes]
        b.step(40)
        out = [m.read("x", "v", "F", "code") for m in members]
        for m in members:
            m.close()
        b.close()
        return out

    want = run(None)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    got = run(pkg.TorchAllocator(torch.cuda.current_device()))
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
    for a, b in zip(want, got):
        for k in a:
            assert np.array_equal(a[k], b[k]), k


def test_server_in_torch_memory_matches_cudamalloc(pkg):
    import torch
    from paper_2609_27342_gb300.serving import Server
    reqs = bi.serving_requests(n_requests=3, seed=5, n_min=3000, n_max=12000,
                               steps_min=30, steps_max=60)

    def serve(allocator):
        srv = Server(budget_bytes=1 << 30, max_scenes=8, max_chunk=8, allocator=allocator)
        for r in reqs:
            srv.submit(r.scene, r.n_substeps, arrival_s=0.0)
        srv.run(realtime=False, timeout_s=300)
        out = {rid: (r.x.copy(), r.wrench.copy()) for rid, r in srv.results.items()}
        srv.close()
        return out

    want = serve(None)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    got = serve(pkg.TorchAllocator(torch.cuda.current_device()))
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
    assert sorted(got) == sorted(want)
    for rid in want:
        assert np.array_equal(got[rid][0], want[rid][0])
        assert np.array_equal(got[rid][1], want[rid][1])
