"""Continuous-batching server (NEXT-1): requests admitted as they arrive and as
the HBM budget frees up, served in one device batch; each result must equal
the same rollout run alone (bit-identical: every sum has a fixed order)."""
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


def _requests():
    reqs = bi.serving_requests(n_requests=5, seed=7, n_min=3000, n_max=40000,
                               steps_min=60, steps_max=160)
    return reqs


def _alone(pkg, req):
    g = pkg.Scene(req.scene)
    g.step(req.n_substeps)
    x = g.read("x")["x"]
    w = g.tool_wrench()
    g.close()
    return x, w


def test_served_results_equal_alone(pkg):
    from paper_2609_27342_gb300.serving import Server
    reqs = _requests()
    srv = Server(budget_bytes=2 << 30, max_scenes=16, max_chunk=8)
    # three arrive together, two join while those are running
    for i, r in enumerate(reqs):
        srv.submit(r.scene, r.n_substeps, arrival_s=0.0 if i < 3 else 0.005 * (i - 2))
    st = srv.run(realtime=True, timeout_s=300)
    assert st["requests"] == len(reqs)
    assert st["step_ms_p99"] >= st["step_ms_p50"] > 0
    overlapped = any(a.admitted_s < b.finished_s and b.admitted_s < a.finished_s
                     for a in srv.results.values() for b in srv.results.values() if a is not b)
    assert overlapped, "requests must share the device"
    for rid, r in enumerate(reqs):
        x, w = _alone(pkg, r)
        res = srv.results[rid]
        assert res.error_bits == 0
        assert np.array_equal(res.x, x)
        assert np.array_equal(res.wrench, w)
    srv.close()


def test_budget_admission_serialises_but_keeps_results(pkg):
    from paper_2609_27342_gb300.serving import Server
    from paper_2609_27342_gb300 import footprint
    reqs = _requests()[:3]
    biggest = max(footprint(r.scene)[3] for r in reqs)
    srv = Server(budget_bytes=int(biggest * 1.05), max_scenes=8, max_chunk=16,
                 max_particles=200000)
    for r in reqs:
        srv.submit(r.scene, r.n_substeps)
    srv.run(realtime=False)
    fp = {rid: footprint(r.scene)[3] for rid, r in enumerate(reqs)}
    res = srv.results
    # at every admission, the resident scenes plus the new one fit the budget
    for b in res.values():
        resident = [a for a in res.values() if a is not b and
                    a.admitted_s <= b.admitted_s < a.finished_s]
        assert sum(fp[a.request_id] for a in resident) + fp[b.request_id] <= srv.budget
    assert any(sum(fp[i] for i in (a, b)) > srv.budget for a in fp for b in fp if a != b), \
        "the budget must have forced some requests to wait"
    for rid, r in enumerate(reqs):
        x, _ = _alone(pkg, r)
        assert np.array_equal(srv.results[rid].x, x)
    srv.close()


def test_stop_substep_freezes_a_scene_exactly(pkg):
    """bm_scene_set_stop: a scene stopped at n substeps inside a batch that
    keeps stepping equals the same scene run alone for n substeps, bit for
    bit; moving the stop lets it continue, again equal to a run alone."""
    reqs = _requests()[:3]
    fps = [pkg.footprint(r.scene) for r in reqs]
    b = pkg.Batch(max_particles=sum(f[0] for f in fps), max_nodes=sum(f[1] for f in fps), max_scenes=3,
                  graph_chunk=8)
    members = [pkg.Scene.in_batch(b, r.scene) for r in reqs]
    members[0].set_stop(13)
    members[1].set_stop(0)  # frozen from the start
    b.step(24)
    assert members[0].info().step == 13 and members[1].info().step == 0 and members[2].info().step == 24

    def alone(sc, n):
        g = pkg.Scene(sc)
        g.step(n)
        out = g.read("x", "v", "F", "code")
        g.close()
        return out

    for m, r, n in zip(members, reqs, (13, 0, 24)):
        got, want = m.read("x", "v", "F", "code"), alone(r.scene, n)
        for k in want:
            assert np.array_equal(got[k], want[k]), (n, k)
    members[0].set_stop(-1)
    b.step(5)
    got, want = members[0].read("x", "v", "F", "code"), alone(reqs[0].scene, 18)
    for k in want:
        assert np.array_equal(got[k], want[k]), k
    b.close()
