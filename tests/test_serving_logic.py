"""Host-side logic of the serving loop on CPU, with the device layer faked:
admission by budget and arrival time, retirement, and latency bookkeeping."""
import types

import numpy as np
import pytest


class FakeEvent:
    def __init__(self, *a, **k):
        self.t = 0.0

    def record(self, stream=None):
        pass

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return 1.0


class FakeBatch:
    def __init__(self, *a, **k):
        self.scenes = []
        self.steps = []

    def step(self, n):
        self.steps.append(n)
        for sc in self.scenes:  # members advance up to their stop substep
            sc.step_count = sc.step_count + n if sc.stop < 0 else min(sc.stop, sc.step_count + n)

    def set_tiles(self, chunk, ntile, variant):
        self.shape = (chunk, ntile, variant)

    def close(self):
        pass


class FakeScene:
    def __init__(self, batch, sc):
        self.n = sc.n
        self.spec = sc
        self.batch = batch
        batch.scenes.append(self)
        self.closed = False
        self.step_count = 0
        self.stop = -1

    def set_stop(self, n):
        self.stop = n

    def read_noalloc(self, *names):
        return {"x": np.full((self.n, 3), float(self.n), np.float32)}

    read = read_noalloc

    def info(self):
        return types.SimpleNamespace(error_bits=0, step=self.step_count)

    def tool_wrench(self):
        return np.zeros(6)

    def close(self):
        self.closed = True
        self.batch.scenes.remove(self)


@pytest.fixture
def server_mod(monkeypatch):
    torch = pytest.importorskip("torch")
    from paper_2609_27342_gb300 import serving
    monkeypatch.setattr(serving, "Batch", FakeBatch)
    monkeypatch.setattr(serving.Scene, "in_batch", classmethod(lambda cls, b, sc: FakeScene(b, sc)))
    monkeypatch.setattr(serving, "footprint", lambda sc: (sc.n, sc.n // 2, 1, sc.n * 100))
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: None)
    return serving


def _sc(n):
    return types.SimpleNamespace(n=n, blade=None)


def test_budget_limits_resident_scenes(server_mod):
    srv = server_mod.Server(budget_bytes=250 * 100, max_scenes=8, max_chunk=10)
    for n, steps in [(100, 20), (100, 35), (100, 10)]:
        srv.submit(_sc(n), steps)
    st = srv.run(realtime=False)
    assert st["requests"] == 3
    # two scenes of 100 fit the 250-particle budget; the third waits
    assert all(k == 10 for k in srv.batch.steps)
    r = srv.results
    assert r[2].admitted_s >= min(r[0].finished_s, r[1].finished_s)
    assert st["particle_substeps"] == 100 * (20 + 35 + 10)


def test_requests_stop_exactly_inside_whole_chunks(server_mod):
    srv = server_mod.Server(budget_bytes=10 ** 9, max_scenes=8, max_chunk=16)
    srv.submit(_sc(10), 7)
    srv.submit(_sc(20), 30)
    st = srv.run(realtime=False)
    # the batch always advances whole chunks; each scene stops on the device at
    # its own length (the server checks the substep count when it retires it)
    assert srv.batch.steps == [16, 16]
    assert srv.results[0].n_substeps == 7 and srv.results[1].n_substeps == 30
    assert st["particle_substeps"] == 10 * 7 + 20 * 30
    assert st["offered_load"] is None  # both arrived at once: no span to divide by


def test_request_larger_than_budget_is_reported(server_mod):
    srv = server_mod.Server(budget_bytes=100, max_scenes=8)
    srv.submit(_sc(10), 5)
    with pytest.raises(RuntimeError):
        srv.run(realtime=False)
