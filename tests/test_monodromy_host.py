"""Host logic of the monodromy loop driver (monodromy.loops) against a fake
serving loop, no GPU: jobs finish out of order, some paths fail, and each
loop's way back lands on one of d hidden points.  The driver must keep at
most `per_round` loops in flight, submit a loop's way back only after its way
out succeeded, find every hidden point, never count a point twice or count a
failed path's end point, and stop once `patience * per_round` loops in a row
found nothing new."""
import numpy as np
import pytest

from paper_1501_06625_gb300 import libph, monodromy, synth


class FakeServer:
    def __init__(self, d, n, L, fail_every, seed):
        self.rng = np.random.default_rng(seed)
        self.pts = [self.rng.standard_normal(n) + 1j * self.rng.standard_normal(n) for _ in range(d)]
        self.n, self.L, self.fail_every = n, L, fail_every
        self.jobs, self.next_id, self.submitted = {}, 1, 0
        self.max_inflight = 0

    def submit(self, f, g, x0):
        jid = self.next_id
        self.next_id += 1
        self.submitted += 1
        ok = self.submitted % self.fail_every != 0
        out = np.zeros((self.L, 2, self.n))
        z = self.pts[self.rng.integers(len(self.pts))] * (1.0 if f == "Fb" else 1e3)
        out[0, 0], out[0, 1] = z.real, z.imag
        self.jobs[jid] = [int(self.rng.integers(1, 4)), ok, out, f]
        self.max_inflight = max(self.max_inflight, len(self.jobs))
        return jid

    def poll(self, jid, x):
        j = self.jobs[jid]
        j[0] -= 1                                   # finishes after a few polls
        if j[0] > 0:
            return False, None, None
        del self.jobs[jid]
        x[...] = j[2]
        st = {"status": libph.PH_OK if j[1] else libph.PH_STEPMIN, "newton_iters": 3}
        return True, st, 1.0


class FakeCtx:
    h = None

    def __init__(self):
        self.loaded = []

    def load(self, spec, L):
        name = {0: "F", 1: "G", 2: "Fb", 3: "Gb"}[len(self.loaded) % 4]
        self.loaded.append(name)
        return name

    def free(self, s):
        pass


@pytest.fixture
def fake(monkeypatch):
    holder = {}

    def create(ctx, max_n, pool_bytes, queue_cap):
        return holder["srv"]

    monkeypatch.setattr(libph, "ph_server_create", create)
    monkeypatch.setattr(libph, "ph_server_submit",
                        lambda ctx, srv, f, g, gs, x0, p: srv.submit(f, g, x0))
    monkeypatch.setattr(libph, "ph_server_poll", lambda ctx, srv, jid, x: srv.poll(jid, x))
    monkeypatch.setattr(libph, "ph_server_destroy", lambda srv: None)
    monkeypatch.setattr(monodromy.time, "sleep", lambda s: None)
    return holder


@pytest.mark.parametrize("d,fail_every", [(4, 7), (8, 5), (1, 1000)])
def test_loops_find_every_point(fake, d, fail_every):
    loop = synth.cyclic_monodromy_loop(1, 16)
    srv = FakeServer(d, 16, 2, fail_every, seed=d)
    fake["srv"] = srv
    res = monodromy.loops(FakeCtx(), loop, 2, {}, rounds=50, per_round=6, patience=3)
    found = res["points"][1:]                        # after the start point
    assert len(found) == d
    for p in srv.pts:                                # every hidden point, once
        assert sum(np.allclose(q[0, 0] + 1j * q[0, 1], p) for q in found) == 1
    assert srv.max_inflight <= 6
    assert res["paths"] == srv.submitted and res["failed"] > 0 or fail_every == 1000
    assert res["loops"] <= 50 * 6
    assert not srv.jobs                              # nothing left in flight


def test_loops_stop_after_patience(fake):
    loop = synth.cyclic_monodromy_loop(1, 16)
    srv = FakeServer(2, 16, 2, 1000, seed=5)
    fake["srv"] = srv
    res = monodromy.loops(FakeCtx(), loop, 2, {}, rounds=1000, per_round=4, patience=2)
    # once both points are known, at most 2 x 4 loops in a row end without a
    # new point before no loop starts, plus the loops then in flight
    assert res["loops"] < 100
    assert len(res["points"]) == 3
