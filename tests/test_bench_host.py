"""Host logic of bench.py's legs against a fake library, no GPU.  Serving: the
sequential rate is measured before the server runs, every request of the
closed loop, the Poisson stream and the sweep of offered loads (0.5, 1 and 2
x the sequential capacity) is submitted and waited for, and the figures come
out with the keys the JSON line carries.  The whole sparse-path leg: x* is
tracked backwards, its end rounded to roots of x_i^{d_i} = 1, the forward path
checked against x*, and a failed backward path ends the leg."""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1501_06625_gb300 import synth  # noqa: E402


class FakeLib:
    def __init__(self):
        self.submitted, self.waited, self.tracked = 0, 0, 0

    def ph_server_create(self, h, max_n, pool_bytes, queue_cap):
        return object()

    def ph_server_submit(self, h, srv, f, g, gam, x0, params):
        self.submitted += 1
        return self.submitted

    def ph_server_wait(self, h, srv, jid, timeout_ms):
        self.waited += 1
        return {"status": 0, "newton_iters": 4}, 2.0

    def ph_server_info(self, srv):
        return {"kernel_launches": 3}

    def ph_server_destroy(self, srv):
        pass

    def ph_track_path(self, h, f, g, gam, x0, params, x):
        self.tracked += 1
        time.sleep(0.002)
        return 0, {}, []


class FakeCtx:
    h = None

    def load(self, spec, L):
        return (spec.n, L)


def test_serving_leg_sweeps_offered_loads():
    lib = FakeLib()
    nreq, m = 20, 12
    out = bench.serve_leg(lib, synth, FakeCtx(), nreq, seed=1, sweep_requests=m)
    assert lib.tracked == 16                                    # the sequential sample
    expected = min(64, nreq) + nreq + nreq + 3 * m
    assert lib.submitted == lib.waited == expected
    seq = out["sequential_single_path"]["paths_per_s"]
    rates = out["poisson_vs_sequential_capacity"]["rates"]
    assert sorted(rates) == ["0.5x", "1x", "2x"]
    for key, mult in (("0.5x", 0.5), ("1x", 1.0), ("2x", 2.0)):
        assert np.isclose(rates[key]["offered_per_s"], mult * seq)
        assert rates[key]["paths_per_s"] > 0 and rates[key]["p99_ms"] == 2.0
    assert out["poisson_vs_sequential_capacity"]["requests_per_rate"] == m
    for key in ("closed_loop", "poisson_0.8", "vs_sequential", "kernel_launches"):
        assert key in out
    # a given sequential rate is used as it is, and nothing is tracked alone
    lib2 = FakeLib()
    out2 = bench.serve_leg(lib2, synth, FakeCtx(), nreq, seed=1, seq_rate=50.0, sweep_requests=m)
    assert lib2.tracked == 0
    assert np.isclose(out2["poisson_vs_sequential_capacity"]["rates"]["2x"]["offered_per_s"], 100.0)


def test_oracle_all_cores_figure():
    """The all-cores oracle figure: one independent path per worker process
    (spawned), all corrector steps over the slowest worker's time."""
    out = bench.oracle_all_cores(1, "dd", 0.5, cores=2)
    assert out["cores"] == 2 and out["kind"] == "oracle" and out["value"] > 0
    assert "seeds 1..2" in out["sample"]


class _FakeTensor:
    def __init__(self, a):
        self.a = np.array(a, dtype=np.float64)

    def cpu(self):
        return self

    def numpy(self):
        return self.a


class _FakeTorch:
    """The few torch calls of the whole-path legs, on the host."""

    class cuda:
        @staticmethod
        def current_stream(dev):
            return None

        class Event:
            def __init__(self, enable_timing=True):
                pass

            def record(self, stream):
                pass

            def synchronize(self):
                pass

            def elapsed_time(self, other):
                return 1500.0

    @staticmethod
    def tensor(a, device=None):
        return _FakeTensor(a)

    @staticmethod
    def empty_like(t):
        return _FakeTensor(np.zeros_like(t.a))


class _PathLib:
    """ph_track_path for the sparse whole-path leg: the backward path (start
    system f as its second argument) ends near a root of x_i^{d_i} = 1, the
    forward path ends at x*."""
    PH_OK = 0

    def __init__(self, xs, back_ok=True):
        from paper_1501_06625_gb300 import libph
        self.STATUS_NAMES = libph.STATUS_NAMES
        self.xs, self.back_ok, self.calls, self.start = xs, back_ok, [], None

    def ph_track_path(self, h, f, g, gam, x0, params, xo):
        self.calls.append("back" if g is not None else "forward")
        n = len(self.xs)
        if g is not None:
            if not self.back_ok:
                return 5, {"steps": 401, "t_final": 0.7}, []
            z = np.exp(2j * np.pi * np.arange(n) / 7.0) * (1 + 1e-9)   # near roots of unity
            xo[0, 0], xo[0, 1] = z.real, z.imag
            return 0, {"steps": 300, "t_final": 1.0}, []
        self.start = x0.a.copy()
        xo.a[0, 0], xo.a[0, 1] = self.xs.real, self.xs.imag
        return 0, {"steps": 310, "accepted": 250, "rejected": 60, "newton_iters": 900,
                   "t_final": 1.0}, []


class _FreeCtx(FakeCtx):
    def free(self, f):
        pass


def test_sparse_whole_path_leg_host_logic():
    _, xs = synth.sparse512_planted(1, "qd")
    lib = _PathLib(xs)
    out = bench.sparse512_whole_path(lib, synth, _FreeCtx(), _FakeTorch, None, seed=1, max_steps=50)
    assert lib.calls == ["back", "forward"]
    # the forward start point: the nearest roots of x_i^{d_i} = 1, exactly on the unit circle
    z = lib.start[0, 0] + 1j * lib.start[0, 1]
    assert np.allclose(np.abs(z), 1.0, atol=1e-15)
    assert out["ok"] and out["err_vs_planted"] == 0.0 and out["status"] == "OK"
    assert out["steps"] == 310 and abs(out["paths_per_s"] - 1 / 1.5) < 1e-12
    assert out["corrector_steps_per_s"] == 900 / 1.5


def test_sparse_whole_path_leg_stops_after_a_failed_backward_path():
    _, xs = synth.sparse512_planted(1, "qd")
    lib = _PathLib(xs, back_ok=False)
    out = bench.sparse512_whole_path(lib, synth, _FreeCtx(), _FakeTorch, None, seed=1, max_steps=50)
    assert lib.calls == ["back"]
    assert out["backward_status"] == "MAXSTEPS" and out["backward_t_final"] == 0.7
    assert "ok" not in out
