"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every function include/ph.h declares, its structs
and the oracle's have the field names and types, in order, that their
headers declare, and its step-size controller (the code the device
controller runs) agrees with the oracle's independent implementation on
scripted and random outcome sequences."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
from paper_1501_06625_gb300 import build, libph, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return libph.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ph.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(ph_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert set(names) == set(libph.EXPORTS)
    for name in names:
        assert hasattr(lib, name), name
    assert "sm_103a" in libph.ph_version()


def _ph_drive(params, outcomes):
    st = libph.CtrlState()
    p = libph.ph_ctrl_init(st, params)
    ts = []
    for ok in outcomes:
        t = libph.ph_ctrl_next_t(st, p)
        if t < 0:
            break
        ts.append(t)
        libph.ph_ctrl_report(st, p, t, ok)
    return ts, {k: getattr(st, k) for k, _ in libph.CtrlState._fields_}


def _orc_drive(orc, params, outcomes):
    c = orc.Controller(params)
    ts = []
    for ok in outcomes:
        t = c.next_t()
        if t < 0:
            break
        ts.append(t)
        c.report(t, ok)
    return ts, c.state


@pytest.mark.parametrize("seed", range(12))
def test_controller_matches_oracle(lib, orc, seed):
    rng = np.random.default_rng(seed)
    params = synth.default_params(2, max_dt=float(rng.choice([0.05, 0.1, 0.25])),
                                  min_dt=float(rng.choice([1e-3, 1e-6])),
                                  max_steps=int(rng.integers(5, 200)),
                                  fixed_steps=int(rng.choice([0, 0, 0, 7])))
    outcomes = rng.random(400) < rng.uniform(0.3, 0.95)
    a = _ph_drive(params, outcomes)
    b = _orc_drive(orc, params, outcomes)
    assert a == b


def test_controller_hand_trace(lib):
    ts, st = _ph_drive(synth.default_params(2, max_dt=0.25, min_dt=0.01), [1, 0, 1, 1, 1, 1, 0, 1, 1])
    assert ts == [0.25, 0.5, 0.375, 0.5, 0.625, 0.875, 1.0, 1.0]
    assert st["done"] == 1 and st["status"] == libph.PH_OK


# ---- struct layouts: the header's typedefs against the ctypes mirrors -----------

_CTYPES = {"double": C.c_double, "int32_t": C.c_int32, "int64_t": C.c_int64}


def _header_structs(path):
    """{typedef name: [(field, C type name), ...]} of the anonymous-struct
    typedefs of a C header, fields in declaration order (comments removed,
    `type a, b;` lists expanded)."""
    import re
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", src, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            ctype, rest = decl.split(None, 1)
            fields += [(f.strip(), ctype) for f in rest.split(",")]
        out[name] = fields
    return out


def _check_mirror(structs, cname, pyclass):
    fields = structs[cname]
    mirror = [(n, t) for n, t in pyclass._fields_]
    assert [n for n, _ in fields] == [n for n, _ in mirror], cname
    for (_, ct), (_, pt) in zip(fields, mirror):
        assert _CTYPES[ct] is pt, (cname, ct, pt)


def test_library_structs_match_the_header():
    structs = _header_structs(os.path.join(ROOT, "include", "ph.h"))
    for cname, py in (("ph_track_params", libph.TrackParams), ("ph_path_stats", libph.PathStats),
                      ("ph_step_record", libph.StepRecord), ("ph_server_config", libph.ServerConfig),
                      ("ph_ctrl_state", libph.CtrlState)):
        _check_mirror(structs, cname, py)


def test_oracle_structs_match_its_header():
    structs = _header_structs(os.path.join(ROOT, "oracle", "oracle.h"))
    for cname, py in (("orc_params", oracle.Params), ("orc_stats", oracle.Stats),
                      ("orc_record", oracle.Record), ("orc_ctrl", oracle.Ctrl)):
        _check_mirror(structs, cname, py)


def test_linear_contraction_rule(lib):
    """The precision form's test on three successive update norms (the code
    the device runs): quadratic convergence passes, a corrector limited by
    its solves (a constant contraction) is caught; stalling, diverging and
    degenerate input are not."""
    lc = libph.ph_ctrl_linear_contraction
    assert not lc(1e-2, 1e-4, 1e-8)            # r0 = r1^2
    assert lc(1e-3, 1e-6, 1e-9)                # r0 = r1
    assert not lc(1e-3, 1e-3, 1e-3)            # not contracting
    assert not lc(1e-3, 1e-2, 1e-1)            # diverging
    for bad in ((0.0, 1.0, 0.5), (1.0, 0.0, 0.0), (1.0, 0.5, float("inf")),
                (1.0, 0.5, float("nan")), (-1.0, 0.5, 0.25)):
        assert not lc(*bad), bad

    def updates(delta, x, steps=3):
        # Newton on x^2 - 2 with the derivative off by a relative delta, as a
        # low-precision solve of relative error delta would leave it
        out = []
        for _ in range(steps):
            dx = (x * x - 2.0) / (2.0 * x * (1.0 + delta))
            out.append(abs(dx))
            x -= dx
        return out

    assert not lc(*updates(0.0, 1.5))          # exact derivative: quadratic
    assert lc(*updates(1e-2, 2.0 ** 0.5 + 1e-3))   # error contracts by ~delta per step
