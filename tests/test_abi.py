"""The C ABI library builds, loads without a GPU, exports every entry point
declared in include/hopf.h, and rejects bad arguments before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1712_08226_gb300 import _lib, build
    build.build()
    return _lib.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hopf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hopf_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "hopf_value" in names and "hopf_time_to_reach" in names and "hopf_trajectory" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_1712_08226_gb300 import _lib
    assert sorted(_lib.EXPORTS) == declared_functions()


def test_struct_layout_matches_header():
    # field order and types of the ctypes mirror follow the header's structs
    from paper_1712_08226_gb300 import _lib
    src = open(os.path.join(ROOT, "include", "hopf.h")).read()
    for cname, py in (("hopf_problem", _lib.HopfProblem), ("hopf_opts", _lib.HopfOpts),
                      ("hopf_mlp", _lib.HopfMlp)):
        body = re.search(r"typedef struct \{((?:(?!typedef struct).)*?)\}\s*" + cname + ";", src, re.S).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S).replace("*", " ")
        fields = []
        for decl in body.split(";"):
            for piece in decl.split(","):
                names = re.findall(r"[A-Za-z_][A-Za-z_0-9]*", piece)
                if names:
                    fields.append(names[-1])
        assert fields == [f[0] for f in py._fields_], (cname, fields)


def test_default_opts(lib):
    from paper_1712_08226_gb300 import _lib
    o = _lib.HopfOpts()
    lib.hopf_default_opts(ctypes.byref(o))
    assert o.N == 100 and o.gap_every == 8 and o.sigma_scale == 1.0 and o.tol_gap == 1e-5


def _call_value(lib, sysd, opts_kw=None, P=4):
    from paper_1712_08226_gb300 import api
    s = api.System.from_dict(sysd)
    opts = api.Options(**(opts_kw or {}))
    prob = s.c_struct()
    o = opts.c_struct(True)
    x = np.zeros((P, s.n), np.float32)
    t = np.ones(1, np.float32)
    outs = [np.zeros(P, np.float32), np.zeros((P, s.n), np.float32), np.zeros(P, np.float32),
            np.zeros(P, np.int32), np.zeros(P, np.int32)]
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    return lib.hopf_value(ctypes.byref(prob), ctypes.byref(o), P, vp(x), vp(t), 0, None,
                          *[vp(a) for a in outs], None)


def test_rejects_non_spd_target(lib):
    from inputs import workloads as wl
    sysd = wl.double_integrator(0.1)
    sysd["W"] = np.array([[1.0, 2.0], [2.0, 1.0]])
    assert _call_value(lib, sysd) == -2
    assert b"positive definite" in lib.hopf_last_error()


def test_rejects_non_finite_and_bad_options(lib):
    from inputs import workloads as wl
    sysd = wl.double_integrator(0.1)
    bad = dict(sysd)
    bad["A"] = np.array([[0.0, np.nan], [0.0, 0.0]])
    assert _call_value(lib, bad) == -5
    assert _call_value(lib, sysd, dict(tau=-1.0)) == -1
    assert _call_value(lib, sysd, dict(N=1, rule=1)) == -1
    assert _call_value(lib, sysd, dict(N=8, rule=2)) == -1      # Simpson needs odd N
    assert _call_value(lib, sysd, dict(N=9, rule=3)) == -1
    assert _call_value(lib, sysd, dict(sigma_scale=1.5)) == -1
    assert _call_value(lib, sysd, dict(gap_every=0)) == -1
    neg_box = dict(sysd)
    neg_box["half_widths"] = np.array([-1.0])
    assert _call_value(lib, neg_box) == -1


def test_empty_batch_needs_no_device(lib):
    from inputs import workloads as wl
    assert _call_value(lib, wl.double_integrator(0.1), P=0) == 0


def test_status_strings(lib):
    assert lib.hopf_status_string(0) == b"ok"
    assert lib.hopf_status_string(3).startswith(b"target unreachable")
    assert lib.hopf_status_string(-2).startswith(b"W not")


def test_stacked_entry_validates_before_touching_a_device(lib):
    # hopf_value_stacked checks copies, base size, every W block, and options
    from paper_1712_08226_gb300 import _lib as L
    from paper_1712_08226_gb300 import api
    from inputs import workloads as wl
    base = api.System.from_dict(wl.double_integrator(0.1))
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731

    def call(blocks, opts_kw=None, P=2):
        blocks = np.ascontiguousarray(blocks, dtype=np.float64)
        sp = L.HopfStacked(base.c_struct(), blocks.shape[0], blocks.ctypes.data_as(L.P_double))
        o = api.Options(**(opts_kw or {})).c_struct(False)
        k = blocks.shape[0]
        x = np.zeros((P, 2 * k), np.float32)
        t = np.ones(1, np.float32)
        outs = [np.zeros(P, np.float32), np.zeros((P, 2 * k), np.float32), np.zeros(P, np.float32),
                np.zeros(P, np.int32), np.zeros(P, np.int32)]
        return lib.hopf_value_stacked(ctypes.byref(sp), ctypes.byref(o), P, vp(x), vp(t), 0, None,
                                      *[vp(a) for a in outs], None)

    good = np.stack([0.1 * np.eye(2)] * 3)
    bad = good.copy()
    bad[2] = np.array([[1.0, 2.0], [2.0, 1.0]])
    assert call(bad) == -2 and b"block 2" in lib.hopf_last_error()
    nan = good.copy()
    nan[1, 0, 0] = np.nan
    assert call(nan) == -5
    assert call(np.stack([0.1 * np.eye(2)] * 65)) == -1          # at most 64 copies
    assert call(good, dict(accel=True)) == -1
    assert call(good, P=0) == 0                                    # empty batch: nothing to do


def test_python_constants_match_header_defines():
    from paper_1712_08226_gb300 import api
    src = open(os.path.join(ROOT, "include", "hopf.h")).read()
    defines = {k: int(v) for k, v in re.findall(r"#define\s+HOPF_([A-Z0-9_]+)\s+(-?\d+)\b", src)}
    pairs = {"LEFT_RIEMANN": api.LEFT_RIEMANN, "TRAPEZOID": api.TRAPEZOID, "SIMPSON": api.SIMPSON,
             "LEFT_FIXED": api.LEFT_FIXED, "BALL": api.BALL, "BOX": api.BOX, "FP32": api.FP32,
             "FP64": api.FP64, "VARS_INITIAL": api.VARS_INITIAL, "VARS_TERMINAL": api.VARS_TERMINAL}
    for name, val in pairs.items():
        assert defines[name] == val, name


def test_fixed_step_rule_validates_before_touching_a_device(lib):
    # the fixed-step rule needs terminal-time variables, a finite t_max and
    # fixed step sizes; unknown rules are refused
    from inputs import workloads as wl
    sysd = wl.double_integrator(0.1)
    assert _call_value(lib, sysd, dict(rule=3, N=16, t_max=2.0)) == -1
    assert b"terminal-time" in lib.hopf_last_error()
    assert _call_value(lib, sysd, dict(rule=3, N=16, t_max=float("inf"), variables=1)) == -1
    assert b"t_max" in lib.hopf_last_error()
    assert _call_value(lib, sysd, dict(rule=3, N=16, t_max=2.0, variables=1, adaptive=True)) == -1
    assert _call_value(lib, sysd, dict(rule=4, N=16)) == -1
    assert b"bad rule" in lib.hopf_last_error()
    # a valid fixed-step request with no points needs no device
    assert _call_value(lib, sysd, dict(rule=3, N=16, t_max=2.0, variables=1), P=0) == 0
