"""Writes the stored expected values used by the GPU parity tests.

Every number here comes from the FP64 oracle (oracle/), run on the seeded
inputs of inputs/workloads.py; nothing is read back from the CUDA path.
Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from inputs import workloads as wl  # noqa: E402
from oracle import hopf as oh  # noqa: E402

OUT = os.path.dirname(os.path.abspath(__file__))


def dump(name, meta, **arrays):
    doc = dict(meta=meta, **{k: np.asarray(v).tolist() for k, v in arrays.items()})
    with open(os.path.join(OUT, name), "w") as f:
        json.dump(doc, f, separators=(",", ":"))
    print("wrote", name)


def random10_values(P=320):
    w = wl.workload_random10(P)
    r = oh.value(w["system"], w["x"], w["t"], w["N"], w["rule"], tau=w["tau"], tol=1e-10,
                 max_iter=400000)
    assert np.all(r["status"] == oh.OK)
    dump("random10_values.json",
         dict(source="oracle.hopf.value", workload="random_n10_m2 (seed 1), x~N(0,4I) seed 2, first P points",
              P=P, t=w["t"], N=w["N"], rule="left_riemann", tau=w["tau"], oracle_tol=1e-10),
         phi=r["phi"], p=r["p"], gap=r["gap"])


def di_values(P=64):
    w = wl.workload_di(P)
    T = 1.5
    r = oh.value(w["system"], w["x"], T, w["N"], w["rule"], tau=w["tau"], tol=1e-12, max_iter=400000)
    assert np.all(r["status"] == oh.OK)
    dump("di_values_T1.5.json",
         dict(source="oracle.hopf.value", workload="double integrator, r=0.1, x~U[-2,2]^2 seed 0",
              P=P, T=T, N=w["N"], rule="trapezoid", tau=w["tau"], oracle_tol=1e-12),
         phi=r["phi"], p=r["p"])


def di_time_to_reach(P=64):
    w = wl.workload_di(P)
    r = oh.time_to_reach(w["system"], w["x"], w["t_max"], w["N"], w["rule"], tau=w["tau"],
                         tol_T=1e-8, tol_gap=1e-10)
    dump("di_time_to_reach.json",
         dict(source="oracle.hopf.time_to_reach", workload="double integrator, r=0.1, x~U[-2,2]^2 seed 0",
              P=P, t_max=w["t_max"], N=w["N"], rule="trapezoid", tau=w["tau"], oracle_tol_T=1e-8),
         T=r["T"], p=r["p"], status=r["status"])


def box_values(P=200):
    # small-state box-control system (m = 1): chain of 2 masses, 4 states
    sysd = wl.spring_chain(masses=2, actuators=1, radius_target=0.5)
    x = wl.normal_points(31, P, 4, 1.0)
    r = oh.value(sysd, x, 1.7, 64, oh.LEFT_RIEMANN, tau=0.5, tol=1e-10, max_iter=400000)
    assert np.all(r["status"] == oh.OK)
    dump("chain2_box_values.json",
         dict(source="oracle.hopf.value", workload="2-mass spring chain (n=4, m=1 box), x~N(0,I) seed 31",
              P=P, T=1.7, N=64, rule="left_riemann", tau=0.5, oracle_tol=1e-10),
         x=x, phi=r["phi"], p=r["p"])


def chain10_time_to_reach(P=4):
    # larger-state box-control system: chain of 10 masses (n = 20, m = 2)
    sysd = wl.spring_chain(masses=10, actuators=2, radius_target=1.0)
    x = wl.normal_points(11, P, 20, 0.7)
    r = oh.time_to_reach(sysd, x, 20.0, 48, oh.LEFT_RIEMANN, tau=0.5, tol_T=1e-7, tol_gap=1e-8)
    assert np.all(r["status"] == oh.OK)
    dump("chain10_time_to_reach.json",
         dict(source="oracle.hopf.time_to_reach", workload="10-mass spring chain (n=20, m=2 box), r=1, "
              "x~N(0,0.49 I) seed 11", P=P, t_max=20.0, N=48, rule="left_riemann", tau=0.5, oracle_tol_T=1e-7),
         x=x, T=r["T"], p=r["p"], status=r["status"])


def unscented_time_to_reach(P=3):
    # §VI.B: double integrator with 5 sigma points sharing one control (n = 10)
    w = wl.workload_unscented(P)
    r = oh.time_to_reach(w["system"], w["x"], w["t_max"], w["N"], w["rule"], tau=w["tau"], tol_T=1e-7,
                         tol_gap=1e-8)
    assert np.all(r["status"] == oh.OK)
    dump("unscented_time_to_reach.json",
         dict(source="oracle.hopf.time_to_reach", workload="unscented double integrator (n=10, m=1 box), "
              "mu~U[-2,2]^2 seed 12, std 0.0667, ell 0.01", P=P, t_max=w["t_max"], N=w["N"], rule="left_riemann",
              tau=w["tau"], oracle_tol_T=1e-7),
         T=r["T"], p=r["p"], status=r["status"])


def chain_values(P=32, stride=4, T=10.0):
    # the 100-mass spring chain at full size (n = 200, m = 10 box, N = 512):
    # every stride-th of the first P seeded points.  The oracle runs in
    # terminal-time variables (the same phi; pinned like the paper's form)
    # because the paper's variable needs ~20x more iterations at this size.
    w = wl.workload_chain(P)
    idx = np.arange(0, P, stride)
    r = oh.value(w["system"], w["x"][idx], T, w["N"], w["rule"], tau=0.1, tol=1e-7, max_iter=2000000,
                 variables="terminal")
    assert np.all(r["status"] == oh.OK)
    dump("chain200_values_T10.json",
         dict(source="oracle.hopf.value (variables=terminal)",
              workload="100-mass spring chain (n=200, m=10 box, r=0.5), x~N(0,I) seed 3, points idx of the first P",
              P=P, T=T, N=w["N"], rule="left_riemann", tau=0.1, oracle_tol=1e-7),
         idx=idx, phi=r["phi"], p=r["p"], gap=r["gap"])


def random128_values(P=8):
    # the largest size of the 64 random systems: n = 128, m = ceil(n/8) = 16
    sysd = wl.random_system(328, 128, 16)
    x = wl.normal_points(428, P, 128, 2.0)
    r = oh.value(sysd, x, 2.0, 256, oh.LEFT_RIEMANN, tau=0.15, tol=1e-8, max_iter=2000000, variables="terminal")
    assert np.all(r["status"] == oh.OK)
    dump("random128_values.json",
         dict(source="oracle.hopf.value (variables=terminal)",
              workload="random system seed 328 (n=128, m=16 ball), x~N(0,4I) seed 428", P=P, T=2.0, N=256,
              rule="left_riemann", tau=0.15, oracle_tol=1e-8),
         phi=r["phi"], p=r["p"], gap=r["gap"])


def chain200_fixed_values():
    # the fixed-step rule at the chain's full size: one table on [0, 40] with
    # dt = 40/2048 (the paper's step at T = 10, N = 512), horizons between
    # multiples of the step (a partial last node), terminal-time variables
    w = wl.workload_chain(8)
    rule = oh.FixedStep(40.0, 2048)
    rows = []
    for T, idx in ((3.3, [0, 1]), (17.77, [2, 3])):
        r = oh.value(w["system"], w["x"][idx], T, 2048, rule, tau=0.1, tol=1e-7, max_iter=2000000,
                     variables="terminal")
        assert np.all(r["status"] == oh.OK)
        rows += [(k, T, r["phi"][j], r["gap"][j]) for j, k in enumerate(idx)]
    dump("chain200_fixed_values.json",
         dict(source="oracle.hopf.value (FixedStep(40, 2048), variables=terminal)",
              workload="100-mass spring chain (n=200, m=10 box, r=0.5), x~N(0,I) seed 3, points idx",
              t_max=40.0, N=2048, rule="fixed_step", tau=0.1, oracle_tol=1e-7),
         idx=[r[0] for r in rows], T=[r[1] for r in rows], phi=[r[2] for r in rows], gap=[r[3] for r in rows])


def chain10_fixed_time_to_reach():
    # fixed-step rule (dt = 20/256) on the 10-mass chain (n = 20, m = 2 box),
    # three of 24 seeded points, terminal-time variables
    sysd = wl.spring_chain(masses=10, actuators=2, radius_target=1.0)
    x = wl.normal_points(11, 24, 20, 0.7)
    idx = [0, 7, 23]
    r = oh.time_to_reach(sysd, x[idx], 20.0, 256, oh.FixedStep(20.0, 256), tau=0.2, tol_T=1e-7, tol_gap=1e-8,
                         variables="terminal")
    assert np.all(r["status"] == oh.OK)
    dump("chain10_fixed_time_to_reach.json",
         dict(source="oracle.hopf.time_to_reach (FixedStep(20, 256), variables=terminal)",
              workload="10-mass spring chain (n=20, m=2 box), r=1, x~N(0,0.49 I) seed 11, 24 points, idx",
              P=24, t_max=20.0, N=256, rule="fixed_step", tau=0.2, oracle_tol_T=1e-7),
         idx=idx, T=r["T"], status=r["status"])


if __name__ == "__main__":
    which = sys.argv[1:] or ["random10", "di", "ttr", "box", "chain10", "unscented", "chain200", "random128"]
    if "chain200" in which:
        chain_values()
    if "chain10_fixed_ttr" in which:
        chain10_fixed_time_to_reach()
    if "chain200_fixed" in which:
        chain200_fixed_values()
    if "random128" in which:
        random128_values()
    if "unscented" in which:
        unscented_time_to_reach()
    if "chain10" in which:
        chain10_time_to_reach()
    if "box" in which:
        box_values()
    if "di" in which:
        di_values()
    if "ttr" in which:
        di_time_to_reach()
    if "random10" in which:
        random10_values()
