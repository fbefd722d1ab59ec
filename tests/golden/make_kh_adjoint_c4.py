"""Writes kh_adjoint_c4.json: central differences of the FP64 oracle for the gradient check of the
adjoint on the 2D Kelvin-Helmholtz set-up at its full size.

Configuration: the Taub-Matthews double shear layer on [-0.5, 0.5] x [-1, 1] (periodic), 128 x 256
elements, p = 3, HLL, Brent con2prim, 200 SSPRK3 steps of dt = oracle.cfl_dt(spec, 0.2), no
physicality action (asserted).  Objective: the transverse kinetic energy at the final time,
J = sum over elements and nodes of (dx/2)(dy/2) w_node rho gamma^2 v_y^2.

Stored:
  * J at the amplitude A = 0.01;
  * dJ/dA by central differences with h = 1e-6 (absolute), and again with 2h;
  * the directional derivative of J along three seeded fields of initial v_x (rho and P held
    fixed), h = 1e-6 and 2h: d = v_x sin^2(2 pi x) exp(-2 y^2/0.01) (1 + r/2) with r from numpy's
    legacy RandomState(seed).standard_normal((E, Nn)) (a stream numpy keeps fixed) -- the
    direct sensitivity of J to v_x (2 rho gamma^4 v_x v_y^2) modulated node by node, so that J
    moves by far more than its rounding;
  * dJ/dv_x at single nodes of the initial state, the nodes with the largest direct sensitivity
    2 rho gamma^4 |v_x| v_y^2 w at t = 0, one per element.  A single node moves J by h 1e-9,
    which at h = 1e-6 is within a few units of J's last place (ulp(J)/(2h) ~ 4e-16 against a
    derivative ~1e-9), so these use h = 1e-4 and 2h and store the Richardson value
    (4 D(h) - D(2h))/3, whose error is O(h^4).
The difference between the h and 2h values bounds the error of the stored differences (their
truncation error grows as h^2, their rounding as 1/h); the script requires it below 1e-8
relative for dJ/dA and the directions.  For the nodes it is the h^2 term itself (about 7e-5 at
h = 1e-4), which the Richardson value removes, leaving O(h^4) and a rounding of about one unit
of J's last place over 2h (5e-9 of the derivative); the script requires it below 1e-3, so
that a check at 1e-6 relative measures the adjoint.

Only the oracle and the input generators are used.  Run from the repository root:
    python tests/golden/make_kh_adjoint_c4.py [--procs N]
It takes about 60 oracle runs of 200 steps (a few minutes each on one core).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "kh_adjoint_c4.json")
NX, NY, DEGREE, NSTEPS, CHECKPOINT, A0, H, H_NODE = 128, 256, 3, 200, 20, 0.01, 1e-6, 1e-4
N_NODES, SEEDS = 10, (20501, 20502, 20503)


def spec_c4():
    import workloads as wl
    return wl.kh2d(nx=NX, ny=NY, degree=DEGREE)


def objective(task):
    """J after NSTEPS oracle steps from W0(A) + eps * (perturbation of v_x)."""
    import oracle
    import workloads as wl
    kind, arg, eps = task
    spec = spec_c4()
    X = oracle.node_coords(spec)
    A = A0 + eps if kind == "A" else A0
    W = wl.kh2d_ic(spec, X, amplitude=A)
    if kind == "node":
        e, i = arg
        W[1, e, i] += eps
    elif kind == "dir":
        W[1] += eps * direction(arg, spec, X, A0)
    U = oracle.prim2cons(spec, W)
    U, st = oracle.step(spec, U, oracle.cfl_dt(spec, 0.2), NSTEPS)
    if st["enforced_cells"] or st["c2p_invalid_input"] or st["c2p_nonconverged"]:
        raise RuntimeError(f"oracle run left the smooth regime: {st}")
    Wf, _, _ = oracle.con2prim(spec, U)
    g2 = 1.0 / (1.0 - (Wf[1:4] ** 2).sum(0))
    w1 = oracle.basis(DEGREE + 1)["w"]
    w = np.multiply.outer(w1, w1).ravel()
    jac = 0.25 * (spec["hi"][0] - spec["lo"][0]) / NX * (spec["hi"][1] - spec["lo"][1]) / NY
    return float((w * jac * Wf[0] * g2 * Wf[2] ** 2).sum())


def direction(seed, spec, X, A):
    """v_x sin^2(2 pi x) exp(-2 y^2 / 0.01) (1 + r/2), r seeded standard normal per node."""
    import workloads as wl
    W = wl.kh2d_ic(spec, X, amplitude=A)
    shape = W.shape[1:]
    r = np.random.RandomState(seed).standard_normal(shape)
    return W[1] * np.sin(2.0 * np.pi * X[0]) ** 2 * np.exp(-2.0 * X[1] ** 2 / 0.01) * (1.0 + 0.5 * r)


def pick_nodes():
    """One node per element, largest 2 rho gamma^4 |v_x| v_y^2 w at t = 0."""
    import oracle
    import workloads as wl
    spec = spec_c4()
    X = oracle.node_coords(spec)
    W = wl.kh2d_ic(spec, X, amplitude=A0)
    g2 = 1.0 / (1.0 - (W[1:4] ** 2).sum(0))
    w1 = oracle.basis(DEGREE + 1)["w"]
    w = np.multiply.outer(w1, w1).ravel()
    score = 2.0 * W[0] * g2 * g2 * np.abs(W[1]) * W[2] ** 2 * w
    best_node = score.argmax(axis=1)
    best = score.max(axis=1)
    elems = np.argsort(-best)[: N_NODES]
    return [(int(e), int(best_node[e])) for e in elems]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    import oracle
    oracle.build()
    nodes = pick_nodes()
    tasks = [("A", None, 0.0)]
    for h in (H, 2 * H):
        tasks += [("A", None, h), ("A", None, -h)]
        for s in SEEDS:
            tasks += [("dir", s, h), ("dir", s, -h)]
    for h in (H_NODE, 2 * H_NODE):
        for n in nodes:
            tasks += [("node", n, h), ("node", n, -h)]
    t0 = time.time()
    with mp.get_context("spawn").Pool(args.procs) as pool:
        vals = pool.map(objective, tasks, chunksize=1)
    got = dict(zip([(k, tuple(a) if isinstance(a, (list, tuple)) else a, e) for k, a, e in tasks], vals))

    def fd(kind, arg, h):
        key = tuple(arg) if isinstance(arg, (list, tuple)) else arg
        return (got[(kind, key, h)] - got[(kind, key, -h)]) / (2 * h)

    def entry(kind, arg, h):
        g1, g2 = fd(kind, arg, h), fd(kind, arg, 2 * h)
        return {"h": h, "fd_h": g1, "fd_2h": g2, "rel_diff_h_2h": abs(g1 - g2) / abs(g1),
                "richardson": (4.0 * g1 - g2) / 3.0}

    node_entries = [{"elem": e, "node": i, **entry("node", (e, i), H_NODE)} for e, i in nodes]
    dir_entries = [{"seed": s, "field": "v_x sin^2(2 pi x) exp(-2 y^2/0.01) (1 + r/2), r = numpy "
                    "RandomState(seed).standard_normal((E, Nn))", **entry("dir", s, H)} for s in SEEDS]
    dA = entry("A", None, H)
    # keep the stored differences whose h and 2h values agree (1e-8 relative at h = 1e-6; for
    # the Richardson-corrected nodes, whose h^2 term is removed, 1e-3)
    kept = [n for n in node_entries if n["rel_diff_h_2h"] < 1e-3]
    bad = [x for x in [dA] + dir_entries if not x["rel_diff_h_2h"] < 1e-8]

    spec = spec_c4()
    out = {
        "source": "central differences of the FP64 oracle (oracle/), written by make_kh_adjoint_c4.py",
        "configuration": {"workload": "kh_2d", "n_elem": [NX, NY], "degree": DEGREE, "eos": "tm",
                          "c2p": "default (Brent)", "flux": spec["flux"], "rk_stages": 3,
                          "nsteps": NSTEPS, "checkpoint_every": CHECKPOINT,
                          "dt": oracle.cfl_dt(spec, 0.2), "cfl": 0.2, "amplitude": A0, "h": H,
                          "h_node": H_NODE},
        "objective": "J = sum (dx/2)(dy/2) w_node rho gamma^2 v_y^2 at t = nsteps dt",
        "J": got[("A", None, 0.0)],
        "dJ_dA": dA,
        "dJ_dvx_nodes": kept,
        "dJ_dvx_nodes_dropped": [n for n in node_entries if n not in kept],
        "dJ_dvx_directions": dir_entries,
        "oracle_runs": len(tasks), "seconds": round(time.time() - t0, 1),
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in ("J", "dJ_dA", "seconds")}))
    if bad or len(kept) < 8:
        raise SystemExit(f"differences not converged: {bad}, {len(kept)} nodes kept of {len(nodes)}")


if __name__ == "__main__":
    main()
