"""The accuracy study of Sec. 3.3 on the GPU con2prim kernel: the paper's 25 x 25 (gamma, P)
grid, prim -> cons -> prim, relative error of the recovered velocity
(claims in tests/golden/con2prim_accuracy_envelope.json)."""
import json
import os

import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "con2prim_accuracy_envelope.json")


def test_gpu_accuracy_on_the_paper_grid(gpu_lib):
    from paper_2205_00095_gb300 import c2p_study
    claims = json.load(open(GOLDEN))["claims"]
    err, it, lor = c2p_study.accuracy("ideal", "analytic")
    assert err[lor < 3].max() < 100 * claims["ideal_analytic_gamma_below_3_max_rel_err_v"]
    assert err[lor == lor.max()].max() < 10 * claims["ideal_analytic_gamma_100_rel_err_v_order"]
    for eos, c2p in (("ideal", "iterative"), ("tm", "analytic"), ("tm", "iterative")):
        err, it, lor = c2p_study.accuracy(eos, c2p)
        assert err.max() < 4e-15, (eos, c2p, err.max())


def test_gpu_throughput_is_measured(gpu_lib):
    from paper_2205_00095_gb300 import c2p_study
    r = c2p_study.throughput("ideal", "iterative", 1 << 20, reps=3)
    assert r > 1e9
