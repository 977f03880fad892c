"""The constants the paper states (tests/golden/paper_constants.txt, each line citing where)
against the defaults of the library, its binding and the oracle, so that a default run is the
paper's configuration: the clamp anneal (Algorithm 3), Adam's moments (Section 3), the
schedule's windows and tolerances (Sections 3 and 4) and the viewgraph's tau and fraction
(Section 3, Eq. 2; Section 4)."""
import inspect
from pathlib import Path

import pytest

import oracle


def paper_constants():
    out = {}
    for ln in (Path(__file__).parent / "golden" / "paper_constants.txt").read_text().splitlines():
        ln = ln.split("#", 1)[0].strip()
        if ln:
            k, v = (x.strip() for x in ln.split("="))
            out[k] = float(v)
    return out


C = paper_constants()


def test_fixture_complete():
    assert set(C) == {"lambda0", "lambda1", "lambda_steps", "beta1", "beta2", "sched_w1", "sched_w2",
                      "sched_eps1", "sched_eps2", "viewgraph_tau", "viewgraph_min_frac"}


def test_library_defaults_are_the_papers():
    epo = pytest.importorskip("paper_2607_00579_gb300")
    o = epo.default_options()
    for k in ("lambda0", "lambda1", "lambda_steps", "beta1", "beta2", "sched_w1", "sched_w2", "sched_eps1",
              "sched_eps2"):
        assert getattr(o, k) == C[k], k
    sig = inspect.signature(epo.build_viewgraph).parameters
    assert sig["tau"].default == C["viewgraph_tau"]
    assert sig["min_frac"].default == C["viewgraph_min_frac"]


def test_oracle_defaults_are_the_papers():
    assert oracle.lambda_at(0) == C["lambda0"]
    assert oracle.lambda_at(int(C["lambda_steps"])) == C["lambda1"]
    assert oracle.lambda_at(int(C["lambda_steps"]) // 2) == pytest.approx((C["lambda0"] + C["lambda1"]) / 2)
    assert inspect.signature(oracle.viewgraph).parameters["tau"].default == C["viewgraph_tau"]
    assert inspect.signature(oracle.viewgraph_pairs).parameters["min_frac"].default == C["viewgraph_min_frac"]
    opt = inspect.signature(oracle.OracleScene.optimize).parameters
    assert opt["beta1"].default == C["beta1"] and opt["beta2"].default == C["beta2"]
    assert opt["lambda0"].default == C["lambda0"] and opt["lambda_steps"].default == C["lambda_steps"]
