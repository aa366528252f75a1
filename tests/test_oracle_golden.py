"""The IP iteration counts printed in tab:IP (Sec. 8.1) against the oracle's barrier schedule."""
import json
import os

import pytest

from oracle import fe, ip
from paper_1606_06201_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


@pytest.mark.parametrize("tau", ["1e-8", "1e-10", "1e-12", "1e-14"])
def test_ip_iteration_count_matches_tab_ip(tau):
    cfg = W.cantilever_2d(8, 8, 0.5)
    prob = ip.Problem(fe.Grid(8, 8), fe.element_stiffness(2), cfg["fixed"], cfg["f"], cfg["V"], 1.0)
    c = GOLDEN["constants"]
    _, info = ip.ip_run(prob, sigma=c["sigma"], tau_nwt=c["tau_nwt"], tau_ip=float(tau),
                        frac=c["step_fraction"])
    assert info["ip"] == GOLDEN["ip_iterations_vs_tau_ip"][tau]
