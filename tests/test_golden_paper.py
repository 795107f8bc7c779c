"""Values printed in the paper, checked against the oracle's readings.

Fixtures: tests/golden/paper_values.json (each entry cites its section or
table).  The liver mesh itself is not available, so these pin the unit
conventions and the error metric rather than whole runs."""
import json
import os

import numpy as np
import pytest

from oracle import Oracle, eq20_error
from synth.meshes import kuhn_tet_box
from synth.problem import Material, Perfusion, Problem

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_td_slopes_of_section_3_1_6():
    g = GOLD["td_properties_sec_3_1_6"]
    m = Material.from_two_points(g["T1"], g["T2"], tuple(g["rho"]), tuple(g["c"]), tuple(g["k"]))
    s = g["slopes_printed"]
    assert m.drho == pytest.approx(s["rho"], abs=1e-4)
    assert m.dk == pytest.approx(s["k"], abs=1e-7)
    assert m.dc == pytest.approx(s["c"], abs=1e-5)


def test_perfusion_and_metabolism_as_per_node_quantities():
    """The paper verifies perfusion as a film condition h = w_b c_b V / N and
    metabolism as a nodal flow Q_m V / N.  On a mesh whose lumped volumes are
    all equal, the oracle's beta_i and Q_i must reduce to exactly these."""
    gp = GOLD["perfusion_as_film_sec_3_1_3"]
    gm = GOLD["metabolic_as_nodal_flux_sec_3_1_4"]
    assert gp["w_b"] * gp["c_b"] * gp["V"] / gp["n_nodes"] == pytest.approx(gp["h_printed"], abs=5e-5)
    assert gm["Q_m"] * gm["V"] / gm["n_nodes"] == pytest.approx(gm["q_printed"], abs=5e-5)
    # a periodic-like check: interior nodes of a Kuhn grid all carry V/N-type equal shares
    mesh = kuhn_tet_box(4, 4, 4, 1e-3)
    p = Problem(4, mesh.xyz, mesh.conn, Material.constant(1060.0, 3700.0, 0.518),
                Perfusion(w_b=gp["w_b"], c_b=gp["c_b"], T_a=39.0, Q_m=gm["Q_m"]))
    orc = Oracle(p)
    g = mesh.grid_index
    inner = np.all((g > 0) & (g < 4), axis=1)
    np.testing.assert_allclose(orc.beta[inner], gp["w_b"] * gp["c_b"] * orc.V[inner], rtol=1e-15)
    np.testing.assert_allclose(orc.V[inner], 1e-9, rtol=1e-12)     # one voxel's volume per node
    np.testing.assert_allclose(orc.Q[inner], gm["Q_m"] * 1e-9, rtol=1e-12)


def test_eq20_matches_the_tables():
    """Eq. 20 equals RMS(D) / RMS(A); the printed E of Tables 1-5 agree with
    the printed RMS rows to their rounding."""
    rng = np.random.default_rng(0)
    for row in GOLD["eq20_tables_1_to_5"]["rows"]:
        n = 1000
        A = np.full(n, row["rms_A"])
        D = row["rms_D"] * np.sign(rng.standard_normal(n))
        E = eq20_error(A, A - D)
        assert E == pytest.approx(row["rms_D"] / row["rms_A"], rel=1e-12)
        # printed RMS(D) carries 2 significant digits for tables 1-4
        assert E == pytest.approx(row["E"], rel=0.07)


def test_table_6_ratios_are_quotients_of_the_printed_timings():
    g = GOLD["timings_sec_3_2_table_6"]
    r = g["ratios_printed"]
    assert g["A_threads"] / g["P_TD_openmp"] == pytest.approx(r["TD_vs_A_threads"], abs=0.01)
    assert g["A_serial"] / g["P_TD_openmp"] == pytest.approx(r["TD_vs_A_serial"], abs=0.01)
    assert g["A_threads"] / g["P_TI_openmp"] == pytest.approx(r["TI_vs_A_threads"], abs=0.01)
    assert g["A_serial"] / g["P_TI_openmp"] == pytest.approx(r["TI_vs_A_serial"], abs=0.01)
    assert g["P_TD_openmp"] / g["P_TI_openmp"] == pytest.approx(r["TI_vs_TD"], abs=0.01)
    assert g["P_TD_serial"] / g["P_TD_openmp"] == pytest.approx(r["TD_openmp_vs_serial"], abs=0.001)
