"""The oracle against the constants the paper prints (tests/golden, each
entry citing its passage)."""
import json
import os
from fractions import Fraction

import numpy as np

from oracle import oracle as O
from paper_1608_06915_gb300 import inputs as I

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def _q(v):
    return float(Fraction(v[0], v[1]))


def test_rest_equilibrium_is_the_product_of_the_printed_weights():
    w1 = GOLDEN["lattice_weights_1d"]
    w = {-1: _q(w1["c=-1"]), 0: _q(w1["c=0"]), 1: _q(w1["c=+1"])}
    want = np.array([w[i % 3 - 1] * w[(i // 3) % 3 - 1] * w[i // 9 - 1] for i in range(27)])
    assert np.max(np.abs(O.feq(1.0, np.zeros(3)) - want)) < 1e-16


def test_interpolation_weights_are_the_printed_ones():
    want = np.array([_q(v) for v in GOLDEN["interpolation_weights"]["weights"]])
    assert np.max(np.abs(O.lagrange_weights() - want)) < 1e-16


def test_gamma_two_is_lbgk_as_printed():
    g = _q(GOLDEN["lbgk_stabiliser"]["gamma"])
    rng = np.random.default_rng(5)
    f = O.feq(1.02, np.array([0.03, -0.01, 0.02])) * (1 + 0.01 * rng.uniform(-1, 1, 27))
    beta = 0.9
    fo, _ = O.collide(f, beta, gamma=g)
    rho = f.sum()
    fe = O.feq(rho, (np.array([[(i % 3) - 1, (i // 3) % 3 - 1, i // 9 - 1] for i in range(27)]).T @ f) / rho)
    assert np.max(np.abs(fo - (f + 2 * beta * (fe - f)))) < 1e-15  # LBGK with omega = 2 beta


def test_level_relaxation_follows_the_printed_viscosity_and_ratio():
    cs2 = _q(GOLDEN["viscosity"]["cs2"])
    r = _q(GOLDEN["refinement_ratio"]["r"])
    nu0 = 0.01
    o = O.Oracle(I.tgv_case(n=16, box=(4, 12), nu=nu0))
    for info in o.patches:
        nu = cs2 * (1.0 / (2.0 * info["beta"]) - 0.5)
        # acoustic scaling: in level units the viscosity grows by r per level
        assert abs(nu - nu0 * r ** info["level"]) < 1e-15
