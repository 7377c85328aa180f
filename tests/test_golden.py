"""Pins against values the paper prints (tests/golden/paper_setup.json, Results).

- Eq. 11 in the oracle, with the paper's three interfacial tensions (droplet = phase 1,
  lubricant = phase 2, ambient = phase 3): the lubricant's coefficient is minus the
  spreading coefficient of oil on water in air, which the paper states is positive (the
  droplet is cloaked), so Upsilon_2 < 0 by exactly that amount. The pairwise tensions are
  recovered as gamma_ij = (Upsilon_i + Upsilon_j) / 2, which fails for any swapped index.
- The micropillar array of the synthetic workloads has the paper's solid fraction
  phi = w_p^2 / (w_p + s_p)^2 = 0.25 (pillar width equal to the spacing).
"""
import json
import os

import numpy as np
import pytest

from paper_2608_12868_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_setup.json")


@pytest.fixture(scope="module")
def paper():
    with open(GOLDEN) as f:
        return json.load(f)


def test_upsilon_of_the_papers_tensions(oracle_mod, paper):
    g_wa, g_ow, g_oa = (paper["gamma_wa_mN_per_m"], paper["gamma_ow_mN_per_m"],
                        paper["gamma_oa_mN_per_m"])
    g12, g13, g23 = g_ow, g_wa, g_oa          # droplet-lubricant, droplet-ambient, lub.-ambient
    Y, YT = oracle_mod.upsilon(g12, g13, g23)
    spreading = g_wa - g_ow - g_oa
    assert spreading > 0                      # the paper's cloaking condition
    assert Y[1] == pytest.approx(-spreading, abs=1e-12)
    assert Y[1] < 0 < Y[0] and Y[2] > 0
    for (i, j), g in {(0, 1): g12, (0, 2): g13, (1, 2): g23}.items():
        assert 0.5 * (Y[i] + Y[j]) == pytest.approx(g, abs=1e-12)
    # equal tensions: every coefficient, and their harmonic combination, equal the tension
    Ye, YTe = oracle_mod.upsilon(7.0, 7.0, 7.0)
    assert np.allclose(Ye, 7.0) and YTe == pytest.approx(7.0)


def test_pillar_solid_fraction(paper):
    w_p, s_p = paper["pillar_width_um"], paper["pillar_spacing_um"]
    assert w_p ** 2 / (w_p + s_p) ** 2 == pytest.approx(paper["solid_fraction"], abs=1e-12)
    w = W.droplet_3d_128x64x64()
    nz, ny, nx = w.shape
    z = 2                                      # a plane through the pillars, above the floor
    frac = float((w.solid[z] == 1).sum()) / (nx * ny)
    assert frac == pytest.approx(paper["solid_fraction"], abs=1e-12)
