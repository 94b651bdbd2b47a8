"""The mapping figures (documentation): they are generated from the oracle's
scalar maps, and the plotted images respect the schemes' bounds: after
iteration k every eigenvalue outside the gap maps into [0, beta_k] (empty
states) or [betabar_k, 1] (occupied ones)."""
import os

import numpy as np

from oracle import mapping_figures as M


def _check(lam, curves):
    occ = lam <= M.HOMO
    unocc = lam >= M.LUMO
    for (k, scaled), (x, b, bb) in curves.items():
        assert np.all(x[unocc] <= b + 1e-12) and np.all(x[unocc] >= -1e-12)
        assert np.all(x[occ] >= bb - 1e-12) and np.all(x[occ] <= 1 + 1e-12)
    # scaling converges faster: the last plotted iteration's bound is tighter
    kmax = max(k for k, _ in curves)
    assert curves[(kmax, True)][1] < curves[(kmax, False)][1]


def test_mapping_curves_respect_the_bounds():
    lam, c = M.fixed_mu_curves((1, 3, 5))
    _check(lam, c)
    lam, c = M.tc_curves((1, 5, 9))
    _check(lam, c)


def test_mapping_figures_written(tmp_path):
    paths = M.main(str(tmp_path))
    for p in paths:
        svg = open(p).read()
        assert svg.startswith("<svg") and svg.count("<polyline") == 6
        assert os.path.getsize(p) < 60_000
