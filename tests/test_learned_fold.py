"""Host-side bookkeeping of the learned warm start's training: folding the
input and output standardisation into the first and last layers gives the same
function on raw inputs (checked with the oracle's FP64 forward)."""
import numpy as np

from paper_2011_00459_gb300 import learned
from paper_2011_00459_gb300 import tds


def test_folded_network_equals_standardised_network(orc):
    g = np.random.Generator(np.random.PCG64(3))
    X = g.normal([1.0, 0.01, 5.0, 0.0, 2.0, 0.0, 6.0, 5.0, 0.3, 1.0],
                 [2.0, 0.005, 30.0, 1e-9, 4.0, 0.0, 2.0, 2.0, 0.5, 0.8], (500, 10))
    T = g.normal([20.0, -5.0, 0.0], [60.0, 20.0, 15.0], (500, 3))
    mx, sx, mt, st = learned.standardise(X, T)
    assert sx[5] == 1.0 and sx[3] == 1.0  # constant (or nearly) columns keep spread 1
    p = tds.init_params(4)
    want = mt + st * orc.mlp_forward((X - mx) / sx, tds.unflatten_params(p))
    got = orc.mlp_forward(X, tds.unflatten_params(learned.fold(p, mx, sx, mt, st, tds)))
    # the folded parameters are stored in FP32: agreement to FP32 rounding
    assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max()
    # a plausible slip (output scale applied to the bias only) is caught
    bad = tds.unflatten_params(learned.fold(p, mx, sx, mt, st, tds))
    bad["W3"] = bad["W3"] / st[:, None]
    assert np.abs(orc.mlp_forward(X, bad) - want).max() > 1e-2 * np.abs(want).max()
