"""The small experiment of Sec. III (Figs. `Gap_All`, `Gap_APG`, `Distance_All`) on the GPU.

Recipe ``xqx`` (N = 100, n = 5, f0 = 1/2 x^T Q x): P-APG (momentum) and the paper's comparator,
dual gradient ascent (the same iteration without momentum).  The paper's two traces -- the
duality gap theta^T C eta and the infeasibility ||(A_1 y + A_2 xi)_-||_2 (both reported
normalized by the N^2 - N pairs) -- are compared with the FP64 oracle along the iterations, and
the qualitative claim of the figures is checked: P-APG's gap and infeasibility fall below dual
gradient ascent's.  The paper splits the data into K = 2 blocks; here every pair is a block
(K = N), so the curves share the figures' shape, not their values.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1407_7220_gb300 import datagen

pytestmark = pytest.mark.gpu

CHECKS = (5, 20, 100, 400, 1500)


@pytest.fixture(scope="module")
def crg():
    import paper_1407_7220_gb300 as m
    return m


def _traces(crg, momentum):
    X, yb, _ = datagen.make("xqx")
    g = crg.Solver(X, yb, gamma=0.1, momentum=momentum, stochastic_round=0, restart=0)
    o = O.Solver(X, yb, gamma=0.1, momentum=bool(momentum), restart=False)
    out, done = [], 0
    for k in CHECKS:
        g.iterate(k - done)
        o.iterate(k - done)
        done = k
        kk = g.kkt_residual()
        out.append((kk["infeas_norm"], kk["gap_norm"], o.metrics["infeas"], o.metrics["gap"]))
    return np.array(out)


def test_traces_match_oracle_and_papg_leads_dual_ascent(crg):
    papg = _traces(crg, 1)
    ascent = _traces(crg, 0)
    for tr in (papg, ascent):
        # FP32 round-to-nearest against FP64 over up to 1,500 iterations; the gap crosses zero,
        # so it is compared on the scale of its largest value
        np.testing.assert_allclose(tr[:, 0], tr[:, 2], rtol=1e-2, atol=1e-12)
        np.testing.assert_allclose(tr[:, 1], tr[:, 3], rtol=1e-2, atol=1e-3 * np.abs(tr[:, 3]).max())
    # Figs. Gap_All / Distance_All: after the first iterations P-APG is below dual ascent on both
    assert np.all(papg[-3:, 0] < ascent[-3:, 0])
    assert np.all(np.abs(papg[-3:, 1]) < np.abs(ascent[-3:, 1]))
    # and both decrease overall
    for tr in (papg, ascent):
        assert tr[-1, 0] < tr[0, 0] and abs(tr[-1, 1]) < abs(tr[0, 1])
