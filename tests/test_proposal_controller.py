"""Host logic of the learned-proposal training loop: the fallback controller and the
proposal parameter layout (no GPU needed)."""
import numpy as np

from paper_2206_14735_gb300.proposal import PROP_PAD, FallbackController, init_proposal_params
from paper_2206_14735_gb300._lib import GS_PROP_PARAMS


def test_controller_starts_on_the_plain_sampler_and_follows_the_5_percent_rule():
    c = FallbackController()
    assert not c.use_proposal
    assert c.update(1.00, 1.00)            # equal: proposal
    assert c.update(1.05, 1.00)            # at the bound: proposal
    assert not c.update(1.0501, 1.00)      # above: fall back
    assert c.update(0.5, 1.00)             # better again: proposal
    assert not c.update(float("nan"), 1.0)  # a broken evaluation never selects the proposal
    assert [h[2] for h in c.history] == [True, True, False, True, False]


def test_controller_tolerance_is_configurable():
    c = FallbackController(tolerance=1.2)
    assert c.update(1.19, 1.0)
    assert not c.update(1.21, 1.0)


def test_initial_parameters_layout():
    q = init_proposal_params(seed=1)
    assert q.shape == (PROP_PAD,) and PROP_PAD % 4 == 0 and PROP_PAD >= GS_PROP_PARAMS
    assert np.all(q[GS_PROP_PARAMS:] == 0)           # padding stays zero
    assert np.all(q[352:384] == 0) and np.all(q[1408:1440] == 0) and q[1472] == 0  # biases
    assert np.abs(q[:352]).max() > 0 and np.abs(q[384:1408]).max() > 0 and np.abs(q[1440:1472]).max() > 0
