"""Host logic of the online lambda tuner (paper_2603_08582_gb300.tuning):
the step rule alone, no GPU."""
import math

import pytest

from paper_2603_08582_gb300.tuning import lambda_update


def test_step_goes_against_the_gradient_in_log_space():
    # the loss grows with lambda: rho shrinks, by exp(-eta g) with g the
    # relative sensitivity lambda dL/dlambda / L
    assert lambda_update(0.1, 2.0, 0.05, 1.0, 0.25) == pytest.approx(0.1 * math.exp(-0.025))
    assert lambda_update(0.1, 2.0, -0.05, 1.0, 0.25) == pytest.approx(0.1 * math.exp(0.025))


def test_step_is_clipped_and_guarded():
    assert lambda_update(0.1, 2.0, 1e9, 1.0, 0.25) == pytest.approx(0.1 * math.exp(-0.25))
    assert lambda_update(0.1, 2.0, -1e9, 1.0, 0.25) == pytest.approx(0.1 * math.exp(0.25))
    assert lambda_update(0.1, 2.0, 1.0, 0.0, 0.25) == 0.1        # zero loss
    assert lambda_update(0.1, 0.0, 1.0, 1.0, 0.25) == 0.1        # lambda 0
    assert lambda_update(0.1, 2.0, float("nan"), 1.0, 0.25) == 0.1
