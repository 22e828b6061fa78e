"""The pipe-rate probes behind the roofline denominators (sim_probe_peak)."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_every_probe_kind_measures_a_positive_rate_and_unknown_kinds_fail():
    from paper_2410_19075_gb300.sim import probe_peak
    from paper_2410_19075_gb300._lib import SimError
    rates = [probe_peak(k) for k in range(5)]
    assert all(math.isfinite(r) and r > 0 for r in rates), rates
    # an unsigned 64-bit multiply-high is never slower than the signed one, which
    # needs the unsigned product and two corrections
    assert rates[1] >= 0.9 * rates[4]
    with pytest.raises(SimError):
        probe_peak(5)
