"""Why binary32 runs carry the populations as compensated deviations (no GPU).

A population relaxes by dt/tau21 ~ 2e-8 of itself per step at the lasing
workload's time step, below half the binary32 unit roundoff (2^-24 ~ 6e-8):
a plain binary32 running sum then never moves, while a Kahan-compensated sum
(the form the step kernels use for dN, with one compensation word per
population) follows the exact decay to the roundoff of its final value.
Emulated here with numpy binary32 arithmetic over 2e5 steps."""
import numpy as np


def test_compensated_binary32_sum_follows_a_decay_below_the_roundoff():
    steps = 200_000
    rate = np.float32(-2e-8)
    x0 = np.float32(1.0) + np.arange(64, dtype=np.float32) * np.float32(0.01)
    plain = x0.copy()
    s, comp = x0.copy(), np.zeros_like(x0)
    for _ in range(steps):
        plain = plain + plain * rate
        y = s * rate - comp
        t = s + y
        comp = (t - s) - y
        s = t
    assert s.dtype == np.float32 and plain.dtype == np.float32
    exact = x0.astype(np.float64) * (1.0 - 2e-8) ** steps
    assert np.array_equal(plain, x0)                                  # stagnates
    assert np.max(np.abs(plain - exact) / exact) > 3e-3               # ... 2e5 x 2e-8 off
    assert np.max(np.abs(s - exact) / exact) < 2.0 ** -24 * 1.01      # within half an ulp
    assert np.max(np.abs((s.astype(np.float64) - comp) - exact) / exact) < 1e-9
