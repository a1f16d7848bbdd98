"""The float64 oracle against its pins (no GPU).

Each pin compares the oracle with something other than itself: brute-force
sums, numpy.fft, exact closed forms, finite differences, invariants the paper
states (mean conservation to ~1e-12, Sec. III.B and III.C).
"""

import pytest

from tests import oracle_pins as pins


@pytest.mark.parametrize("name", sorted(pins.PINS))
def test_pin(name):
    fn, bound = pins.PINS[name]
    err = fn()
    assert err <= bound, f"{name}: {err:.3e} > {bound:.1e}"


def test_paper_mean_conservation_bound():
    """The paper reports the normalised mean of u staying at 1 within ~1e-12
    for diffusion and for the source-free wave (tests/golden/paper_facts.txt)."""
    from tests.golden import load_facts

    facts = load_facts()
    assert pins.pin_diffusion_invariants() <= facts["diffusion_mean_conservation_rel"]
    assert pins.pin_wave_invariants() <= facts["wave_mean_conservation_rel"]


def test_hand_dft4():
    """DFT of (1, 2, 3, 4) by hand with omega = e^{-2 pi i/4} = -i."""
    import numpy as np
    import oracle

    got = oracle.dft1(np.array([1.0, 2.0, 3.0, 4.0]), sign=-1)
    want = np.array([10, -2 + 2j, -2, -2 - 2j])
    assert np.max(np.abs(got - want)) < 1e-14
