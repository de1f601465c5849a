"""Host post-processing of the force record: Strouhal number and drag
coefficient against closed forms."""
import numpy as np
import pytest

from paper_2606_16765_gb300 import wake


@pytest.mark.parametrize("f", [0.0031, 0.0123, 0.041])
def test_dominant_frequency_of_a_noisy_sinusoid(f):
    t = np.arange(12000)
    x = 2.0 + np.sin(2 * np.pi * f * t + 0.7) + 0.3 * np.random.default_rng(1).normal(size=t.size)
    # bin width 1/12000; the parabolic refinement lands well inside one bin
    assert abs(wake.dominant_frequency(x) - f) < 0.15 / len(t)


def test_strouhal_scales_with_sampling_interval_and_geometry():
    t = np.arange(4000)
    lift = np.cos(2 * np.pi * 0.002 * t * 5)          # sampled every 5 steps: 0.002 cycles per step
    assert abs(wake.strouhal(lift, 16.0, 0.05, every=5) - 0.002 * 16 / 0.05) < 2e-3


def test_drag_coefficient_closed_form():
    fx = np.full(100, 0.8)
    # C_d = 2 F / (rho U^2 D H)
    assert wake.drag_coefficient(fx, 16.0, 128.0, 0.05) == pytest.approx(2 * 0.8 / (0.0025 * 16 * 128))


def test_short_signal_is_rejected():
    with pytest.raises(ValueError):
        wake.dominant_frequency(np.ones(4))


def test_band_limited_peak_ignores_a_stronger_mode_outside_the_band():
    t = np.arange(10000)
    x = 5 * np.sin(2 * np.pi * 0.00225 * t) + np.sin(2 * np.pi * 0.0006 * t)
    assert wake.strouhal(x, 16.0, 0.05) == pytest.approx(0.00225 * 16 / 0.05, abs=0.01)
    assert wake.strouhal(x, 16.0, 0.05, st_band=(0.1, 0.5)) == pytest.approx(0.0006 * 16 / 0.05, abs=0.01)


def test_recirculation_length_of_a_synthetic_wake():
    x = np.arange(200.0)
    rear, L = 40.0, 23.5
    u = np.where(x <= rear, 0.0, 0.05 * np.tanh((x - rear - L) / 4.0))   # backflow until rear + L
    assert wake.recirculation_length(u, rear) == pytest.approx(L, abs=2e-3)
    assert wake.recirculation_length(np.abs(u) + 0.01, rear) == 0.0     # no backflow
