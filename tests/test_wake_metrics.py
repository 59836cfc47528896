"""The wake-angle and steepness post-processing of the supercritical runs
(Sec. 5.2, Fig. 6), on CPU, against a synthetic V-shaped ridge whose angle
and maximum outer slope are known in closed form."""
import math

import numpy as np
import pytest

from paper_1709_08803_gb300 import workloads as W
from paper_1709_08803_gb300.paper_scale import wake_metrics


def _v_ridge(theta_deg, A, k, x0=2.0):
    """zeta = A sech^2(k (|y| - t (x - x0))), t = tan(theta): crests on the
    lines |y| = t (x - x0).  With s = k (|y| - t (x - x0)), |grad s| =
    k sqrt(1 + t^2) and max |d sech^2 / ds| = 4 / (3 sqrt 3) (at tanh^2 s = 1/3),
    so the largest slope outside the ridge is A k sqrt(1 + t^2) 4 / (3 sqrt 3)."""
    mesh, _, _ = W.config_supercritical_281(0.1)
    x, y = mesh.x(), mesh.y()
    X, Y = np.meshgrid(x, y)
    t = math.tan(math.radians(theta_deg))
    s = k * (np.abs(Y) - t * (X - x0))
    sech2 = 1.0 / np.cosh(s) ** 2
    dz_ds = -2.0 * A * sech2 * np.tanh(s)
    zx = dz_ds * (-k * t)
    zy = dz_ds * k * np.sign(Y)
    steep = A * k * math.sqrt(1.0 + t * t) * 4.0 / (3.0 * math.sqrt(3.0))
    return x, y, A * sech2, zx, zy, steep


@pytest.mark.parametrize("theta,A,k", [(19.47, 0.1, 1.0), (24.0, 0.5, 0.7), (14.5, 0.05, 1.3)])
def test_angle_and_steepness_of_a_synthetic_v(theta, A, k):
    x, y, z, zx, zy, steep = _v_ridge(theta, A, k)
    m = wake_metrics(x, y, z, zx, zy)
    assert m["wake_angle_deg"] == pytest.approx(theta, abs=0.05)
    for side in m["wake_angle_sides_deg"]:
        assert side == pytest.approx(theta, abs=0.05)
    assert m["ridge_fit_rms"] < 0.01
    # sampled on the mesh (dy = 0.257), the largest outer slope is within a few per cent
    assert steep * 0.97 <= m["steepness"] <= steep * 1.0000001


def test_steepness_ignores_the_inside_of_the_v():
    """A steeper feature between the two arms of the V does not count."""
    x, y, z, zx, zy, steep = _v_ridge(20.0, 0.1, 1.0)
    inner = np.abs(y)[:, None] < 1.0
    zy2 = np.where(inner, 50.0, zy)
    assert wake_metrics(x, y, z, zx, zy2)["steepness"] == pytest.approx(wake_metrics(x, y, z, zx, zy)["steepness"])


def test_needs_columns_in_range():
    x, y, z, zx, zy, _ = _v_ridge(20.0, 0.1, 1.0)
    with pytest.raises(ValueError):
        wake_metrics(x, y, z, zx, zy, x_from=100.0, x_to=200.0)


def test_wave_heights_of_a_synthetic_subcritical_wake():
    """Transverse waves A cos(k x) confined near the centreline plus one
    divergent crest of height D at 19 degrees: the heights come back."""
    from paper_1709_08803_gb300.paper_scale import wave_heights
    mesh, _, _ = W.config_subcritical_281(0.1)
    x, y = mesh.x(), mesh.y()
    X, Y = np.meshgrid(x, y)
    A, D, k = 0.03, 0.08, 2.78
    xc, yc = 10.0, 10.0 * math.tan(math.radians(19.0))
    z = A * np.cos(k * X) * np.exp(-Y * Y) * (X > 0) \
        + D * np.exp(-((X - xc) ** 2 + (np.abs(Y) - yc) ** 2) / 0.1)
    zx, zy = np.gradient(z, x, axis=1), np.gradient(z, y, axis=0)
    h = wave_heights(x, y, z, zx, zy)
    assert h["transverse_height"] == pytest.approx(A, rel=2e-3)
    assert h["divergent_crest"] == pytest.approx(D, rel=2e-2)
    assert h["downstream_steepness"] >= D * math.sqrt(2.0 / 0.1) * math.exp(-0.5) * 0.9
