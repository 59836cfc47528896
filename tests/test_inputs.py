"""Input generators checked against independent computations, on CPU.

The applied pressure equivalent to a Gaussian bump is built for the solver
from the paper's radial (Hankel) integral (Sec. 6); the oracle builds the same
pressure from the transform relation of Sec. 4.1 by a 2-D FFT.  The two
routes share nothing but the definition."""
import math

import numpy as np
import pytest

from oracle import linear_fft as LF
from paper_1709_08803_gb300 import workloads as W


@pytest.mark.parametrize("eps,delta,F", [(0.285, 0.5, 0.6),            # the Sec. 6 comparison
                                         (0.1, 1.0 / math.sqrt(2.0), 0.7),
                                         (1.0, 3.0, 3.0)])               # a Sec. 5.2 bump
def test_equivalent_pressure_hankel_matches_fft(eps, delta, F):
    mesh = W.Mesh(N=41, M=31, x1=-4.0, y1=-3.0, dx=0.2, dy=0.2, half=0)  # nodes on the FFT grid
    p = W.gaussian_equivalent_pressure(mesh, eps, delta, F)
    ref = LF.equivalent_pressure(lambda X, Y: eps * np.exp(-(X * X + Y * Y) / (2 * delta * delta)), F,
                                 mesh.x(), mesh.y()).ravel()
    assert np.abs(p - ref).max() <= 5e-5 * np.abs(ref).max()


def test_equivalent_pressure_scales_with_eps_over_F_squared():
    mesh = W.mesh_box(21, 11, 0.3, 0.3)
    a = W.gaussian_equivalent_pressure(mesh, 0.2, 0.5, 0.6)
    b = W.gaussian_equivalent_pressure(mesh, 0.4, 0.5, 1.2)
    assert np.allclose(b, 0.5 * a, rtol=1e-12, atol=0.0)
