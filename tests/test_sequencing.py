"""Mesh sequencing (host side): the unknown vector carried from a coarse mesh
to a finer one.  Checked against what interpolation of the Sec. 3.1 unknowns
must preserve: the uniform stream exactly, the data at coincident nodes
exactly, and a smooth field to the fourth order of bicubic splines."""
import numpy as np
import pytest

from paper_1709_08803_gb300 import workloads as W
from paper_1709_08803_gb300.sequencing import interpolate_u


def _mesh(h, N0=19, M0=7, half=0):
    # the same rectangle [-4, 5] x [-3, 3] (or [0, 3] for a half mesh) at spacing h and h/2
    r = int(round(0.5 / h))
    return W.Mesh(N=(N0 - 1) * r + 1, M=(M0 - 1) * r + 1, x1=-4.0, y1=0.0 if half else -3.0,
                  dx=h, dy=h if half else 2 * h, half=half)


def _analytic_u(mesh):
    """u of zeta = 0.05 sin(0.7 x) cos(0.4 y), phi = x + 0.03 cos(0.5 x) sin(0.3 y + 0.2),
    psi = x - 0.02 sin(0.9 x + 0.1) cos(0.6 y): upstream values and exact x-derivatives."""
    x, y = mesh.x(), mesh.y()
    X, Y = np.meshgrid(x, y)
    qx = [0.035 * np.cos(0.7 * X) * np.cos(0.4 * Y),
          1.0 - 0.015 * np.sin(0.5 * X) * np.sin(0.3 * Y + 0.2),
          1.0 - 0.018 * np.cos(0.9 * X + 0.1) * np.cos(0.6 * Y)]
    x1 = mesh.x1
    q1 = [0.05 * np.sin(0.7 * x1) * np.cos(0.4 * y),
          x1 + 0.03 * np.cos(0.5 * x1) * np.sin(0.3 * y + 0.2),
          x1 - 0.02 * np.sin(0.9 * x1 + 0.1) * np.cos(0.6 * y)]
    u = np.empty((3, mesh.M, mesh.N + 1))
    for f in range(3):
        u[f, :, 0] = q1[f]
        u[f, :, 1:] = qx[f]
    return u.reshape(-1)


@pytest.mark.parametrize("half", [0, 1])
def test_uniform_stream_is_kept_exactly(half):
    mc, mf = _mesh(0.5, half=half), _mesh(0.25, half=half)
    u = interpolate_u(mc, W.flat_guess(mc), mf)
    assert np.abs(u - W.flat_guess(mf)).max() <= 1e-12


def test_single_slice_meshes():
    mc = W.Mesh(N=19, M=1, x1=-4.0, y1=0.0, dx=0.5, dy=0.5, half=0)
    mf = W.Mesh(N=37, M=1, x1=-4.0, y1=0.0, dx=0.25, dy=0.25, half=0)
    assert np.abs(interpolate_u(mc, W.flat_guess(mc), mf) - W.flat_guess(mf)).max() <= 1e-12
    u = interpolate_u(mc, _analytic_u(mc), mf)
    assert np.abs(u - _analytic_u(mf)).max() <= 1e-3


def test_coincident_nodes_are_exact():
    """Fine to coarse, the coarse nodes being every other fine node: the
    splines interpolate, so every coarse unknown is the fine one."""
    mf, mc = _mesh(0.25), _mesh(0.5)
    uf = W.smooth_guess(mf, seed=4)
    u = interpolate_u(mf, uf, mc).reshape(3, mc.M, mc.N + 1)
    ref = uf.reshape(3, mf.M, mf.N + 1)[:, ::2, :]
    assert np.abs(u[:, :, 0] - ref[:, :, 0]).max() <= 1e-12
    assert np.abs(u[:, :, 1:] - ref[:, :, 1::2]).max() <= 1e-12


def test_smooth_field_to_fourth_order():
    """The error at the finer mesh's nodes falls by about 2^4 when the coarse
    spacing halves (bicubic splines on a smooth field)."""
    fine = _mesh(0.0625)
    exact = _analytic_u(fine)
    errs = []
    for h in (0.5, 0.25):
        mc = _mesh(h)
        errs.append(np.abs(interpolate_u(mc, _analytic_u(mc), fine) - exact).max())
    assert errs[0] <= 1e-4, errs  # 2.5e-5 measured; 21x and 16x per halving
    assert errs[0] / errs[1] >= 10.0, errs


def test_nodes_outside_take_the_nearest_edge():
    mc = _mesh(0.5)
    mf = W.Mesh(N=25, M=9, x1=-4.0, y1=-4.0, dx=0.5, dy=1.0, half=0)  # extends past x = 5 and |y| = 3
    u = interpolate_u(mc, W.smooth_guess(mc, seed=2), mf).reshape(3, mf.M, mf.N + 1)
    assert np.array_equal(u[:, 0], u[:, 1])      # y = -4 takes y = -3
    assert np.array_equal(u[:, :, 20:], np.repeat(u[:, :, 19:20], 6, axis=2))  # x > 5 takes x = 5


def test_bad_arguments():
    mc, mf = _mesh(0.5), _mesh(0.25, half=1)
    with pytest.raises(ValueError):
        interpolate_u(mc, W.flat_guess(mc), mf)
    with pytest.raises(ValueError):
        interpolate_u(mc, np.zeros(5), _mesh(0.25))
