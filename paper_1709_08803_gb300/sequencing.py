"""Mesh sequencing: an unknown vector carried from a coarse mesh to a finer
one, as the start of Newton on the finer mesh (host-side, once per solve)."""
from __future__ import annotations

import numpy as np

from .workloads import Mesh


def interpolate_u(mesh_c: Mesh, u_c: np.ndarray, mesh_f: Mesh) -> np.ndarray:
    """The unknown vector on mesh_f carried over from one on mesh_c.

    Per field (zeta, phi, psi) the unknowns of a slice are the value at the
    upstream edge and the x-derivatives at the N nodes (Sec. 3.1).  The nodal
    values of mesh_c follow from the trapezoid rule along x, as the residual
    reconstructs them.  The x-derivatives and the nodal values are then taken
    from interpolating bicubic splines at mesh_f's nodes and at its upstream
    edge; the splines drop to a lower degree where a mesh has fewer than four
    nodes in a direction.  Nodes of mesh_f outside mesh_c's rectangle take
    the value at its nearest edge.  Both meshes must be of the same kind
    (full, or half with y1 = 0)."""
    from scipy.interpolate import RectBivariateSpline, make_interp_spline

    if mesh_c.half != mesh_f.half:
        raise ValueError("both meshes must be full, or both half")
    u_c = np.asarray(u_c, dtype=np.float64)
    if u_c.shape != (mesh_c.n_unknowns,):
        raise ValueError(f"u_c has shape {u_c.shape}, expected ({mesh_c.n_unknowns},)")
    Nc, Mc, Nf, Mf = mesh_c.N, mesh_c.M, mesh_f.N, mesh_f.M
    xc, yc, xf, yf = mesh_c.x(), mesh_c.y(), mesh_f.x(), mesh_f.y()
    xq = np.clip(xf, xc[0], xc[-1])
    yq = np.clip(yf, yc[0], yc[-1])
    x1q = np.array([min(max(mesh_f.x1, xc[0]), xc[-1])])
    kx, ky = min(3, Nc - 1), min(3, Mc - 1)
    f3 = u_c.reshape(3, Mc, Nc + 1)
    out = np.empty((3, Mf, Nf + 1))
    for f in range(3):
        q1, qx = f3[f, :, 0], f3[f, :, 1:]
        q = np.empty_like(qx)
        q[:, 0] = q1
        q[:, 1:] = q1[:, None] + np.cumsum(0.5 * mesh_c.dx * (qx[:, 1:] + qx[:, :-1]), axis=1)
        if Mc == 1:  # a single slice: splines in x only
            out[f, :, 1:] = make_interp_spline(xc, qx[0], k=kx)(xq)[None, :]
            out[f, :, 0] = make_interp_spline(xc, q[0], k=kx)(x1q)[0]
            continue
        # first coordinate y (degree ky), second x (degree kx)
        out[f, :, 1:] = RectBivariateSpline(yc, xc, qx, kx=ky, ky=kx)(yq, xq)
        out[f, :, 0] = RectBivariateSpline(yc, xc, q, kx=ky, ky=kx)(yq, x1q)[:, 0]
    return out.reshape(-1)
