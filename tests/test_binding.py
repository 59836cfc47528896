"""The Python binding's argument checks, without a GPU: a buffer of the wrong
length, type or device is refused before its pointer reaches the library,
also under python -O (the checks are not asserts)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1709_08803_gb300 import bfs
from paper_1709_08803_gb300 import surrogate as S
from paper_1709_08803_gb300 import workloads as W


def _bare_context(n):
    ctx = bfs.Context.__new__(bfs.Context)  # no device context behind it
    ctx.n, ctx._ctx = n, None
    return ctx


@pytest.mark.parametrize("t", [torch.zeros(12, dtype=torch.float64),            # host memory
                               torch.zeros(12, dtype=torch.float32),            # wrong type
                               torch.zeros(11, dtype=torch.float64),            # wrong length
                               np.zeros(12)])                                   # not a tensor
def test_device_vectors_are_checked(t):
    with pytest.raises(ValueError):
        _bare_context(12)._vec(t)


@pytest.mark.parametrize("a", [np.zeros(11), np.zeros(12, dtype=np.float32), np.zeros((12, 2))[:, 0],
                               torch.zeros(12, dtype=torch.float64)])
def test_host_vectors_are_checked(a):
    with pytest.raises(ValueError):
        _bare_context(12)._host_vec(a)


def test_host_vector_accepted():
    a = np.zeros(12)
    assert _bare_context(12)._host_vec(a).value == a.ctypes.data


def test_static_residual_checks_every_buffer():
    mesh = W.mesh_box(9, 5, 0.4, 0.4)
    z = torch.zeros(mesh.N * mesh.M, dtype=torch.float64)
    u = torch.zeros(mesh.n_unknowns, dtype=torch.float64)
    with pytest.raises(ValueError):
        bfs.residual_static(mesh, z, z, z, 0.7, u)


def _bare_net(H=9, Wd=37, batch_max=2):
    net = S.CNO.__new__(S.CNO)
    net.H, net.W, net.batch_max, net._n = H, Wd, batch_max, None
    return net


@pytest.mark.parametrize("shape,dtype", [((2, 9, 37, 4), torch.float32),   # host memory
                                         ((2, 9, 37, 4), torch.float64),
                                         ((9, 37, 4), torch.float32),
                                         ((3, 9, 37, 4), torch.float32),
                                         ((2, 37, 9, 4), torch.float32)])
def test_network_images_are_checked(shape, dtype):
    with pytest.raises(ValueError):
        _bare_net()._images(torch.zeros(shape, dtype=dtype), 4)


def test_network_parameter_count_is_checked():
    net = _bare_net()
    net.np = S.num_params()
    with pytest.raises(ValueError):
        net.set_params(np.zeros(net.np - 1, dtype=np.float32))
    with pytest.raises(ValueError):
        net.set_params(np.zeros(net.np, dtype=np.float32), scale=np.ones(2, dtype=np.float32))


def test_batch_vector_count_is_checked():
    b = bfs.Batch.__new__(bfs.Batch)
    b.B, b.n, b._b = 2, [12, 12], None
    with pytest.raises(ValueError):
        b._ptrs([torch.zeros(12, dtype=torch.float64)])
    with pytest.raises(ValueError):
        b._ptrs([torch.zeros(12, dtype=torch.float64)] * 2)  # host memory
