"""The inversions of the block factorisation (App. B: the inverted diagonal
blocks of the block LU and the two-ended order's middle system) on seeded
matrices, through the C ABI: the FP64 rows kernel (method 0) and the blocked
double-float kernels, with panels spread over a CTA cluster where they fit
(method 1) and with one CTA per panel (method 2), against numpy's LU-based
inverse.

Sizes: one panel (37), the 181 x 61 slice block (546: method 1 eight panels
of 64 and a ragged one of 34 over eight CTAs; method 2 seventeen panels of 32
and a ragged one of 2), a wide-mesh block (1086) and the 181 x 61 middle
system (1638: method 2 panels of 16, ragged 6).  The matrices are
I + 0.5 G / sqrt(n) (G standard normal, condition number near 10) with their
rows shuffled, so that no diagonal entry is a usable pivot and partial
pivoting decides every column.

Bars (max |X - A^-1| over max |A^-1|): 1e-12 for FP64, 3e-12 for
double-float (46-bit products and sums, panels rounded to FP64 between
panels), about a hundred times the largest error measured on these matrices
(8e-15 and 2.6e-14).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_08803_gb300 import build
    build.build()


def _matrix(n, seed):
    rng = np.random.default_rng(seed)
    B = np.eye(n) + 0.5 * rng.standard_normal((n, n)) / np.sqrt(n)
    return B[rng.permutation(n)]


BARS = {0: 1e-12, 1: 3e-12, 2: 3e-12}


@pytest.mark.parametrize("method", [0, 1, 2])
@pytest.mark.parametrize("n", [1, 37, 546, 1086, 1638])
def test_inverse_matches_numpy(n, method):
    from paper_1709_08803_gb300 import bfs
    A = _matrix(n, 100 + n)
    X = bfs.gj_invert(torch.tensor(A, device="cuda"), method).cpu().numpy()
    ref = np.linalg.inv(A)
    err = np.abs(X - ref).max() / np.abs(ref).max()
    print(f"n={n} method={method}: max |X - inv(A)| / max |inv(A)| = {err:.2e}")
    assert err <= BARS[method], err


@pytest.mark.parametrize("method", [0, 1, 2])
def test_two_matrices_at_once(method):
    """The factorisation inverts the diagonal blocks of the two chains in one
    launch; each matrix gets its own pivots."""
    from paper_1709_08803_gb300 import bfs
    n = 546
    A = np.stack([_matrix(n, 7), _matrix(n, 8)])
    X = bfs.gj_invert(torch.tensor(A, device="cuda"), method).cpu().numpy()
    for q in range(2):
        ref = np.linalg.inv(A[q])
        assert np.abs(X[q] - ref).max() / np.abs(ref).max() <= BARS[method]


@pytest.mark.parametrize("method", [0, 1, 2])
@pytest.mark.parametrize("n", [100, 300])
def test_zero_column_is_singular(method, n):
    from paper_1709_08803_gb300 import bfs
    A = _matrix(n, 3)
    A[:, 61] = 0.0
    with pytest.raises(bfs.BfsError) as e:
        bfs.gj_invert(torch.tensor(A, device="cuda"), method)
    assert e.value.code == bfs.BFS_ESINGULAR


def test_sizes_the_tiles_do_not_take_are_refused():
    from paper_1709_08803_gb300 import bfs
    A = torch.zeros((4000, 4000), dtype=torch.float64, device="cuda")
    with pytest.raises(bfs.BfsError) as e:
        bfs.gj_invert(A, 1)  # a panel of 8 columns needs 4000 x 8 x 8 bytes and more
    assert e.value.code == bfs.BFS_EINVAL
