"""The dense coarsest-level solve of the multigrid preconditioner
(cahn_lap5_coarse_inverse, host only): checked on the CPU against the
5-point operator assembled here from its definition and against numpy's
dense linear algebra.  The zero-flux operator without a diagonal term is
singular; its P must be the pseudo-inverse in the wall-weighted inner
product (constants to zero, exact on compatible right-hand sides, weighted
mean zero, self-adjoint in that inner product)."""
import numpy as np
import pytest

from paper_1811_11842_gb300 import binding
from paper_1811_11842_gb300 import build as B


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    binding.load()


def assemble(nx, ny, walls, c0, cx, cy):
    """A of the 5-point operator, x periodic, rows 0..ny; walls 0: the row
    beyond a wall reflected; walls 1: wall rows c0 x (held at zero by the
    solve)."""
    n = nx * (ny + 1)
    A = np.zeros((n, n))
    for j in range(ny + 1):
        for i in range(nx):
            e = j * nx + i
            if walls == 1 and j in (0, ny):
                A[e, e] = c0
                continue
            js = (1 if j == 0 else j - 1) if walls == 0 else j - 1
            jn = (ny - 1 if j == ny else j + 1) if walls == 0 else j + 1
            A[e, e] += c0 + 2 * cx + 2 * cy
            A[e, j * nx + (i - 1) % nx] -= cx
            A[e, j * nx + (i + 1) % nx] -= cx
            A[e, js * nx + i] -= cy
            A[e, jn * nx + i] -= cy
    return A


def weights(nx, ny):
    w = np.ones((ny + 1, nx))
    w[0] = w[-1] = 0.5
    return w.ravel()


@pytest.mark.parametrize("nx,ny,cx,cy", [(32, 8, 64.0, 64.0), (8, 4, 3.0, 5.0), (2, 1, 1.0, 7.0),
                                         (16, 6, 0.25, 40.0)])
def test_singular_zero_flux_pseudo_inverse(nx, ny, cx, cy):
    _, P = binding.cahn_lap5_coarse_inverse(nx, ny, 0, 0.0, cx, cy)
    A = assemble(nx, ny, 0, 0.0, cx, cy)
    w = weights(nx, ny)
    n = A.shape[0]
    # the constants are the null space: A 1 = 0, and P 1 = 0
    assert np.abs(A @ np.ones(n)).max() == 0.0
    scale = np.abs(P).max()
    assert np.abs(P @ np.ones(n)).max() <= 1e-12 * scale * n
    # compatible b (weighted sum zero): A P b = b, weighted sum of P b zero
    rng = np.random.default_rng(5)
    for _ in range(3):
        b = rng.standard_normal(n)
        b -= (w @ b) / w.sum()
        x = P @ b
        assert np.linalg.norm(A @ x - b) <= 1e-11 * np.linalg.norm(b)
        assert abs(w @ x) <= 1e-11 * np.linalg.norm(x) * np.sqrt(n)
    # self-adjoint in the weighted inner product: W P symmetric
    WP = w[:, None] * P
    assert np.abs(WP - WP.T).max() <= 1e-11 * np.abs(WP).max()
    # the pseudo-inverse: agrees with numpy's Moore-Penrose inverse of the
    # symmetrised operator W^1/2 A W^-1/2
    s = np.sqrt(w)
    Ahat = s[:, None] * A / s[None, :]
    Phat = np.linalg.pinv(Ahat, rcond=1e-12)
    assert np.allclose(s[:, None] * P / s[None, :], Phat, rtol=0, atol=1e-10 * np.abs(Phat).max())


@pytest.mark.parametrize("nx,ny,c0,cx,cy", [(8, 4, 2.0, 3.0, 5.0), (4, 2, 1e4, 1.0, 1.0)])
def test_zero_flux_with_diagonal_is_the_inverse(nx, ny, c0, cx, cy):
    _, P = binding.cahn_lap5_coarse_inverse(nx, ny, 0, c0, cx, cy)
    A = assemble(nx, ny, 0, c0, cx, cy)
    Ainv = np.linalg.inv(A)
    assert np.abs(P - Ainv).max() <= 1e-12 * np.abs(Ainv).max()


@pytest.mark.parametrize("nx,ny,c0", [(8, 4, 1e3), (16, 8, 0.0), (4, 2, 5.0)])
def test_held_walls_invert_the_interior(nx, ny, c0):
    cx, cy = 2.0, 9.0
    _, P = binding.cahn_lap5_coarse_inverse(nx, ny, 1, c0, cx, cy)
    A = assemble(nx, ny, 1, c0, cx, cy)
    n = A.shape[0]
    wall = np.zeros(n, dtype=bool)
    wall[:nx] = wall[-nx:] = True
    assert np.all(P[wall] == 0.0) and np.all(P[:, wall] == 0.0)
    inner = ~wall
    Ainv = np.linalg.inv(A[np.ix_(inner, inner)])
    assert np.abs(P[np.ix_(inner, inner)] - Ainv).max() <= 1e-12 * np.abs(Ainv).max()


@pytest.mark.parametrize("args", [(1, 4, 0, 0.0, 1.0, 1.0), (4, 0, 0, 0.0, 1.0, 1.0),
                                  (64, 64, 0, 0.0, 1.0, 1.0), (4, 2, 2, 0.0, 1.0, 1.0),
                                  (4, 2, 0, -1.0, 1.0, 1.0), (4, 2, 0, 0.0, 0.0, 0.0),
                                  (4, 2, 0, 0.0, float("nan"), 1.0)])
def test_bad_arguments_rejected(args):
    code, _ = binding.cahn_lap5_coarse_inverse(*args, check=False)
    assert code == binding.CAHN_ERR_ARG
    assert "cahn_lap5_coarse_inverse" in binding.load().cahn_last_error(None).decode()
