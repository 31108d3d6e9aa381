"""Pins of the FP64 completion ADMM (oracle/completion.py) against what the
paper and the mathematics fix: the DCT against scipy's, the least-squares
step against LAPACK on the stacked K, the first iterate from the all-ones
start, recovery of the block matrix of Section V, Comparison with Existing Methods with the exact shrinkage, and
the FP64 CPA run tracking the exact run."""
import numpy as np
import pytest

from oracle import admm as A
from oracle import completion as C
from paper_1705_07112_gb300 import inputs

RNG = np.random.default_rng(20240705)


def test_dct_matrix_is_scipys_orthonormal_dct():
    fft = pytest.importorskip("scipy.fft")
    for p in (1, 2, 7, 16, 33):
        T = C.dct_matrix(p)
        assert np.allclose(T, fft.dct(np.eye(p), norm="ortho", axis=0), atol=1e-13)
        assert np.allclose(T @ T.T, np.eye(p), atol=1e-13)


def test_psi_is_the_2d_dct_and_psi_t_its_inverse():
    fft = pytest.importorskip("scipy.fft")
    L = RNG.standard_normal((9, 13))
    Cm, Cn = C.dct_matrix(9), C.dct_matrix(13)
    P = C.psi(L, Cm, Cn)
    assert np.allclose(P, fft.dctn(L, norm="ortho"), atol=1e-12)
    assert np.allclose(C.psi_t(P, Cm, Cn), L, atol=1e-12)


def test_least_squares_step_equals_lstsq_on_the_stacked_K():
    m, n = 4, 3
    omega = (RNG.random((m, n)) < 0.7).astype(np.float64)
    Cm, Cn = C.dct_matrix(m), C.dct_matrix(n)
    a = [RNG.standard_normal((m, n)) for _ in range(4)]
    # row-major vec: vec(C_m L C_n^T) = (C_m kron C_n) vec(L)
    Id = np.eye(m * n)
    K = np.vstack([Id, np.kron(Cm, Cn), np.diag(omega.ravel()), Id])
    rhs = np.concatenate([x.ravel() for x in a])
    ref = np.linalg.lstsq(K, rhs, rcond=None)[0].reshape(m, n)
    got = C.ls_update(a[0], a[1], a[2], a[3], omega, Cm, Cn)
    assert np.allclose(got, ref, atol=1e-12)


def test_first_iterate_from_the_all_ones_start():
    """a = z_0 - u_0 = (0, Psi 1 - 1, omega - 1, 0) and omega (omega - 1) = 0,
    so l_1 = (1 - Psi^T 1) / (3 + omega)."""
    D, I, mask = inputs.block_completion(0, 20, 4, 0.2)
    omega = mask.astype(np.float64)
    Cm = C.dct_matrix(20)
    ones = np.ones((20, 20))
    l1, _, E = C.completion_admm(I, mask, 0.1, 1, A.svt_exact(0.5))
    ref = (ones - C.psi_t(ones, Cm, Cm)) / (3.0 + omega)
    assert np.allclose(l1, ref, atol=1e-13)
    assert abs(E[0] - np.linalg.norm(ref - ones) / np.linalg.norm(ref)) < 1e-13


@pytest.mark.parametrize("size,rank", [(60, 6), (60, 30)])
def test_exact_run_completes_the_block_matrix(size, rank):
    """The matrix of Section V, Comparison with Existing Methods, J - blkdiag(0.5 1 1^T, n) with 10 % of its entries
    zeroed is restored: the missing entries to 2e-3, the observed ones kept,
    the range constraint met, within the paper's stop rule E_t < 1e-4."""
    D, I, mask = inputs.block_completion(0, size, rank, 0.10)
    D = D.astype(np.float64)
    miss = mask == 0
    l, z1, E = C.completion_admm(I, mask, 0.1, 400, A.svt_exact(0.5), tol=1e-4)
    assert E[-1] < 1e-4 and len(E) < 400
    assert np.linalg.norm((l - D)[miss]) / np.linalg.norm(D[miss]) < 2e-3
    assert np.max(np.abs((l - D)[~miss])) < 5e-3
    assert l.min() > -5e-3 and l.max() < 1 + 5e-3
    # the shrinkage output agrees with l at convergence
    assert np.linalg.norm(z1 - l) / np.linalg.norm(l) < 5e-3


def test_cpa_run_tracks_the_exact_run():
    D, I, mask = inputs.block_completion(1, 40, 4, 0.10)
    le, _, _ = C.completion_admm(I, mask, 0.1, 30, A.svt_exact(0.5))
    lc, _, _ = C.completion_admm(I, mask, 0.1, 30, A.svt_cpa(0.5, 120))
    assert np.linalg.norm(lc - le) / np.linalg.norm(le) < 2e-3
