"""Tensor-core dense SPD solve (FP32 factor with BF16-split trailing updates on tcgen05, FP64
conjugate gradients) against LAPACK on seeded SPD matrices of set condition numbers, sizes that
span one to three 128-row slabs with ragged padding, and the failure cases."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


def spd(rng, n, kappa):
    """Q diag(lambda) Q^T with eigenvalues log-spaced over [1, kappa], then a random diagonal
    scaling (what the Jacobi scaling has to undo)."""
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.logspace(0, np.log10(kappa), n)
    A = (q * lam) @ q.T
    s = np.exp(rng.uniform(-3, 3, n))
    return A * s[:, None] * s[None, :]


def batch(seed, B, n, kappa):
    rng = np.random.default_rng(seed)
    A = np.stack([spd(rng, n, kappa) for _ in range(B)])
    b = rng.standard_normal((B, n))
    return A, b


def run(A, b, steps, tol):
    from paper_2207_09442_b300 import dense
    x, st, res = dense.spd_solve(torch.as_tensor(A, device=DEV), torch.as_tensor(b, device=DEV), steps, tol)
    torch.cuda.synchronize()
    return x.cpu().numpy(), st.cpu().numpy(), res.cpu().numpy()


@pytest.mark.parametrize("n", [1, 6, 96, 128, 200, 256, 384])
@pytest.mark.parametrize("kappa", [1e2, 1e6])
def test_refined_solution_matches_lapack(n, kappa):
    A, b = batch(7 + n, 5, n, kappa)
    x, st, res = run(A, b, 40, 1e-13)
    for k in range(len(A)):
        ref = np.linalg.solve(A[k], b[k])
        r = np.linalg.norm(b[k] - A[k] @ x[k]) / np.linalg.norm(b[k])
        e = np.linalg.norm(x[k] - ref) / np.linalg.norm(ref)
        assert st[k] >= 0 and st[k] <= 15, (k, st[k])
        # the scaled system D A D y = D b stops at a (recurrence) relative residual <= 1e-13;
        # the solution error is kappa(A) times the rounding of either route (LAPACK's included),
        # and the true residual carries ~1e-16 kappa(A) cond(D) of rounding in the products
        assert res[k] <= 1e-13, res[k]
        assert e <= max(1e-11, kappa * 2e-15), (k, e)
        dg = 2.0 ** -np.floor(np.log2(np.diag(A[k])) / 2)
        assert r <= max(1e-12, 1e-15 * kappa) * dg.max() / dg.min(), (k, r)


@pytest.mark.parametrize("n", [64, 384])
def test_factor_alone_is_fp32_accurate(n):
    """max_steps = 0: x = M^-1 b with the tensor-core factor.  A split into one BF16 term would
    leave ~4e-3 relative error; the three-term split keeps FP32 accuracy (kappa * ~1e-6)."""
    A, b = batch(11, 4, n, 1e2)
    x, st, _ = run(A, b, 0, 0.0)
    for k in range(len(A)):
        ref = np.linalg.solve(A[k], b[k])
        e = np.linalg.norm(x[k] - ref) / np.linalg.norm(ref)
        assert st[k] == 0
        assert e < 2e-5, e


def test_large_batch_uses_every_problem_independently():
    A, b = batch(3, 40, 384, 1e4)
    A[5] = A[0]
    b[5] = b[0]
    x, st, res = run(A, b, 40, 1e-12)
    assert np.array_equal(x[5], x[0])  # bitwise: fixed-order arithmetic, no atomics
    for k in range(len(A)):
        ref = np.linalg.solve(A[k], b[k])
        assert np.linalg.norm(x[k] - ref) / np.linalg.norm(ref) < 1e-9


def test_indefinite_matrix_is_reported_not_solved():
    rng = np.random.default_rng(5)
    A = np.stack([spd(rng, 96, 1e2) for _ in range(3)])
    b = rng.standard_normal((3, 96))
    q, _ = np.linalg.qr(rng.standard_normal((96, 96)))
    A[1] = (q * np.linspace(-1.0, 2.0, 96)) @ q.T  # eigenvalues of both signs
    x, st, _ = run(A, b, 40, 1e-12)
    assert st[1] in (-1, -2)
    assert not np.isfinite(x[1]).all() or st[1] == -2
    for k in (0, 2):
        ref = np.linalg.solve(A[k], b[k])
        assert np.linalg.norm(x[k] - ref) / np.linalg.norm(ref) < 1e-10


def test_rejects_orders_beyond_the_limit():
    from paper_2207_09442_b300 import dense, dnls
    A = torch.zeros(1, 385, 385, dtype=torch.float64, device=DEV)
    with pytest.raises(dnls.DnlsError) as e:
        dense.spd_solve(A, torch.zeros(1, 385, dtype=torch.float64, device=DEV))
    assert e.value.status == dnls.ERR_UNSUPPORTED
