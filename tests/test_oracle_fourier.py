"""Pins for the oracle's structured (Fourier) operator of Sec. 4, Phi_t = Omega_t F: the FFT
form of A = beta Re(Phi^H Phi) + diag(alpha) and of b0 = beta Re(Phi^H y) against the dense
real matrix [Re Phi; Im Phi] built entry by entry from the DFT's definition, and a
closed-form special case (every frequency sampled: Phi^H Phi = I)."""
import numpy as np
import pytest

from oracle import cofem
from paper_2310_00420_gb300 import synth


@pytest.fixture(scope="module")
def wl():
    return synth.make_fourier("pin", 3, 2, 64, 16, sparsity=0.1, K=4, seed=5)


def test_fourier_operator_matches_dense(wl):
    rng = np.random.default_rng(1)
    alpha = rng.uniform(0.1, 3.0, size=wl.D)
    V = rng.standard_normal((wl.D, 5))
    for t in range(wl.T):
        P = wl.phi_real(t)
        dense = cofem.apply_A(P, wl.beta, alpha, V)
        fast = cofem.apply_A_fourier(wl.mask[t], wl.beta, alpha, V)
        np.testing.assert_allclose(fast, dense, rtol=1e-12, atol=1e-10 * np.abs(dense).max())
        v = V[:, 0]
        np.testing.assert_allclose(cofem.apply_A_fourier(wl.mask[t], wl.beta, alpha, v),
                                   dense[:, 0], rtol=1e-12, atol=1e-10 * np.abs(dense).max())


def test_fourier_rhs_matches_dense(wl):
    for t in range(wl.T):
        dense = cofem.rhs_mean(wl.phi_real(t), wl.y_real(t), wl.beta)
        fast = cofem.rhs_mean_fourier(wl.mask[t], wl.yt(t), wl.beta)
        np.testing.assert_allclose(fast, dense, rtol=1e-10, atol=1e-9 * np.abs(dense).max())


def test_full_sampling_is_the_identity():
    """All D frequencies sampled: Phi = F is unitary, so A = beta I + diag(alpha) and
    b0 = beta z for noiseless data."""
    D = 32
    rng = np.random.default_rng(2)
    alpha = rng.uniform(0.1, 2.0, size=D)
    v = rng.standard_normal(D)
    mask = np.ones(D, dtype=np.uint8)
    np.testing.assert_allclose(cofem.apply_A_fourier(mask, 7.0, alpha, v), (7.0 + alpha) * v,
                               rtol=1e-13)
    z = rng.standard_normal(D)
    y = np.fft.fft(z) / np.sqrt(D)
    np.testing.assert_allclose(cofem.rhs_mean_fourier(mask, y, 3.0), 3.0 * z, rtol=1e-12,
                               atol=1e-12)


def test_fourier_sensing_estep_equals_dense_estep():
    """The E-step on FourierSensing tasks (FFT-form A v, b0 and diagonal) equals the E-step on
    the dense real-stacked matrices, plain and Jacobi-preconditioned, at a length that is not
    a power of two."""
    wl = synth.make_fourier("f", 3, 2, 160, 40, K=4, cg_tol=1e-12, cg_max_iter=200, seed=2)
    alpha = np.random.default_rng(3).uniform(0.5, 50.0, size=(2, 160))
    Y = [wl.y_real(t) for t in range(wl.T)]
    dense = [wl.phi_real(t) for t in range(wl.T)]
    ops = [cofem.FourierSensing(wl.mask[t]) for t in range(wl.T)]
    for t in range(wl.T):
        np.testing.assert_allclose(ops[t].diag(wl.beta, alpha[0]),
                                   cofem.jacobi_diag(dense[t], wl.beta, alpha[0]), rtol=1e-12)
    for pc in (False, True):
        a = cofem.cofem_estep(dense, Y, alpha, wl.pi, wl.beta, wl.K, 1, 0, 1e-12, 200,
                              precond=pc)
        b = cofem.cofem_estep(ops, Y, alpha, wl.pi, wl.beta, wl.K, 1, 0, 1e-12, 200, precond=pc)
        for key in ("mu", "s", "logdet", "q"):
            np.testing.assert_allclose(b[key], a[key], rtol=1e-8, atol=1e-12)


def test_fourier_workload_subset_keeps_tasks():
    wl = synth.fourier_small()
    sub = wl.subset([1, 3])
    assert sub.T == 2 and list(sub.N) == [wl.N[1], wl.N[3]]
    np.testing.assert_array_equal(sub.mask, wl.mask[[1, 3]])
    for i, t in enumerate((1, 3)):
        np.testing.assert_array_equal(sub.yt(i), wl.yt(t))
        np.testing.assert_array_equal(sub.phi_real(i), wl.phi_real(t))
    assert sub.row_off[-1] == sub.y.shape[0]
