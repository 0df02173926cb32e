"""Pins of the boundary-data spectral oracle (Eqs. SCVS_bc and mode_error) and
of its a posteriori side (mode energies, reconstruction increments) against
closed forms and an independent library transform."""
import numpy as np
import pytest
import scipy.sparse as spm

from oracle import bcspec


def _cosines(n_t, a0, amps, phases, T=1.0):
    t = np.arange(n_t) * T / n_t
    g = np.full(n_t, a0, dtype=np.float64)
    for k, (a, ph) in enumerate(zip(amps, phases), start=1):
        g += a * np.cos(2 * np.pi * k * t / T + ph)
    return g


def test_coefficients_of_a_cosine_series():
    rng = np.random.default_rng(0)
    n_t, K = 48, 9
    amps, ph = rng.uniform(0.1, 2.0, K), rng.uniform(0, 2 * np.pi, K)
    g = np.stack([_cosines(n_t, 0.7, amps, ph), _cosines(n_t, -1.3, amps[::-1], ph[::-1])], axis=1)
    G = bcspec.fourier_coefficients(g, K + 1)
    # g~_0 = mean, g~_k = a_k e^{j phi_k} / 2 (Eq. SCVS_bc with e^{-j omega t})
    assert np.allclose(G[0], [0.7, -1.3], atol=1e-14)
    assert np.allclose(G[1:, 0], amps * np.exp(1j * ph) / 2, atol=1e-13)
    assert np.allclose(G[1:, 1], amps[::-1] * np.exp(1j * ph[::-1]) / 2, atol=1e-13)
    c = bcspec.solver_modes(G)
    assert np.allclose(c[1:, 0], amps * np.exp(1j * ph), atol=1e-13) and c[0, 0] == G[0, 0]
    # the full series gives back the samples
    assert np.allclose(bcspec.truncated_series(c, n_t, K), g, atol=1e-12)


def test_coefficients_match_a_real_fft():
    rng = np.random.default_rng(1)
    g = rng.standard_normal((40, 7, 3))
    G = bcspec.fourier_coefficients(g, 20)
    ref = np.fft.rfft(g, axis=0)[:20] / 40
    assert np.allclose(G, ref, atol=1e-14)


def test_truncation_error_closed_form():
    # c_k = k^-2 e^{j phi_k} (|c_k| ~ omega^-2), c_0 = 1, band limit K: the mean of
    # cos^2 is 1/2 and distinct harmonics are orthogonal on the samples, so
    # e_M^2(N) = sum_{k>N} k^-4 / 2 / (1 + sum_k k^-4 / 2)
    n_t, K = 64, 12
    rng = np.random.default_rng(2)
    ph = rng.uniform(0, 2 * np.pi, K)
    k = np.arange(1, K + 1)
    g = _cosines(n_t, 1.0, k ** -2.0, ph)[:, None]
    e2 = bcspec.truncation_errors([(g, np.ones(1))], K + 3)
    total = 1.0 + np.sum(k ** -4.0) / 2
    for N in range(K + 3):
        tail = np.sum(k[k > N] ** -4.0) / 2
        assert e2[N] == pytest.approx(tail / total, rel=1e-10, abs=1e-28)
    assert np.all(np.diff(e2) <= 1e-30) and e2[K] < 1e-28


def test_weighted_norm_and_sum_of_fields():
    n_t = 32
    g1 = _cosines(n_t, 1.0, [1.0, 0.5], [0.0, 1.0])
    g2 = _cosines(n_t, 0.0, [0.0, 0.0, 2.0], [0.0, 0.0, 0.3])
    g = np.stack([g1, g2], axis=1)
    w = np.array([3.0, 0.25])
    e2 = bcspec.truncation_errors([(g, w)], 5)
    tot = 3.0 * (1.0 + 0.5 + 0.125) + 0.25 * 2.0
    tails = [3.0 * (0.5 + 0.125) + 0.25 * 2.0, 3.0 * 0.125 + 0.25 * 2.0, 0.25 * 2.0, 0.0, 0.0]
    assert np.allclose(e2, np.array(tails) / tot, atol=1e-14)
    # the Dirichlet and Neumann terms of Eq. mode_error add
    h = np.stack([g2, g1], axis=1)
    both = bcspec.truncation_errors([(g, w), (h, np.ones(2))], 5)
    assert np.allclose(both, e2 + bcspec.truncation_errors([(h, np.ones(2))], 5), atol=1e-14)
    # a zero field adds nothing
    assert np.allclose(bcspec.truncation_errors([(g, w), (np.zeros((n_t, 2)), w)], 5), e2, atol=0)


def test_select_modes():
    n_t, K = 64, 12
    k = np.arange(1, K + 1)
    g = _cosines(n_t, 1.0, k ** -2.0, np.zeros(K))[:, None]
    N, e2 = bcspec.select_modes([(g, np.ones(1))], 1e-3, 16)
    assert np.sqrt(e2[N]) < 1e-3 <= np.sqrt(e2[N - 1])
    assert bcspec.select_modes([(g, np.ones(1))], 1e-20, 4)[0] is None
    with pytest.raises(ValueError):
        bcspec.truncation_errors([(g, np.ones(1))], 33)


def _mass(n, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n))
    return spm.csr_matrix(B @ B.T + n * np.eye(n))


def test_mode_energies_closed_form():
    # time averages over one period of harmonics: ||Re U_0||^2 for omega_0 = 0 and
    # (1/2) U_k^H M U_k for omega_k = 2 pi k / T (the e^{2 j omega t} term averages out)
    N, d, m, T = 9, 3, 5, 2.0
    Ms = _mass(N, 3)
    rng = np.random.default_rng(4)
    U = rng.standard_normal((m, N, d)) + 1j * rng.standard_normal((m, N, d))
    om = 2 * np.pi * np.arange(m) / T
    E = bcspec.mode_energies(Ms, U, om, T, 32)
    M = Ms.toarray()
    assert E[0] == pytest.approx(sum(U[0, :, c].real @ M @ U[0, :, c].real for c in range(d)), rel=1e-12)
    for k in range(1, m):
        ref = 0.5 * sum(np.real(np.conj(U[k, :, c]) @ M @ U[k, :, c]) for c in range(d))
        assert E[k] == pytest.approx(ref, rel=1e-12)


def test_increments_closed_form_and_orthogonality():
    N, d, m, T = 7, 2, 6, 1.0
    Ms = _mass(N, 5)
    rng = np.random.default_rng(6)
    U = rng.standard_normal((m, N, d)) + 1j * rng.standard_normal((m, N, d))
    U[0] = U[0].real  # real steady mode
    om = 2 * np.pi * np.arange(m) / T
    E = bcspec.mode_energies(Ms, U, om, T, 32)
    inc = bcspec.a_posteriori_increments(Ms, U, om, T, 32)
    # distinct harmonics are orthogonal in L2(Omega x T): the truncated series'
    # energy is the sum of the modes' energies and the change is mode N alone
    assert np.allclose(inc, E / np.cumsum(E), rtol=1e-11)
    assert inc[0] == pytest.approx(1.0)
    # a zero mode changes nothing
    U[3] = 0
    inc = bcspec.a_posteriori_increments(Ms, U, om, T, 32)
    assert abs(inc[3]) < 1e-28
