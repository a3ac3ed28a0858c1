"""Pins of the oracle's FFT and operator exponentials against the defining
sums, a library FFT, closed forms and a truncated Taylor series."""
import numpy as np
import pytest

from oracle import fourier, operators


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


@pytest.mark.parametrize("N", [1, 2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("inverse", [False, True])
def test_fft_matches_direct_dft(N, inverse):
    x = _rand((3, N, 5), N)
    a = fourier.fft_axis(x, 1, inverse)
    b = fourier.dft_axis(x, 1, inverse)
    assert np.max(np.abs(a - b)) <= 1e-13 * max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("N", [128, 1024, 4096])
def test_fft_matches_library_fft(N):
    x = _rand((2, N), N)
    assert np.max(np.abs(fourier.fft_axis(x, 1) - np.fft.fft(x, axis=1))) < 1e-12 * np.sqrt(N) * 10
    assert np.max(np.abs(fourier.fft_axis(x, 1, True) - np.fft.ifft(x, axis=1))) < 1e-14 * 10


def test_fft_closed_forms():
    N = 64
    e = np.zeros(N, complex)
    e[0] = 1.0
    assert np.allclose(fourier.fft_axis(e, 0), np.ones(N), atol=0, rtol=1e-15)
    m = 5
    tone = np.exp(2j * np.pi * m * np.arange(N) / N)
    out = fourier.fft_axis(tone, 0)
    ref = np.zeros(N, complex)
    ref[m] = N
    assert np.max(np.abs(out - ref)) < 1e-12


def test_fft_roundtrip_and_parseval():
    x = _rand((2, 32, 16, 8), 7)
    f = fourier.fftn_grid(x)
    assert np.max(np.abs(fourier.fftn_grid(f, inverse=True) - x)) < 1e-14
    P = 32 * 16 * 8
    assert np.sum(np.abs(f) ** 2) / P == pytest.approx(np.sum(np.abs(x) ** 2), rel=1e-13)


def test_momenta_layout():
    n, qmin, qmax = 8, -2.0, 2.0
    dq = 0.5
    p = operators.axis_momenta(n, qmin, qmax)
    k = np.array([0, 1, 2, 3, -4, -3, -2, -1], float)
    assert np.allclose(p, 2 * np.pi * k / (n * dq), rtol=0, atol=1e-15)
    q = operators.axis_positions(n, qmin, qmax)
    assert q[0] == qmin and q[-1] == pytest.approx(qmax - dq)


def _taylor_expm(M, terms=60):
    out = np.eye(M.shape[0], dtype=complex)
    term = np.eye(M.shape[0], dtype=complex)
    for k in range(1, terms):
        term = term @ M / k
        out = out + term
    return out


@pytest.mark.parametrize("S", [2, 3, 4])
def test_potential_exponential_vs_taylor(S):
    rng = np.random.default_rng(S)
    P = 7
    A = rng.normal(size=(S, S, P)) * 0.3
    Vf = 0.5 * (A + A.transpose(1, 0, 2))
    tau = 0.7
    U = operators.expm_potential(Vf, tau)
    for g in range(P):
        ref = _taylor_expm(-1j * tau * Vf[:, :, g])
        assert np.max(np.abs(U[:, :, g] - ref)) < 1e-14
    if S == 2:
        U2 = operators.expm_potential_2x2(Vf, tau)
        assert np.max(np.abs(U2 - U)) < 1e-14


def test_2x2_closed_form_limits_and_unitarity():
    rng = np.random.default_rng(3)
    P = 50
    Vf = np.zeros((2, 2, P))
    Vf[0, 0] = rng.normal(size=P)
    Vf[1, 1] = rng.normal(size=P)
    Vf[0, 1] = Vf[1, 0] = rng.normal(size=P)
    Vf[:, :, :5] = 0.0                      # r = 0 and v0 = 0: identity
    Vf[0, 0, 5:10] = Vf[1, 1, 5:10] = 0.3   # r = 0, v0 != 0: pure phase
    Vf[0, 1, 5:10] = Vf[1, 0, 5:10] = 0.0
    tau = 3.3
    U = operators.expm_potential_2x2(Vf, tau)
    assert np.allclose(U[:, :, :5], np.eye(2)[:, :, None], atol=1e-16)
    assert np.allclose(U[0, 0, 5:10], np.exp(-1j * tau * 0.3), atol=1e-15)
    assert np.allclose(U[0, 1, 5:10], 0, atol=1e-16)
    for g in range(P):
        u = U[:, :, g]
        assert np.max(np.abs(u.conj().T @ u - np.eye(2))) < 1e-14
        assert abs(u[0, 1] - u[1, 0]) == 0          # complex symmetric
    assert np.max(np.abs(U - operators.expm_potential(Vf, tau))) < 1e-13


def test_unpack_potential_layout():
    S = 3
    Vp = np.arange(6, dtype=float).reshape(6, 1)
    Vf = operators.unpack_potential(Vp, S)[:, :, 0]
    assert np.array_equal(Vf, np.array([[0, 1, 2], [1, 3, 4], [2, 4, 5]], float))


def test_apply_potential_is_matvec():
    rng = np.random.default_rng(9)
    U = rng.normal(size=(3, 3, 4)) + 1j * rng.normal(size=(3, 3, 4))
    psi = rng.normal(size=(3, 4)) + 1j * rng.normal(size=(3, 4))
    out = operators.apply_potential(U, psi)
    for g in range(4):
        assert np.allclose(out[:, g], U[:, :, g] @ psi[:, g], rtol=0, atol=1e-15)
