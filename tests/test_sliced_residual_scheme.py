"""The digit-plane scheme of the mixed-path recompute residual, on the host.

The GPU forms R = I - A N0 (A = N^-1 in FP64, N0 the drifted FP32 N) from
exponent-aligned digit planes (Ozaki, Ogita, Oishi, Rump, Numer. Algorithms
59, 2012): each row of A as five signed 9-bit digits under one power of two,
each column of N0 as four, the plane products with s + t <= 5 summed per group
s + t, groups 0 and 1 exactly per 128 terms of K, groups 2..5 in FP32.  These
tests check that scheme's parameters in numpy, independently of the GPU:

- the digits are integers of magnitude <= 256 (exact in FP16) and rebuild each
  row (column) to 2^-44 (2^-35) of its largest entry;
- the partial sums of the exact groups stay within 2^24 over a chunk of 128;
- on an oracle configuration at beta = 20 (kappa(N) ~ 1e6) with N0 the FP32 N
  drifted by 1e-5, one Newton step with the sliced residual, FP32 rounding of
  groups 2..5 every 16 terms included, leaves N at the error the exact residual
  leaves (the FP32 storage of N), while one digit fewer on A or s + t <= 4 does
  not.
"""
import numpy as np
import pytest

from oracle import ctaux
from tests.helpers import problem

BETA = 9


def _digits(M, axis, S):
    """Digits D[s] (integers) and exponents e with M ~= 2^e sum_s D[s] 2^(-9 (s + 1));
    e per row (axis = 1) or per column (axis = 0), |M| 2^-e < 1/2."""
    mx = np.abs(M).max(axis=axis, keepdims=True)
    e = np.where(mx > 0, np.frexp(np.where(mx > 0, mx, 1.0))[1] + 1, 0).astype(np.float64)
    x = M / 2.0 ** e
    D = []
    for _ in range(S):
        y = x * 2.0 ** BETA
        d = np.rint(y)
        D.append(d)
        x = y - d
    return np.array(D), e


def _sliced_residual(A, N0, SA, SB, T, kstep=16):
    DA, ea = _digits(A, 1, SA)
    DB, eb = _digits(N0, 0, SB)
    k = A.shape[0]
    tot = np.zeros_like(A)
    for g in range(T + 1):
        pairs = [(s, g - s) for s in range(SA) if 0 <= g - s < SB]
        if g < 2:
            acc = sum(DA[s] @ DB[t] for s, t in pairs)
        else:
            acc = np.zeros(A.shape, np.float32)
            for k0 in range(0, k, kstep):
                part = sum(DA[s][:, k0:k0 + kstep] @ DB[t][k0:k0 + kstep, :] for s, t in pairs)
                acc = (acc + part.astype(np.float32)).astype(np.float32)
            acc = acc.astype(np.float64)
        tot += acc * 2.0 ** (-BETA * (g + 2))
    return np.eye(k) - tot * 2.0 ** ea * 2.0 ** eb


@pytest.fixture(scope="module")
def config():
    c, eps, kr, G0 = problem(16, 1.0, -0.15, 6.0, 20.0, 2.85, 2048)
    ow = ctaux.OracleWalker(16, c.site_sub, 6.0, 20.0, 1.0, G0, warmup_sweeps=5, n_tau_meas=8, seed=2)
    ow.sweep(60)
    N = ow.state()["N"][0]
    assert N.shape[0] > 200
    rng = np.random.default_rng(0)
    N0 = (N * (1 + 1e-5 * rng.standard_normal(N.shape))).astype(np.float32).astype(np.float64)
    return N, np.linalg.inv(N), N0


def test_digits_are_small_integers_that_rebuild_the_matrix(config):
    N, A, N0 = config
    for M, axis, S, tol in ((A, 1, 5, 2.0 ** -44), (N0, 0, 4, 2.0 ** -35)):
        D, e = _digits(M, axis, S)
        assert np.all(D == np.rint(D)) and np.abs(D).max() <= 2 ** (BETA - 1)
        back = sum(D[s] * 2.0 ** (-BETA * (s + 1)) for s in range(S)) * 2.0 ** e
        scale = np.abs(M).max(axis=axis, keepdims=True)
        assert np.all(np.abs(back - M) <= tol * scale)


def test_exact_groups_fit_fp32_over_a_chunk(config):
    N, A, N0 = config
    DA, _ = _digits(A, 1, 5)
    DB, _ = _digits(N0, 0, 4)
    bound = 0.0
    for k0 in range(0, A.shape[0], 128):
        sl = slice(k0, k0 + 128)
        g0 = np.abs(DA[0][:, sl]) @ np.abs(DB[0][sl, :])
        g1 = np.abs(DA[0][:, sl]) @ np.abs(DB[1][sl, :]) + np.abs(DA[1][:, sl]) @ np.abs(DB[0][sl, :])
        bound = max(bound, g0.max(), g1.max())
    assert bound <= 2.0 ** 24


def test_newton_step_with_the_sliced_residual_reaches_fp32_rounding(config):
    N, A, N0 = config
    scale = np.abs(N).max()

    def newton(R):
        return np.abs((N0 + N0 @ R).astype(np.float32).astype(np.float64) - N).max() / scale

    exact = newton(np.eye(N.shape[0]) - A @ N0)
    assert np.abs(N0 - N).max() / scale > 1e-6  # the drift the step removes
    sliced = newton(_sliced_residual(A, N0, 5, 4, 5))
    assert sliced <= 2.0 * exact, (sliced, exact)
    # one digit fewer on A, or the pairs with s + t = 5 dropped, leave more
    assert newton(_sliced_residual(A, N0, 4, 4, 5)) > 2.0 * exact
    assert newton(_sliced_residual(A, N0, 5, 4, 4)) > 2.0 * exact
