"""Two-particle Green's function of the particle-particle up-down channel
from the walker's accumulators (TEST INFRASTRUCTURE ONLY: only tests/ may
import this module).

Sec. 2.5 (Eq. bse_cluster and the non-interacting G2^{0,pp} after it) defines
G2(K, K', q) with the combined index K = (K, i w_n) and the transfer
q = (Q, i nu_m); the cluster solver provides it.  Per configuration the two
spins are independent and
    G2(K, K', q) = < G_up(K, K') G_dn(q - K, q - K') >,
    G_sigma(k1, k2) = G0_sigma(k1) delta_{k1 k2} - G0_sigma(k1) M_sigma(k1, k2) G0_sigma(k2)
(the paper's sign; M as in the walker's accumulators).  Expanding the
product, with delta = delta_{K K'}:
    G2 <sign> = G0u(K) G0d(q-K) [ delta (<sign> - <sign Mu(K,K)> G0u(K) - <sign Md(q-K,q-K)> G0d(q-K))
                                  + <sign Mu(K,K') Md(q-K,q-K')> G0u(K') G0d(q-K') ].
At U = 0 this is G0u(K) G0d(q - K) delta_{K K'}, the paper's G2^{0,pp}.
"""
import numpy as np


def points(nc, n_w4, m4, k_dn):
    """Measured points: for s = K * 2 n_w4 + (n + n_w4), n = -n_w4 .. n_w4 - 1,
    the spin-up point (K, n) and the spin-down point (k_dn[K], m4 - n - 1),
    as arrays (K_up, n_up, K_dn, n_dn) of length S = nc * 2 n_w4 (n the
    fermionic index, w_n = (2n + 1) pi / beta)."""
    K = np.repeat(np.arange(nc), 2 * n_w4)
    n = np.tile(np.arange(-n_w4, n_w4), nc)
    return K, n, np.asarray(k_dn)[K], m4 - n - 1


def assemble(A, D, sign_sum, G0u, G0d):
    """G2 [S, S] from the accumulators A [S, S], D [2, S] and the sign sum,
    with G0u [S] = G0_up at the spin-up points and G0d [S] = G0_dn at the
    spin-down points (the walker's bare propagator, paper sign)."""
    S = A.shape[0]
    P = G0u * G0d
    G2 = (A * P[None, :]) * P[:, None]
    diag = P * (sign_sum - D[0] * G0u - D[1] * G0d)
    G2[np.arange(S), np.arange(S)] += diag
    return G2 / sign_sum
