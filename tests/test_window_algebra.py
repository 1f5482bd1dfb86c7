"""The algebra behind the submatrix window's handling of a spin changed twice
(Sec. 2.3, "Submatrix updates"; the in-place rule of the walker), on the host.

With the window's vertex list P (positions p, vertex indices P_p, repeats
allowed) and changes a_p, the window matrix is B = I + M diag(a) with
M_pq = delta(P_p, P_q) - G[P_p, P_q].  Checked in numpy on a random
well-conditioned G:

- det B equals det(I + (I - G) U diag(a) U^T), U the selection columns of P,
  also when a vertex appears twice (Sylvester's identity): the window's ratio
  is the single-spin chain's;
- changing a_q to a' changes column q of B by c (B e_q - e_q), c = (a' - a)/a,
  so det B'/det B = 1 + c (1 - (B^-1)_qq) and B'^-1 follows by Sherman-Morrison
  (the kernel's rank-1 correction);
- an entry with a = 0 (a spin inserted and removed again, or flipped back)
  leaves det B and the rows of L B^-1 of the other entries as without it.
"""
import numpy as np


def _setup(seed, n=12):
    rng = np.random.default_rng(seed)
    G = 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)
    return rng, G


def _window(G, P, a):
    M = np.array([[(1.0 if P[p] == P[q] else 0.0) - G[P[p], P[q]] for q in range(len(P))] for p in range(len(P))])
    return np.eye(len(P)) + M * np.asarray(a)[None, :]


def _full(G, P, a):
    n = G.shape[0]
    U = np.zeros((n, len(P)))
    for p, x in enumerate(P):
        U[x, p] = 1.0
    return np.eye(n) + (np.eye(n) - G) @ U @ np.diag(a) @ U.T


def test_window_determinant_is_the_full_one_with_repeated_vertices():
    for seed in range(5):
        rng, G = _setup(seed)
        P = [3, 7, 1, 7, 5, 3]  # vertices 7 and 3 each changed twice
        a = rng.uniform(-0.9, 2.0, len(P))
        assert np.isclose(np.linalg.det(_window(G, P, a)), np.linalg.det(_full(G, P, a)), rtol=1e-12)


def test_column_change_ratio_and_sherman_morrison():
    for seed in range(5):
        rng, G = _setup(seed)
        P = [2, 9, 4, 0, 6]
        a = rng.uniform(0.2, 2.0, len(P))
        B = _window(G, P, a)
        Bi = np.linalg.inv(B)
        for q in range(len(P)):
            a2 = a.copy()
            a2[q] = rng.uniform(-0.9, 2.0)
            c = (a2[q] - a[q]) / a[q]
            B2 = _window(G, P, a2)
            assert np.allclose(B2[:, q] - B[:, q], c * (B[:, q] - np.eye(len(P))[:, q]), atol=1e-14)
            rho = 1.0 + c * (1.0 - Bi[q, q])
            assert np.isclose(np.linalg.det(B2) / np.linalg.det(B), rho, rtol=1e-12)
            e = np.eye(len(P))[:, q]
            Bi2 = Bi - (c / rho) * np.outer(e - Bi[:, q], Bi[q, :])
            assert np.allclose(Bi2, np.linalg.inv(B2), rtol=1e-11, atol=1e-12)


def test_zero_entry_drops_out():
    rng, G = _setup(7)
    P = [5, 1, 8, 1, 2]  # entry 1 (vertex 1) is undone later in the window: a = 0
    a = rng.uniform(0.2, 2.0, len(P))
    a[1] = 0.0
    keep = [0, 2, 3, 4]
    B = _window(G, P, a)
    Bk = _window(G, [P[i] for i in keep], a[keep])
    assert np.isclose(np.linalg.det(B), np.linalg.det(Bk), rtol=1e-12)
    # L = (G[:, P] - delta) diag(a) has a zero column there, and L B^-1 restricted
    # to the other entries is the reduced window's
    n = G.shape[0]
    L = (G[:, P] - np.eye(n)[:, P]) * a[None, :]
    Lk = (G[:, [P[i] for i in keep]] - np.eye(n)[:, [P[i] for i in keep]]) * a[keep][None, :]
    assert np.allclose((L @ np.linalg.inv(B))[:, keep], Lk @ np.linalg.inv(Bk), rtol=1e-11, atol=1e-13)
    assert np.allclose((L @ np.linalg.inv(B))[:, 1], 0.0, atol=1e-14)
