"""ctypes wrapper around the oracle's C CT-AUX walker (test infrastructure only).

The C code (``ctaux_oracle.c``) follows Sec. 2.3 of the DCA++ paper: the
expansion of Z with the constant K, the auxiliary-spin decoupling, the weight
(K / 2 beta Nc)^k prod_sigma det N_sigma^-1 of Eq. Zk, single-spin Metropolis
insert / remove moves as rank-1 updates, sign tracking, and the measurement of
G from M = (e^V - 1) N.  See the C file's header for every reading taken where
the paper is silent.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class _Params(C.Structure):
    _fields_ = [
        ("nc", C.c_int32),
        ("site_sub", C.POINTER(C.c_int32)),
        ("U", C.c_double),
        ("beta", C.c_double),
        ("K", C.c_double),
        ("n_tau", C.c_int32),
        ("G0", C.POINTER(C.c_double)),
        ("warmup_sweeps", C.c_int32),
        ("n_tau_meas", C.c_int32),
        ("seed", C.c_uint64),
        ("walker_id", C.c_uint32),
        ("init_config_size", C.c_int32),
        ("tie_eps", C.c_double),
        ("flip_frac", C.c_double),
        ("neglect_ks", C.c_int32),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        L.orc_g0_interp.argtypes = [C.POINTER(C.c_double), C.c_int32, C.c_double, C.c_double]
        L.orc_g0_interp.restype = C.c_double
        L.orc_create.argtypes = [C.POINTER(_Params), C.POINTER(C.c_int)]
        L.orc_create.restype = P
        L.orc_destroy.argtypes = [P]
        L.orc_sweep.argtypes = [P, C.c_int32]
        L.orc_order.argtypes = [P]
        L.orc_order.restype = C.c_int32
        L.orc_sign.argtypes = [P]
        L.orc_sign.restype = C.c_double
        L.orc_gamma.argtypes = [P]
        L.orc_gamma.restype = C.c_double
        L.orc_get_state.argtypes = [P, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_counters.argtypes = [P, C.POINTER(C.c_int64)]
        L.orc_k_sum.argtypes = [P]
        L.orc_k_sum.restype = C.c_double
        L.orc_get_G.argtypes = [P, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
        L.orc_reset_accumulators.argtypes = [P]
        L.orc_enable_log.argtypes = [P, C.c_int64]
        L.orc_get_log.argtypes = [P, C.c_void_p, C.c_int64]
        L.orc_get_log.restype = C.c_int64
        L.orc_set_hints.argtypes = [P, C.c_void_p, C.c_int64]
        L.orc_sweep_length.argtypes = [P]
        L.orc_sweep_length.restype = C.c_int64
        L.orc_fresh_N.argtypes = [P, C.c_int32, C.c_void_p]
        L.orc_build_A.argtypes = [P, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_set_config.argtypes = [P, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_try_insert.argtypes = [P, C.c_int32, C.c_double, C.c_int8, C.c_int32]
        L.orc_try_remove.argtypes = [P, C.c_int32, C.c_int32]
        L.orc_ratio.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_int8,
                                C.POINTER(C.c_double)]
        L.orc_enable_freq.argtypes = [P, C.c_int32]
        L.orc_try_flip.argtypes = [P, C.c_int32, C.c_int32, C.POINTER(C.c_double)]
        L.orc_neglected.argtypes = [P]
        L.orc_neglected.restype = C.c_int64
        L.orc_get_M.argtypes = [P, C.c_void_p]
        L.orc_enable_g4.argtypes = [P, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]
        L.orc_get_g4.argtypes = [P, C.c_void_p, C.c_void_p]
        L.orc_m2.argtypes = [P, C.c_int32, C.c_void_p]
        _lib = L
    return _lib


def philox4x32_10(counter, key):
    """Philox4x32-10 block: four 32-bit counter words and two key words."""
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in counter])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def g0_interp(row, n_tau, beta, dtau):
    row = np.ascontiguousarray(row, dtype=np.float64)
    return lib().orc_g0_interp(row.ctypes.data_as(C.POINTER(C.c_double)), int(n_tau), float(beta),
                               float(dtau))


def _ptr(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


class OracleWalker:
    """One CT-AUX Markov chain on the CPU (FP64, single-spin updates)."""

    def __init__(self, nc, site_sub, U, beta, K, G0, warmup_sweeps=20, n_tau_meas=64, seed=0,
                 walker_id=0, init_config_size=10, tie_eps=1e-10, flip_frac=0.0, neglect_ks=0):
        self.nc = int(nc)
        self._site_sub = np.ascontiguousarray(site_sub, dtype=np.int32).reshape(-1)
        G0 = np.ascontiguousarray(G0, dtype=np.float64)
        assert G0.ndim == 3 and G0.shape[0] == 2 and G0.shape[1] == self.nc
        self._G0 = G0
        self.n_tau = G0.shape[2] - 1
        self.n_tau_meas = int(n_tau_meas)
        p = _Params()
        p.nc = self.nc
        p.site_sub = self._site_sub.ctypes.data_as(C.POINTER(C.c_int32))
        p.U, p.beta, p.K = float(U), float(beta), float(K)
        p.n_tau = self.n_tau
        p.G0 = self._G0.ctypes.data_as(C.POINTER(C.c_double))
        p.warmup_sweeps = int(warmup_sweeps)
        p.n_tau_meas = self.n_tau_meas
        p.seed = int(seed)
        p.walker_id = int(walker_id)
        p.init_config_size = int(init_config_size)
        p.tie_eps = float(tie_eps)
        p.flip_frac = float(flip_frac)
        p.neglect_ks = int(neglect_ks)
        err = C.c_int(0)
        self._h = lib().orc_create(C.byref(p), C.byref(err))
        if not self._h:
            raise ValueError("oracle create failed with code %d" % err.value)
        self.beta = float(beta)
        self._hints = None

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    # --- running -------------------------------------------------------
    def sweep(self, n):
        rc = lib().orc_sweep(self._h, int(n))
        if rc != 0:
            raise RuntimeError("oracle sweep failed with code %d" % rc)

    def enable_log(self, cap):
        rc = lib().orc_enable_log(self._h, int(cap))
        if rc != 0:
            raise MemoryError("oracle log")

    def log(self):
        n = lib().orc_get_log(self._h, None, 0)
        out = np.zeros(max(n, 1), dtype=np.uint8)
        lib().orc_get_log(self._h, _ptr(out), int(n))
        return out[:n]

    def set_hints(self, hints):
        self._hints = np.ascontiguousarray(hints, dtype=np.uint8)
        lib().orc_set_hints(self._h, _ptr(self._hints), int(self._hints.size))

    # --- state ---------------------------------------------------------
    @property
    def order(self):
        return int(lib().orc_order(self._h))

    @property
    def sign(self):
        return float(lib().orc_sign(self._h))

    @property
    def gamma(self):
        return float(lib().orc_gamma(self._h))

    def state(self):
        k = self.order
        site = np.zeros(k, np.int32)
        tau = np.zeros(k, np.float64)
        s = np.zeros(k, np.int8)
        Nu = np.zeros((k, k), np.float64)
        Nd = np.zeros((k, k), np.float64)
        lib().orc_get_state(self._h, _ptr(site), _ptr(tau), _ptr(s), _ptr(Nu), _ptr(Nd))
        return dict(site=site, tau=tau, s=s, N=(Nu, Nd))

    def counters(self):
        out = (C.c_int64 * 8)()
        lib().orc_counters(self._h, out)
        keys = ["proposals", "accepts", "near_ties", "adopted", "next_q", "sweeps_done", "n_meas",
                "k_samples"]
        d = dict(zip(keys, [int(x) for x in out]))
        d["k_sum"] = float(lib().orc_k_sum(self._h))
        return d

    def G(self):
        """Accumulated sum of sign * G (paper convention), the sign sum, #measurements."""
        g = np.zeros((2, self.nc, self.n_tau_meas), np.float64)
        ss = C.c_double(0)
        nm = C.c_int64(0)
        lib().orc_get_G(self._h, _ptr(g), C.byref(ss), C.byref(nm))
        return g, ss.value, nm.value

    def reset_accumulators(self):
        lib().orc_reset_accumulators(self._h)

    def enable_freq(self, n_omega):
        """Measure M(dr, i w_n) for the first n_omega positive fermionic frequencies as well."""
        rc = lib().orc_enable_freq(self._h, int(n_omega))
        if rc != 0:
            raise ValueError("enable_freq failed with code %d" % rc)
        self.n_omega = int(n_omega)

    def M(self):
        """Accumulated sum of sign * M(dr, i w_n), complex [2, nc, n_omega]."""
        out = np.zeros((2, self.nc, self.n_omega, 2), np.float64)
        rc = lib().orc_get_M(self._h, _ptr(out))
        if rc != 0:
            raise ValueError("frequency measurement is off")
        return out[..., 0] + 1j * out[..., 1]

    def enable_g4(self, n_w4, m4, kdotr, k_dn):
        """Measure the particle-particle up-down two-particle function on the
        points s = (K, n), n = -n_w4 .. n_w4 - 1, with the bosonic transfer
        index m4 and k_dn[K] = index of Q - K (kdotr [nc, nc] = K . r)."""
        self._kdotr = np.ascontiguousarray(kdotr, np.float64)
        self._k_dn = np.ascontiguousarray(k_dn, np.int32)
        rc = lib().orc_enable_g4(self._h, int(n_w4), int(m4), _ptr(self._kdotr), _ptr(self._k_dn))
        if rc != 0:
            raise ValueError("enable_g4 failed with code %d" % rc)
        self.n_w4 = int(n_w4)

    def g4(self):
        """Accumulators (A [S, S], D [2, S]) complex, S = nc * 2 n_w4: A = sum sign
        M_up(s1, s2) M_dn(q - s1, q - s2), D[sigma] = sum sign M_sigma(s, s)."""
        S = self.nc * 2 * self.n_w4
        A = np.zeros((S, S, 2), np.float64)
        D = np.zeros((2, S, 2), np.float64)
        rc = lib().orc_get_g4(self._h, _ptr(A), _ptr(D))
        if rc != 0:
            raise ValueError("two-particle measurement is off or failed (%d)" % rc)
        return A[..., 0] + 1j * A[..., 1], D[..., 0] + 1j * D[..., 1]

    def m2(self, spin):
        """M_sigma(s1, s2) of the current configuration (no sign), complex [S, S]."""
        S = self.nc * 2 * self.n_w4
        out = np.zeros((S, S, 2), np.float64)
        rc = lib().orc_m2(self._h, int(spin), _ptr(out))
        if rc != 0:
            raise ValueError("m2 failed (%d)" % rc)
        return out[..., 0] + 1j * out[..., 1]

    def fresh_N(self, spin):
        k = self.order
        out = np.zeros((k, k), np.float64)
        sg = lib().orc_fresh_N(self._h, int(spin), _ptr(out))
        return out, sg

    def build_A(self, spin, site, tau, s):
        site = np.ascontiguousarray(site, np.int32)
        tau = np.ascontiguousarray(tau, np.float64)
        s = np.ascontiguousarray(s, np.int8)
        n = site.size
        A = np.zeros((n, n), np.float64)
        lib().orc_build_A(self._h, int(spin), int(n), _ptr(site), _ptr(tau), _ptr(s), _ptr(A))
        return A

    def set_config(self, site, tau, s):
        site = np.ascontiguousarray(site, np.int32)
        tau = np.ascontiguousarray(tau, np.float64)
        s = np.ascontiguousarray(s, np.int8)
        rc = lib().orc_set_config(self._h, int(site.size), _ptr(site), _ptr(tau), _ptr(s))
        if rc != 0:
            raise ValueError("set_config failed with code %d" % rc)

    def try_insert(self, site, tau, s, accept=True):
        rc = lib().orc_try_insert(self._h, int(site), float(tau), int(s), 1 if accept else 0)
        if rc != 0:
            raise RuntimeError("try_insert failed %d" % rc)

    def try_remove(self, p, accept=True):
        rc = lib().orc_try_remove(self._h, int(p), 1 if accept else 0)
        if rc != 0:
            raise RuntimeError("try_remove failed %d" % rc)

    def try_flip(self, p, accept=True):
        """Flip the auxiliary spin of vertex p (forced); returns the ratio per spin."""
        out = (C.c_double * 2)()
        rc = lib().orc_try_flip(self._h, int(p), 1 if accept else 0, out)
        if rc != 0:
            raise RuntimeError("try_flip failed %d" % rc)
        return out[0], out[1]

    @property
    def neglected(self):
        return int(lib().orc_neglected(self._h))

    def ratio_insert(self, site, tau, s):
        out = (C.c_double * 2)()
        rc = lib().orc_ratio(self._h, 0, 0, int(site), float(tau), int(s), out)
        assert rc == 0
        return out[0], out[1]

    def ratio_remove(self, p):
        out = (C.c_double * 2)()
        rc = lib().orc_ratio(self._h, 1, int(p), 0, 0.0, 1, out)
        assert rc == 0
        return out[0], out[1]
