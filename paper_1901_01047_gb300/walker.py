"""Thin ctypes binding of the C ABI in ``include/dca_walker.h``.

Argument marshalling only: every step of a sweep runs in the CUDA kernels of
``libdcawalker.so``.  If the library has not been built, ``load()`` raises;
there is no fallback path.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdcawalker.so")

DCA_OK = 0
ERRORS = {-1: "ARG", -2: "CUDA", -3: "OOM", -4: "TIMEOUT", -5: "NUMERIC", -6: "STATE", -7: "CAPACITY"}
PRECISIONS = {"fp64": 0, "mixed": 1, "tf32x3": 1, "tf32": 2}
GAMMA_PRECISIONS = {"fp64": 0, "double_float": 1}

EXPORTS = [
    "dca_g0_isolated_cluster", "dca_walker_create", "dca_walker_sweep", "dca_walker_measure_G",
    "dca_walker_reset_measurements", "dca_walker_stats", "dca_walker_get_state",
    "dca_walker_get_decision_log", "dca_walker_set_forced_decisions", "dca_walker_capacity",
    "dca_walker_destroy", "dca_walker_last_error", "dca_walker_update_G0", "dca_walker_set_timing",
    "dca_walker_get_timing", "dca_walker_set_tuning", "dca_fresh_N", "dca_fresh_N_noalloc",
    "dca_walker_sync", "dca_walker_set_schedule", "dca_walker_set_limits", "dca_walker_save", "dca_walker_load",
    "dca_walker_measure_M", "dca_coarse_grain", "dca_sigma_update", "dca_g0_table_from_freq",
    "dca_walker_set_recompute", "dca_walker_measure_G4", "dca_g4_assemble", "dca_walker_update_G0_all",
    "dca_walker_set_update_tile",
]
UPDATE_KERNELS = {"auto": 0, "cuda_core": 1, "tcgen05": 2}
# lockstep: every walker runs n more sweeps per sweep(n); pooled: the walkers
# together run n * n_walkers more sweeps, all of them in every window
SCHEDULES = {"lockstep": 0, "pooled": 1}
GROUPS = ["propose", "extend", "metropolis", "update", "measure", "recompute", "update_pre", "update_post",
          "recompute_pre", "recompute_post"]


class Problem(C.Structure):
    _fields_ = [
        ("nc", C.c_int32),
        ("site_sub", C.POINTER(C.c_int32)),
        ("U", C.c_double),
        ("beta", C.c_double),
        ("K", C.c_double),
        ("n_tau", C.c_int32),
        ("G0", C.POINTER(C.c_double)),
        ("k_dot_r", C.POINTER(C.c_double)),
        ("k_sub", C.POINTER(C.c_int32)),
    ]


class Params(C.Structure):
    _fields_ = [
        ("n_problems", C.c_int32),
        ("problems", C.POINTER(Problem)),
        ("n_walkers", C.c_int32),
        ("walker_problem", C.POINTER(C.c_int32)),
        ("k_sub", C.c_int32),
        ("recompute_every", C.c_int32),
        ("warmup_sweeps", C.c_int32),
        ("n_tau_meas", C.c_int32),
        ("precision", C.c_int32),
        ("init_config_size", C.c_int32),
        ("capacity", C.c_int32),
        ("seed", C.c_uint64),
        ("tie_eps", C.c_double),
        ("log_capacity", C.c_int64),
        ("update_kernel", C.c_int32),
        ("recompute_sweeps", C.c_int32),
        ("recompute_method", C.c_int32),
        ("schedule", C.c_int32),
        ("gamma_precision", C.c_int32),
        ("recompute_at_measure", C.c_int32),
        ("n_omega_meas", C.c_int32),
        ("flip_fraction", C.c_double),
        ("duplicate_rule", C.c_int32),
        ("freq_method", C.c_int32),
        ("n_w4", C.c_int32),
        ("w4_transfer", C.c_int32),
        ("q4_transfer", C.c_int32),
    ]


class Lattice(C.Structure):
    _fields_ = [
        ("nc", C.c_int32),
        ("kpts", C.POINTER(C.c_double)),
        ("k_dot_r", C.POINTER(C.c_double)),
        ("recip", C.c_double * 4),
        ("t", C.c_double),
        ("tp", C.c_double),
        ("mu", C.c_double),
        ("U", C.c_double),
        ("beta", C.c_double),
        ("n_fine", C.c_int32),
    ]


class Vertex(C.Structure):
    _fields_ = [("site", C.c_int32), ("s", C.c_int32), ("tau", C.c_double)]


class Stats(C.Structure):
    _fields_ = [
        ("proposals", C.c_int64),
        ("accepts", C.c_int64),
        ("near_ties", C.c_int64),
        ("aborts", C.c_int64),
        ("windows", C.c_int64),
        ("sweeps", C.c_int64),
        ("measurements", C.c_int64),
        ("recomputes", C.c_int64),
        ("sweep_length", C.c_int64),
        ("order", C.c_int32),
        ("status", C.c_int32),
        ("sign", C.c_double),
        ("k_sum", C.c_double),
        ("max_drift", C.c_double),
        ("n_update_flops", C.c_double),
        ("n_update_bytes", C.c_double),
        ("extend_flops", C.c_double),
        ("extend_bytes", C.c_double),
        ("recompute_flops", C.c_double),
        ("neglected", C.c_int64),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load(path=LIB_PATH):
    """Load libdcawalker.so; raise if it is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libdcawalker.so is not built (%s); run __graft_entry__.build()" % path)
    L = C.CDLL(path)
    P = C.c_void_p
    L.dca_g0_isolated_cluster.argtypes = [C.c_int32, P, P, C.c_double, C.c_double, C.c_double, C.c_int32, P]
    L.dca_walker_create.argtypes = [C.POINTER(Params), P, C.POINTER(P)]
    L.dca_walker_sweep.argtypes = [P, C.c_int32]
    L.dca_walker_sync.argtypes = [P]
    L.dca_walker_set_schedule.argtypes = [P, C.c_int32]
    L.dca_walker_set_limits.argtypes = [P, C.c_int64, C.c_int64]
    L.dca_walker_set_recompute.argtypes = [P, C.c_int32, C.c_int32, C.c_int32]
    L.dca_walker_save.argtypes = [P, P, C.c_size_t, C.POINTER(C.c_size_t)]
    L.dca_walker_load.argtypes = [P, P, C.c_size_t]
    L.dca_walker_measure_G.argtypes = [P, P, P, P]
    L.dca_walker_measure_M.argtypes = [P, P, P, P]
    L.dca_walker_measure_G4.argtypes = [P, P, P, P, P]
    L.dca_g4_assemble.argtypes = [C.c_int32, P, P, C.c_double, P, P, P]
    L.dca_walker_reset_measurements.argtypes = [P]
    L.dca_walker_stats.argtypes = [P, P]
    L.dca_walker_get_state.argtypes = [P, C.c_int32, P, C.POINTER(C.c_int32), P, P]
    L.dca_walker_get_decision_log.argtypes = [P, C.c_int32, P, C.c_int64, C.POINTER(C.c_int64)]
    L.dca_walker_set_forced_decisions.argtypes = [P, C.c_int32, P, C.c_int64]
    L.dca_walker_capacity.argtypes = [P, C.c_int32, C.POINTER(C.c_int32)]
    L.dca_walker_update_G0.argtypes = [P, C.c_int32, P]
    L.dca_walker_update_G0_all.argtypes = [P, P]
    L.dca_walker_set_update_tile.argtypes = [P, C.c_int32]
    L.dca_walker_set_timing.argtypes = [P, C.c_uint32]
    L.dca_walker_set_tuning.argtypes = [P, C.c_int32, C.c_int32]
    L.dca_walker_get_timing.argtypes = [P, P, P, C.POINTER(C.c_int64), C.c_int32]
    L.dca_fresh_N.argtypes = [C.POINTER(Problem), C.c_int32, P, P, P, C.POINTER(C.c_int32)]
    L.dca_fresh_N_noalloc.argtypes = [C.POINTER(Problem), C.c_int32, P, P, P, C.POINTER(C.c_int32)]
    L.dca_coarse_grain.argtypes = [C.POINTER(Lattice), C.c_int32, P, P, P, P, P]
    L.dca_sigma_update.argtypes = [C.POINTER(Lattice), C.c_int32, P, C.c_int32, P, P, P, C.c_double, P]
    L.dca_g0_table_from_freq.argtypes = [C.POINTER(Lattice), C.c_int32, P, P, C.c_int32, P]
    L.dca_walker_destroy.argtypes = [P]
    L.dca_walker_destroy.restype = None
    L.dca_walker_last_error.argtypes = [P]
    L.dca_walker_last_error.restype = C.c_char_p
    _lib = L
    return L


class WalkerError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


def _ptr(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def g0_isolated_cluster(eps_K, k_dot_r, mu, U, beta, n_tau):
    """G0[2][nc][n_tau+1] (paper convention) of an isolated cluster, built on the GPU."""
    L = load()
    eps = np.ascontiguousarray(eps_K, np.float64)
    kr = np.ascontiguousarray(k_dot_r, np.float64)
    nc = eps.size
    out = np.zeros((2, nc, n_tau + 1), np.float64)
    rc = L.dca_g0_isolated_cluster(nc, _ptr(eps), _ptr(kr), float(mu), float(U), float(beta), int(n_tau),
                                   _ptr(out))
    if rc != DCA_OK:
        raise WalkerError(rc, L.dca_walker_last_error(None).decode())
    return out


def _problem_struct(pr, keep):
    ss = np.ascontiguousarray(pr["site_sub"], np.int32).reshape(-1)
    g0 = np.ascontiguousarray(pr["G0"], np.float64)
    keep += [ss, g0]
    p = Problem()
    p.nc = int(pr["nc"])
    p.site_sub = ss.ctypes.data_as(C.POINTER(C.c_int32))
    p.U = float(pr["U"])
    p.beta = float(pr["beta"])
    p.K = float(pr.get("K", 1.0))
    p.n_tau = int(g0.shape[-1] - 1)
    p.G0 = g0.ctypes.data_as(C.POINTER(C.c_double))
    return p


def g4_assemble(A, D, sign_sum, G0_up, G0_dn):
    """G2 [S, S] (complex) from one set of two-particle accumulators and the bare
    propagator at the measured points (dca_g4_assemble, on the GPU)."""
    L = load()
    S = A.shape[0]
    a = np.ascontiguousarray(np.stack([A.real, A.imag], -1), np.float64)
    d = np.ascontiguousarray(np.stack([D.real, D.imag], -1), np.float64)
    gu = np.ascontiguousarray(np.stack([np.real(G0_up), np.imag(G0_up)], -1), np.float64)
    gd = np.ascontiguousarray(np.stack([np.real(G0_dn), np.imag(G0_dn)], -1), np.float64)
    out = np.zeros((S, S, 2), np.float64)
    rc = L.dca_g4_assemble(int(S), _ptr(a), _ptr(d), float(sign_sum), _ptr(gu), _ptr(gd), _ptr(out))
    if rc != DCA_OK:
        raise WalkerError(rc, L.dca_walker_last_error(None).decode())
    return out[..., 0] + 1j * out[..., 1]


def _vertices(site, tau, s):
    n = len(site)
    verts = (Vertex * max(n, 1))()
    for i in range(n):
        verts[i].site = int(site[i])
        verts[i].s = int(s[i])
        verts[i].tau = float(tau[i])
    return verts


def fresh_N(problem, site, tau, s, fn="dca_fresh_N"):
    """(N_up, N_dn, det_sign) from scratch for an all-interacting vertex list."""
    L = load()
    keep = []
    pr = _problem_struct(problem, keep)
    n = len(site)
    verts = _vertices(site, tau, s)
    Nu = np.zeros((n, n), np.float64)
    Nd = np.zeros((n, n), np.float64)
    sg = C.c_int32(0)
    rc = getattr(L, fn)(C.byref(pr), n, verts, _ptr(Nu), _ptr(Nd), C.byref(sg))
    if rc != DCA_OK:
        raise WalkerError(rc, L.dca_walker_last_error(None).decode())
    return Nu, Nd, int(sg.value)


class Walkers:
    """A batch of CT-AUX walkers living on the GPU.

    problems: list of dicts with keys nc, site_sub [nc,nc], U, beta, K, G0 [2,nc,n_tau+1].
    """

    def __init__(self, problems, n_walkers=1, walker_problem=None, k_sub=32, recompute_every=64,
                 warmup_sweeps=20, n_tau_meas=64, precision="fp64", init_config_size=10, capacity=0,
                 seed=0, tie_eps=1e-10, log_capacity=0, update_kernel="auto", recompute_sweeps=0,
                 recompute_method="auto", schedule="lockstep", gamma_precision="fp64", recompute_at_measure=False,
                 n_omega_meas=0, flip_fraction=0.0, duplicate_rule="abort", freq_method="nfft", n_w4=0,
                 w4_transfer=0, q4_transfer=0, stream=None):
        L = load()
        self._keep = []
        probs = (Problem * len(problems))()
        self.nc = []
        for i, pr in enumerate(problems):
            ss = np.ascontiguousarray(pr["site_sub"], np.int32).reshape(-1)
            g0 = np.ascontiguousarray(pr["G0"], np.float64)
            self._keep += [ss, g0]
            probs[i].nc = int(pr["nc"])
            probs[i].site_sub = ss.ctypes.data_as(C.POINTER(C.c_int32))
            probs[i].U = float(pr["U"])
            probs[i].beta = float(pr["beta"])
            probs[i].K = float(pr.get("K", 1.0))
            probs[i].n_tau = int(g0.shape[-1] - 1)
            probs[i].G0 = g0.ctypes.data_as(C.POINTER(C.c_double))
            if pr.get("k_dot_r") is not None:
                kr = np.ascontiguousarray(pr["k_dot_r"], np.float64).reshape(-1)
                ks = np.ascontiguousarray(pr["k_sub"], np.int32).reshape(-1)
                self._keep += [kr, ks]
                probs[i].k_dot_r = kr.ctypes.data_as(C.POINTER(C.c_double))
                probs[i].k_sub = ks.ctypes.data_as(C.POINTER(C.c_int32))
        p = Params()
        p.n_problems = len(problems)
        p.problems = probs
        p.n_walkers = int(n_walkers)
        if walker_problem is not None:
            wp = np.ascontiguousarray(walker_problem, np.int32)
            self._keep.append(wp)
            p.walker_problem = wp.ctypes.data_as(C.POINTER(C.c_int32))
            self.walker_problem = wp
        else:
            self.walker_problem = np.arange(n_walkers, dtype=np.int32) % len(problems)
        self.nc = [int(problems[i]["nc"]) for i in self.walker_problem]
        p.k_sub = int(k_sub)
        self.k_sub = int(k_sub)
        p.recompute_every = int(recompute_every)
        p.warmup_sweeps = int(warmup_sweeps)
        p.n_tau_meas = int(n_tau_meas)
        p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        p.init_config_size = int(init_config_size)
        p.capacity = int(capacity)
        p.seed = int(seed)
        p.tie_eps = float(tie_eps)
        p.log_capacity = int(log_capacity)
        p.recompute_sweeps = int(recompute_sweeps)
        p.recompute_method = {"auto": 0, "gj": 1, "newton_df": 2}[recompute_method]
        p.schedule = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
        p.gamma_precision = GAMMA_PRECISIONS[gamma_precision] if isinstance(gamma_precision, str) \
            else int(gamma_precision)
        p.recompute_at_measure = 1 if recompute_at_measure else 0
        p.n_omega_meas = int(n_omega_meas)
        p.flip_fraction = float(flip_fraction)
        p.freq_method = {"nfft": 0, "dft": 1}[freq_method] if isinstance(freq_method, str) else int(freq_method)
        p.duplicate_rule = {"abort": 0, "neglect": 1, "update": 2}[duplicate_rule] if isinstance(duplicate_rule, str) \
            else int(duplicate_rule)
        self.n_omega_meas = int(n_omega_meas)
        p.n_w4 = int(n_w4)
        p.w4_transfer = int(w4_transfer)
        p.q4_transfer = int(q4_transfer)
        self.n_w4 = int(n_w4)
        p.update_kernel = UPDATE_KERNELS[update_kernel] if isinstance(update_kernel, str) else int(update_kernel)
        self.n_walkers = int(n_walkers)
        self.n_tau_meas = int(n_tau_meas)
        h = C.c_void_p()
        st = C.c_void_p(int(stream)) if stream else None
        rc = L.dca_walker_create(C.byref(p), st, C.byref(h))
        if rc != DCA_OK:
            raise WalkerError(rc, L.dca_walker_last_error(None).decode())
        self._h = h
        self._L = L

    def _check(self, rc):
        if rc != DCA_OK:
            raise WalkerError(rc, self._L.dca_walker_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.dca_walker_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n, sync=True):
        """Run n more sweeps (see dca_walker_sweep).  The library call only
        enqueues them; with sync=True the binding then calls dca_walker_sync,
        so that a walker error raises here."""
        self._check(self._L.dca_walker_sweep(self._h, int(n)))
        if sync:
            self.sync()

    def sync(self):
        self._check(self._L.dca_walker_sync(self._h))

    def set_schedule(self, schedule):
        s = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
        self._check(self._L.dca_walker_set_schedule(self._h, s))

    def set_recompute(self, recompute_every=0, recompute_sweeps=0, recompute_at_measure=False):
        """Change the recompute schedule between sweeps (same chains)."""
        self._check(self._L.dca_walker_set_recompute(self._h, int(recompute_every), int(recompute_sweeps),
                                                     1 if recompute_at_measure else 0))

    def set_limits(self, max_windows=0, wait_cycles=0):
        self._check(self._L.dca_walker_set_limits(self._h, int(max_windows), int(wait_cycles)))

    def save(self):
        """Checkpoint of every walker's chain as bytes."""
        n = C.c_size_t(0)
        self._check(self._L.dca_walker_save(self._h, None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(self._L.dca_walker_save(self._h, buf, n.value, C.byref(n)))
        return buf.raw[:n.value]

    def load(self, data):
        buf = C.create_string_buffer(bytes(data), len(data))
        self._check(self._L.dca_walker_load(self._h, buf, len(data)))

    def measure_G(self):
        """(G_sum list per walker [2, nc, n_tau_meas], sign sums, measurement counts)."""
        total = sum(2 * nc * self.n_tau_meas for nc in self.nc)
        g = np.zeros(total, np.float64)
        ss = np.zeros(self.n_walkers, np.float64)
        nm = np.zeros(self.n_walkers, np.int64)
        self._check(self._L.dca_walker_measure_G(self._h, _ptr(g), _ptr(ss), _ptr(nm)))
        out, off = [], 0
        for nc in self.nc:
            m = 2 * nc * self.n_tau_meas
            out.append(g[off:off + m].reshape(2, nc, self.n_tau_meas))
            off += m
        return out, ss, nm

    def measure_M(self):
        """(sum of sign * M(dr, i w_n) per walker as complex [2, nc, n_omega], sign sums, counts)."""
        total = sum(2 * nc * self.n_omega_meas * 2 for nc in self.nc)
        m = np.zeros(max(total, 1), np.float64)
        ss = np.zeros(self.n_walkers, np.float64)
        nm = np.zeros(self.n_walkers, np.int64)
        self._check(self._L.dca_walker_measure_M(self._h, _ptr(m), _ptr(ss), _ptr(nm)))
        out, off = [], 0
        for nc in self.nc:
            k = 2 * nc * self.n_omega_meas * 2
            a = m[off:off + k].reshape(2, nc, self.n_omega_meas, 2)
            out.append(a[..., 0] + 1j * a[..., 1])
            off += k
        return out, ss, nm

    def measure_G4(self):
        """Two-particle accumulators per walker: (A complex [S, S], D complex [2, S]) with
        S = nc * 2 n_w4, the sign sums and the measurement counts."""
        sizes = [nc * 2 * self.n_w4 for nc in self.nc]
        A = np.zeros(max(sum(2 * S * S for S in sizes), 1), np.float64)
        D = np.zeros(max(sum(4 * S for S in sizes), 1), np.float64)
        ss = np.zeros(self.n_walkers, np.float64)
        nm = np.zeros(self.n_walkers, np.int64)
        self._check(self._L.dca_walker_measure_G4(self._h, _ptr(A), _ptr(D), _ptr(ss), _ptr(nm)))
        out, oa, od = [], 0, 0
        for S in sizes:
            a = A[oa:oa + 2 * S * S].reshape(S, S, 2)
            d = D[od:od + 4 * S].reshape(2, S, 2)
            out.append((a[..., 0] + 1j * a[..., 1], d[..., 0] + 1j * d[..., 1]))
            oa += 2 * S * S
            od += 4 * S
        return out, ss, nm

    def reset_measurements(self):
        self._check(self._L.dca_walker_reset_measurements(self._h))

    def stats(self):
        arr = (Stats * self.n_walkers)()
        self._check(self._L.dca_walker_stats(self._h, arr))
        return [s.as_dict() for s in arr]

    def capacity(self, wi=0):
        c = C.c_int32(0)
        self._check(self._L.dca_walker_capacity(self._h, int(wi), C.byref(c)))
        return c.value

    def state(self, wi=0):
        cap = self.capacity(wi)
        verts = (Vertex * cap)()
        k = C.c_int32(0)
        self._check(self._L.dca_walker_get_state(self._h, int(wi), verts, C.byref(k), None, None))
        n = k.value
        Nu = np.zeros((n, n), np.float64)
        Nd = np.zeros((n, n), np.float64)
        self._check(self._L.dca_walker_get_state(self._h, int(wi), None, C.byref(k), _ptr(Nu), _ptr(Nd)))
        site = np.array([verts[i].site for i in range(n)], np.int32)
        s = np.array([verts[i].s for i in range(n)], np.int8)
        tau = np.array([verts[i].tau for i in range(n)], np.float64)
        return dict(site=site, tau=tau, s=s, N=(Nu, Nd))

    def decision_log(self, wi=0):
        n = C.c_int64(0)
        self._check(self._L.dca_walker_get_decision_log(self._h, int(wi), None, 0, C.byref(n)))
        out = np.zeros(max(n.value, 1), np.uint8)
        self._check(self._L.dca_walker_get_decision_log(self._h, int(wi), _ptr(out), out.size, C.byref(n)))
        return out[:n.value]

    def update_G0(self, problem, G0):
        """Upload a new bare propagator (host array, paper convention) for a problem."""
        G0 = np.ascontiguousarray(G0, np.float64)
        self._check(self._L.dca_walker_update_G0(self._h, int(problem), _ptr(G0)))

    def update_G0_all(self, G0_all):
        """Upload every problem's bare propagator at once: a 1-D float64 array holding the
        tables back to back in problem order (pinned memory makes the copy asynchronous;
        keep it unchanged until the stream has passed the copy), or a list of per-problem
        tables."""
        if isinstance(G0_all, (list, tuple)):
            G0_all = np.concatenate([np.ascontiguousarray(g, np.float64).reshape(-1) for g in G0_all])
        G0_all = np.ascontiguousarray(G0_all, np.float64)
        self._check(self._L.dca_walker_update_G0_all(self._h, _ptr(G0_all)))

    def set_update_tile(self, tile_n):
        """Column tile of the tensor-core N update: 32, 64 or 0 (default 64; 32 when k_s > 64)."""
        self._check(self._L.dca_walker_set_update_tile(self._h, int(tile_n)))
        self.update_tile = int(tile_n)

    def set_tuning(self, k_sub, update_kernel="auto"):
        """Change the submatrix size and the N-update kernel between sweeps (same Markov chain)."""
        uk = UPDATE_KERNELS[update_kernel] if isinstance(update_kernel, str) else int(update_kernel)
        self._check(self._L.dca_walker_set_tuning(self._h, int(k_sub), uk))
        self.k_sub = int(k_sub)

    def set_timing(self, groups):
        """Time the named kernel groups with CUDA events on the walker's stream."""
        mask = 0
        for g in groups:
            mask |= 1 << GROUPS.index(g)
        self._check(self._L.dca_walker_set_timing(self._h, mask))

    def timing(self, reset=False):
        """{group: (ms, launches)} and the total number of library kernel launches."""
        ms = np.zeros(len(GROUPS), np.float64)
        ln = np.zeros(len(GROUPS), np.int64)
        tot = C.c_int64(0)
        self._check(self._L.dca_walker_get_timing(self._h, _ptr(ms), _ptr(ln), C.byref(tot), 1 if reset else 0))
        return {g: (float(ms[i]), int(ln[i])) for i, g in enumerate(GROUPS)}, int(tot.value)

    def set_forced_decisions(self, wi, log):
        log = np.ascontiguousarray(log, np.uint8)
        self._check(self._L.dca_walker_set_forced_decisions(self._h, int(wi), _ptr(log), int(log.size)))


# ---------------------------------------------------------------------------
# Outer DCA loop (marshalling of the three C calls)
# ---------------------------------------------------------------------------
def _lattice(nc, kpts, k_dot_r, recip, t, tp, mu, U, beta, n_fine, keep):
    kp = np.ascontiguousarray(kpts, np.float64)
    kr = np.ascontiguousarray(k_dot_r, np.float64)
    rc = np.ascontiguousarray(recip, np.float64).reshape(-1)
    keep += [kp, kr]
    lat = Lattice()
    lat.nc = int(nc)
    lat.kpts = kp.ctypes.data_as(C.POINTER(C.c_double))
    lat.k_dot_r = kr.ctypes.data_as(C.POINTER(C.c_double))
    for i in range(4):
        lat.recip[i] = float(rc[i])
    lat.t, lat.tp, lat.mu, lat.U, lat.beta = float(t), float(tp), float(mu), float(U), float(beta)
    lat.n_fine = int(n_fine)
    return lat


def _c2(a):
    a = np.ascontiguousarray(a, np.complex128)
    return np.ascontiguousarray(np.stack([a.real, a.imag], axis=-1))


def _from2(a):
    return a[..., 0] + 1j * a[..., 1]


class DCALoop:
    """The outer DCA loop on the GPU for one cluster (dca_coarse_grain,
    dca_sigma_update, dca_g0_table_from_freq)."""

    def __init__(self, nc, kpts, k_dot_r, recip, t, tp, mu, U, beta, n_fine, n_omega):
        self._keep = []
        self.lat = _lattice(nc, kpts, k_dot_r, recip, t, tp, mu, U, beta, n_fine, self._keep)
        self.nc, self.n_omega = int(nc), int(n_omega)
        self._L = load()

    def _check(self, rc):
        if rc != DCA_OK:
            raise WalkerError(rc, self._L.dca_walker_last_error(None).decode())

    def coarse_grain(self, sigma):
        """(Gbar, calG0, calG0', xi') from the cluster self-energy [nc, n_omega] (complex)."""
        sig = _c2(sigma)
        shp = (self.nc, self.n_omega, 2)
        gb, g0, g0s = np.zeros(shp), np.zeros(shp), np.zeros(shp)
        xi = np.zeros(self.nc)
        self._check(self._L.dca_coarse_grain(C.byref(self.lat), self.n_omega, _ptr(sig), _ptr(gb), _ptr(g0),
                                             _ptr(g0s), _ptr(xi)))
        return _from2(gb), _from2(g0), _from2(g0s), xi

    def sigma_update(self, G0w_shifted, M_sets, sign_sums, sigma_old, alpha):
        """New Sigma from the walkers' accumulators M_sets [n_sets, 2, nc, n_omega] (complex)."""
        g0s = _c2(G0w_shifted)
        m = _c2(np.asarray(M_sets))
        ss = np.ascontiguousarray(sign_sums, np.float64)
        old = _c2(sigma_old)
        out = np.zeros((self.nc, self.n_omega, 2))
        self._check(self._L.dca_sigma_update(C.byref(self.lat), self.n_omega, _ptr(g0s), int(ss.size), _ptr(m),
                                             _ptr(ss), _ptr(old), float(alpha), _ptr(out)))
        return _from2(out)

    def g0_table(self, G0w_shifted, xi, n_tau):
        g0s = _c2(G0w_shifted)
        x = np.ascontiguousarray(xi, np.float64)
        out = np.zeros((2, self.nc, n_tau + 1))
        self._check(self._L.dca_g0_table_from_freq(C.byref(self.lat), self.n_omega, _ptr(g0s), _ptr(x), int(n_tau),
                                                   _ptr(out)))
        return out
