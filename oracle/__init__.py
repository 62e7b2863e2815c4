"""Plain FP64 CPU oracle for asynchronous replica-exchange LJ molecular dynamics.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_0812_1633_gb300``) never imports it and
shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, FP64, ``-O2 -ffp-contract=off``);
this module builds it with gcc and marshals numpy arrays through ctypes.  The
paper is G. Bussi, "A simple asynchronous replica-exchange implementation"
(arXiv:0812.1633): section "Implementation" (exchange protocol) and section
"Example" (LJ liquid, Verlet list, time step, thermostat, temperature ladder).

Parity status: every oracle function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_pins.py`` (library routines, closed forms, brute force,
invariants) except the long-run statistics, which are pinned only
statistically.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

TAG_VEL, TAG_SVR_R1, TAG_SVR_GAM, TAG_EXCH, TAG_PARITY = 1, 2, 3, 4, 5


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, FP64, no contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Rep(C.Structure):
    _fields_ = [
        ("N", C.c_int), ("shift", C.c_int),
        ("L", C.c_double), ("rc", C.c_double), ("skin", C.c_double), ("dt", C.c_double),
        ("tau", C.c_double), ("T", C.c_double),
        ("seed", C.c_uint64), ("stream", C.c_uint64),
        ("step", C.c_int64), ("nrebuild", C.c_int64),
        ("U", C.c_double), ("K", C.c_double), ("econs", C.c_double),
        ("x", C.POINTER(C.c_double)), ("v", C.POINTER(C.c_double)),
        ("f", C.POINTER(C.c_double)), ("xref", C.POINTER(C.c_double)),
        ("pi", C.POINTER(C.c_int)), ("pj", C.POINTER(C.c_int)),
        ("npairs", C.c_int), ("maxpairs", C.c_int),
        ("list_valid", C.c_int), ("status", C.c_int),
        ("lam", C.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            u64p = C.POINTER(C.c_uint64)
            L.orc_philox4x64_10.argtypes = [u64p, u64p, u64p]
            L.orc_uniform4.argtypes = [C.c_uint64] * 5 + [dp]
            L.orc_box_muller.argtypes = [C.c_double, C.c_double, dp, dp]
            L.orc_gamma_mt.argtypes = [C.c_double, C.c_uint64, C.c_uint64, C.c_uint64,
                                       C.c_uint64, C.POINTER(C.c_int)]
            L.orc_gamma_mt.restype = C.c_double
            L.orc_svr_alpha.argtypes = [C.c_double, C.c_double, C.c_int, C.c_double,
                                        C.c_double, C.c_double, dp]
            L.orc_svr_alpha.restype = C.c_double
            L.orc_lj_pair.argtypes = [C.c_double, C.c_double, dp]
            L.orc_lj_pair.restype = C.c_double
            L.orc_lj_shift.argtypes = [C.c_double, C.c_int]
            L.orc_lj_shift.restype = C.c_double
            L.orc_forces_brute.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int, dp, dp]
            L.orc_forces_brute.restype = C.c_double
            ip = C.POINTER(C.c_int)
            L.orc_build_list.argtypes = [C.c_int, C.c_double, C.c_double, dp, C.c_int, ip, ip]
            L.orc_forces_list.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int, dp,
                                          C.c_int, ip, ip, dp]
            L.orc_forces_list.restype = C.c_double
            L.orc_fcc_lattice.argtypes = [C.c_int, C.c_double, dp]
            L.orc_init_velocities.argtypes = [C.c_int, C.c_double, C.c_uint64, C.c_uint64, dp]
            L.orc_kinetic.argtypes = [C.c_int, dp]
            L.orc_kinetic.restype = C.c_double
            rp = C.POINTER(Rep)
            L.orc_init_replica.argtypes = [rp]
            L.orc_refresh.argtypes = [rp]
            L.orc_md_steps.argtypes = [rp, C.c_int]
            L.orc_advance.argtypes = [C.POINTER(rp), C.c_int, C.POINTER(C.c_int32), C.c_int]
            L.orc_exchange.argtypes = [C.c_int, dp, dp, C.c_uint64, C.c_int64, C.c_int,
                                       C.POINTER(C.c_int32), C.POINTER(C.c_uint8), dp]
            L.orc_exchange.restype = C.c_int
            L.orc_apply_exchange.argtypes = [C.POINTER(rp), C.c_int, dp, dp]
            L.orc_exchange_h.argtypes = [C.c_int, dp, dp, dp, C.c_uint64, C.c_int64, C.c_int,
                                         C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_uint8),
                                         dp, dp]
            L.orc_exchange_h.restype = C.c_int
            L.orc_apply_exchange_h.argtypes = [C.POINTER(rp), C.c_int, dp, dp, dp, dp]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


# ----------------------------------------------------------------- primitives
def philox4x64(ctr, key):
    c = (C.c_uint64 * 4)(*[int(v) & (2**64 - 1) for v in ctr])
    k = (C.c_uint64 * 2)(*[int(v) & (2**64 - 1) for v in key])
    o = (C.c_uint64 * 4)()
    lib().orc_philox4x64_10(c, k, o)
    return [int(v) for v in o]


def uniform4(seed, stream, index, tag, sub=0):
    u = np.zeros(4)
    lib().orc_uniform4(seed & (2**64 - 1), stream & (2**64 - 1), index, tag, sub, _dp(u))
    return u


def box_muller(u0, u1):
    g0, g1 = C.c_double(), C.c_double()
    lib().orc_box_muller(u0, u1, C.byref(g0), C.byref(g1))
    return g0.value, g1.value


def gamma_mt(a, seed, stream, index, tag=TAG_SVR_GAM):
    nt = C.c_int()
    g = lib().orc_gamma_mt(a, seed, stream, index, tag, C.byref(nt))
    return g, nt.value


def svr_alpha(K, Kbar, Nf, c, R1, S):
    kn = C.c_double()
    a = lib().orc_svr_alpha(K, Kbar, Nf, c, R1, S, C.byref(kn))
    return a, kn.value


def lj_pair(r2, Uc=0.0):
    fs = C.c_double()
    u = lib().orc_lj_pair(r2, Uc, C.byref(fs))
    return u, fs.value


def lj_shift(rc, shift=1):
    return lib().orc_lj_shift(rc, shift)


def forces_brute(x, L, rc=2.5, shift=1):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    f = np.zeros_like(x)
    U = lib().orc_forces_brute(len(x), L, rc, shift, _dp(x), _dp(f))
    return f, U


def build_list(x, L, rlist, maxpairs=None):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    N = len(x)
    if maxpairs is None:
        maxpairs = N * 120
    pi = np.zeros(maxpairs, np.int32)
    pj = np.zeros(maxpairs, np.int32)
    n = lib().orc_build_list(N, L, rlist, _dp(x), maxpairs, _ip(pi), _ip(pj))
    if n < 0:
        raise RuntimeError("oracle neighbour list overflow")
    return pi[:n].copy(), pj[:n].copy()


def forces_list(x, L, pi, pj, rc=2.5, shift=1):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    f = np.zeros_like(x)
    pi = np.ascontiguousarray(pi, np.int32)
    pj = np.ascontiguousarray(pj, np.int32)
    U = lib().orc_forces_list(len(x), L, rc, shift, _dp(x), len(pi), _ip(pi), _ip(pj), _dp(f))
    return f, U


def fcc_lattice(N, L):
    x = np.zeros((N, 3))
    lib().orc_fcc_lattice(N, L, _dp(x))
    return x


def init_velocities(N, T, seed, stream):
    v = np.zeros((N, 3))
    lib().orc_init_velocities(N, T, seed, stream, _dp(v))
    return v


def exchange(T, U, seed, attempt, parity_mode=0):
    """One exchange attempt; returns (T_new, partner, accepted, vscale, n_accepted)."""
    T = np.array(T, dtype=np.float64)
    U = np.ascontiguousarray(U, dtype=np.float64)
    R = len(T)
    partner = np.zeros(R, np.int32)
    acc = np.zeros(R, np.uint8)
    vs = np.zeros(R)
    n = lib().orc_exchange(R, _dp(T), _dp(U), seed & (2**64 - 1), attempt, parity_mode,
                           partner.ctypes.data_as(C.POINTER(C.c_int32)),
                           acc.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(vs))
    return T, partner, acc, vs, n


def exchange_h(T, lam, U, seed, attempt, parity_mode=0, distance=1):
    """Generalised exchange (parameters (T, lam), pairs at ladder distance d);
    returns (T_new, lam_new, partner, accepted, vscale, uscale, n_accepted)."""
    T = np.array(T, dtype=np.float64)
    lam = np.ones(len(T)) if lam is None else np.array(lam, dtype=np.float64)
    U = np.ascontiguousarray(U, dtype=np.float64)
    R = len(T)
    partner = np.zeros(R, np.int32)
    acc = np.zeros(R, np.uint8)
    vs = np.zeros(R)
    us = np.zeros(R)
    n = lib().orc_exchange_h(R, _dp(T), _dp(lam), _dp(U), seed & (2**64 - 1), attempt,
                             parity_mode, distance,
                             partner.ctypes.data_as(C.POINTER(C.c_int32)),
                             acc.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(vs), _dp(us))
    return T, lam, partner, acc, vs, us, n


# ------------------------------------------------------------------ replicas
class Replica:
    """One LJ replica with numpy-owned arrays, stepped by the C oracle."""

    def __init__(self, N, L, T, seed, stream, rc=2.5, skin=0.5, dt=0.005, tau=0.5,
                 shift=1, x=None, v=None, step=0, maxpairs=None, lam=1.0):
        self.x = np.zeros((N, 3))
        self.v = np.zeros((N, 3))
        self.f = np.zeros((N, 3))
        self.xref = np.zeros((N, 3))
        if maxpairs is None:
            rl = rc + skin
            dens = N / L**3
            maxpairs = int(N * max(64.0, 1.6 * dens * 4.0 / 3.0 * np.pi * rl**3 / 2)) + 64
            maxpairs = min(maxpairs, N * (N - 1) // 2 + 1)
        self.pi = np.zeros(maxpairs, np.int32)
        self.pj = np.zeros(maxpairs, np.int32)
        r = Rep()
        r.N, r.shift = N, shift
        r.L, r.rc, r.skin, r.dt, r.tau, r.T = L, rc, skin, dt, tau, T
        r.seed, r.stream = seed & (2**64 - 1), stream & (2**64 - 1)
        r.step, r.nrebuild = step, 0
        r.U = r.K = r.econs = 0.0
        r.x, r.v, r.f, r.xref = _dp(self.x), _dp(self.v), _dp(self.f), _dp(self.xref)
        r.pi, r.pj = _ip(self.pi), _ip(self.pj)
        r.npairs, r.maxpairs, r.list_valid, r.status = 0, maxpairs, 0, 0
        r.lam = float(lam)
        self.rep = r
        if x is None:
            if lib().orc_init_replica(C.byref(r)) != 0:
                raise RuntimeError("oracle init failed (N must be 4k^3)")
        else:
            self.x[:] = np.asarray(x).reshape(N, 3)
            self.v[:] = np.asarray(v).reshape(N, 3)
            if lib().orc_refresh(C.byref(r)) != 0:
                raise RuntimeError("oracle list overflow")

    def refresh(self):
        if lib().orc_refresh(C.byref(self.rep)) != 0:
            raise RuntimeError("oracle list overflow")

    def steps(self, n):
        if lib().orc_md_steps(C.byref(self.rep), n) != 0:
            raise RuntimeError("oracle list overflow")

    def __getattr__(self, name):
        if name in ("N", "L", "rc", "skin", "dt", "tau", "T", "seed", "stream", "step",
                    "nrebuild", "U", "K", "econs", "npairs", "status", "shift", "lam"):
            return getattr(self.__dict__["rep"], name)
        raise AttributeError(name)

    @property
    def H(self):
        return self.rep.U + self.rep.K + self.rep.econs


class Ensemble:
    """Replicas of one system at different temperatures (one ladder)."""

    def __init__(self, N, L, temps, seed, rc=2.5, skin=0.5, dt=0.005, tau=0.5, shift=1,
                 parity_mode=0, lams=None, distance=1):
        lams = [1.0] * len(temps) if lams is None else lams
        self.reps = [Replica(N, L, float(T), seed, k, rc, skin, dt, tau, shift, lam=lams[k])
                     for k, T in enumerate(temps)]
        self.seed = seed
        self.attempt = 0
        self.parity_mode = parity_mode
        self.distance = distance
        R = len(self.reps)
        self._arr = (C.POINTER(Rep) * R)(*[C.pointer(r.rep) for r in self.reps])

    @classmethod
    def from_state(cls, N, L, temps, seed, x, v, **kw):
        """An ensemble whose replica k starts at positions x[k], velocities v[k]
        (arrays of shape (R, N, 3)) instead of the lattice."""
        ens = cls.__new__(cls)
        rc, skin = kw.get("rc", 2.5), kw.get("skin", 0.5)
        dt, tau, shift = kw.get("dt", 0.005), kw.get("tau", 0.5), kw.get("shift", 1)
        lams = kw.get("lams")
        lams = [1.0] * len(temps) if lams is None else lams
        ens.reps = [Replica(N, L, float(T), seed, k, rc, skin, dt, tau, shift, x=x[k], v=v[k],
                            lam=lams[k])
                    for k, T in enumerate(temps)]
        ens.seed = seed
        ens.attempt = 0
        ens.parity_mode = kw.get("parity_mode", 0)
        ens.distance = kw.get("distance", 1)
        ens._arr = (C.POINTER(Rep) * len(ens.reps))(*[C.pointer(r.rep) for r in ens.reps])
        return ens

    @property
    def R(self):
        return len(self.reps)

    def advance(self, steps, nthreads=0):
        s = np.ascontiguousarray(steps, np.int32)
        if lib().orc_advance(self._arr, self.R, s.ctypes.data_as(C.POINTER(C.c_int32)),
                             nthreads) != 0:
            raise RuntimeError("oracle list overflow")

    def temps(self):
        return np.array([r.T for r in self.reps])

    def energies(self):
        return np.array([r.U for r in self.reps])

    def lams(self):
        return np.array([r.lam for r in self.reps])

    def exchange(self):
        T = self.temps()
        U = self.energies()
        Tn, ln, partner, acc, vs, us, n = exchange_h(T, self.lams(), U, self.seed, self.attempt,
                                                     self.parity_mode, self.distance)
        lib().orc_apply_exchange_h(self._arr, self.R, _dp(Tn), _dp(ln), _dp(vs), _dp(us))
        self.attempt += 1
        return partner, acc
