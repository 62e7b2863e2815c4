"""GB300 (sm_103a) asynchronous replica-exchange Lennard-Jones molecular dynamics.

A thin ctypes binding of the C ABI in ``include/re.h``; every step of the
method runs in the library's CUDA kernels.  The library must have been built
(``paper_0812_1633_gb300.build.build()``); importing the package does not
build it, and every call fails loudly if the shared library is missing.

Method: G. Bussi, "A simple asynchronous replica-exchange implementation",
arXiv:0812.1633 (Implementation section: exchange protocol; Example section:
LJ liquid, Verlet list, velocity Verlet, stochastic velocity rescaling).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

RE_OK, RE_EINVAL, RE_ECUDA, RE_ENOMEM, RE_ENUMERIC, RE_EOVERFLOW, RE_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
PREC = {"fp64": 0, "mixed": 1}
PATH = {"batched": 0, "plain": 1}


class REError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"re error {code}: {msg}")
        self.code = code


class _Opts(C.Structure):
    _fields_ = [("dt", C.c_double), ("skin", C.c_double), ("tau_T", C.c_double),
                ("shift_energy", C.c_int), ("precision", C.c_int), ("path", C.c_int),
                ("pair_parity", C.c_int), ("nx", C.c_int), ("nbr_capacity", C.c_int),
                ("cell_div", C.c_int), ("cluster", C.c_int), ("atom_threads", C.c_int),
                ("sort_interval", C.c_int), ("exch_distance", C.c_int), ("id_offset", C.c_int),
                ("lists_smem", C.c_int), ("wide_launch", C.c_int), ("group_launch", C.c_int)]


_lib = None


def lib():
    """The loaded shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise ImportError(f"CUDA library not built: {path} (run paper_0812_1633_gb300.build.build())")
        L = C.CDLL(path)
        vp, dp, i32p, i64p, u8p = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32), \
            C.POINTER(C.c_int64), C.POINTER(C.c_uint8)
        L.re_default_opts.argtypes = [C.POINTER(_Opts)]
        L.re_default_opts.restype = None
        L.re_create.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int, dp, C.c_uint64,
                                C.POINTER(_Opts), C.POINTER(vp)]
        L.re_create_h.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int, dp, dp, C.c_uint64,
                                  C.POINTER(_Opts), C.POINTER(vp)]
        L.re_group.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(vp)]
        L.re_advance.argtypes = [vp, i32p]
        L.re_exchange.argtypes = [vp, i32p, u8p]
        L.re_run.argtypes = [vp, C.c_int, i32p, C.c_int]
        L.re_run_record.argtypes = [vp, C.c_int, i32p, C.c_int, i32p, u8p, dp, dp, dp, dp]
        L.re_advance_async.argtypes = [vp, C.c_int]
        L.re_run_async.argtypes = [vp, C.c_int, C.c_int, C.c_int]
        L.re_run_free.argtypes = [vp, C.c_int, C.c_int, C.POINTER(C.c_int64),
                                  C.POINTER(C.c_double), C.POINTER(C.c_int32),
                                  C.POINTER(C.c_uint8)]
        L.re_set_wait_limit.argtypes = [vp, C.c_double]
        L.re_inject_stall.argtypes = [vp, C.c_int, C.c_int]
        L.re_energies.argtypes = [vp, dp, dp, dp]
        L.re_temps.argtypes = [vp, dp]
        L.re_lambdas.argtypes = [vp, dp]
        L.re_config_ex.argtypes = [vp] + [C.POINTER(C.c_int)] * 5
        L.re_config_wide.argtypes = [vp] + [C.POINTER(C.c_int)] * 4
        L.re_config_class.argtypes = [vp, C.c_int] + [C.POINTER(C.c_int)] * 5
        L.re_apply_exchange.argtypes = [vp, dp, dp, dp, dp]
        L.re_get_state.argtypes = [vp, dp, dp]
        L.re_set_state.argtypes = [vp, dp, dp]
        L.re_forces.argtypes = [vp, dp]
        L.re_checkpoint_size.argtypes = [vp, C.POINTER(C.c_size_t)]
        L.re_checkpoint_save.argtypes = [vp, vp, C.c_size_t]
        L.re_checkpoint_load.argtypes = [vp, vp, C.c_size_t]
        L.re_counters.argtypes = [vp, i64p, i64p]
        L.re_accept_stats.argtypes = [vp, i64p, i64p]
        L.re_info.argtypes = [vp, C.POINTER(C.c_int), i64p, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.re_config.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                C.POINTER(C.c_int)]
        L.re_autotune.argtypes = [vp, C.c_int]
        L.re_set_stream.argtypes = [vp, vp]
        L.re_sync.argtypes = [vp]
        L.re_last_error.argtypes = [vp]
        L.re_last_error.restype = C.c_char_p
        L.re_destroy.argtypes = [vp]
        L.re_destroy.restype = None
        L.re_exchange_device.argtypes = [C.c_int, vp, vp, C.c_uint64, C.c_int64, C.c_int, vp, vp,
                                         vp, vp, vp]
        L.re_exchange_device_h.argtypes = [C.c_int, vp, vp, vp, C.c_uint64, C.c_int64, C.c_int,
                                           C.c_int, vp, vp, vp, vp, vp, vp, vp]
        L.re_lj_forces_device.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, vp,
                                          vp, vp, vp]
        L.re_lj_forces_device_noalloc.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int, vp, vp,
                                                  vp, vp]
        _lib = L
    return _lib


def _check(code, ctx=None):
    if code != RE_OK:
        msg = lib().re_last_error(ctx)
        raise REError(code, msg.decode() if msg else "")


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def default_opts() -> dict:
    o = _Opts()
    lib().re_default_opts(C.byref(o))
    return {name: getattr(o, name) for name, _ in _Opts._fields_}


class Context:
    """Replica-exchange context: one ensemble (``Context(...)``) or a group of
    ensembles advanced by one launch (``Context.group([...])``)."""

    def __init__(self, N, L, rc, temps, seed, *, dt=0.005, skin=0.5, tau=0.5, shift=True,
                 precision="mixed", path="batched", pair_parity=0, nx=10, nbr_capacity=0,
                 cell_div=0, cluster=0, atom_threads=0, sort_interval=0, lam=None,
                 exch_distance=1, id_offset=0, lists_smem=0, wide_launch=0, group_launch=0,
                 _handle=None):
        self._h = C.c_void_p()
        if _handle is not None:
            self._h = _handle
        else:
            o = _Opts()
            lib().re_default_opts(C.byref(o))
            o.dt, o.skin, o.tau_T = dt, skin, tau
            o.shift_energy = 1 if shift else 0
            o.precision, o.path = PREC[precision], PATH[path]
            o.pair_parity, o.nx, o.nbr_capacity = pair_parity, nx, nbr_capacity
            o.cell_div, o.cluster, o.atom_threads = cell_div, cluster, atom_threads
            o.sort_interval = sort_interval
            o.exch_distance = exch_distance
            o.id_offset = id_offset
            o.lists_smem = lists_smem
            o.wide_launch = wide_launch
            o.group_launch = group_launch
            t = np.ascontiguousarray(temps, dtype=np.float64)
            lp = None
            if lam is not None:
                lam = np.ascontiguousarray(lam, dtype=np.float64)
                lp = _p(lam, C.c_double)
            _check(lib().re_create_h(int(N), float(L), float(rc), len(t), _p(t, C.c_double), lp,
                                     int(seed) & (2**64 - 1), C.byref(o), C.byref(self._h)))
        n_rep, n_ens, n_pairs = C.c_int(), C.c_int(), C.c_int()
        n_atoms = C.c_int64()
        lib().re_info(self._h, C.byref(n_rep), C.byref(n_atoms), C.byref(n_ens), C.byref(n_pairs))
        self.n_rep, self.n_atoms = n_rep.value, n_atoms.value
        self.n_ens, self.n_pairs = n_ens.value, n_pairs.value

    @classmethod
    def group(cls, members):
        arr = (C.c_void_p * len(members))(*[m._h.value for m in members])
        h = C.c_void_p()
        _check(lib().re_group(arr, len(members), C.byref(h)))
        return cls(0, 0, 0, [], 0, _handle=h)

    # -- lifecycle
    def close(self):
        if self._h is not None and self._h.value:
            lib().re_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- hot path
    def advance(self, steps=None):
        if steps is None:
            _check(lib().re_advance(self._h, None), self._h)
            return
        s = np.ascontiguousarray(np.broadcast_to(np.asarray(steps, np.int32), (self.n_rep,)))
        _check(lib().re_advance(self._h, _p(s, C.c_int32)), self._h)

    def advance_async(self, nx):
        """Free-running advance: each ensemble's master (rotating) does nx steps,
        the others stop at their next step boundary after it finishes."""
        _check(lib().re_advance_async(self._h, int(nx)), self._h)

    def run_async(self, cycles, nx, graph=True):
        _check(lib().re_run_async(self._h, int(cycles), int(nx), 1 if graph else 0), self._h)

    def run_free(self, attempts, nx, log=False):
        """The asynchronous scheme in one persistent launch: `attempts` exchange
        attempts per ensemble, the rotating master issuing each after nx of its
        own steps.  With log=True returns per attempt and replica the step
        count, temperature afterwards, partner (-1 none) and acceptance."""
        if not log:
            _check(lib().re_run_free(self._h, int(attempts), int(nx), None, None, None, None),
                   self._h)
            return None
        shape = (int(attempts), self.n_rep)
        st = np.zeros(shape, np.int64)
        T = np.zeros(shape, np.float64)
        pa = np.zeros(shape, np.int32)
        ac = np.zeros(shape, np.uint8)
        code = lib().re_run_free(self._h, int(attempts), int(nx), _p(st, C.c_int64),
                                 _p(T, C.c_double), _p(pa, C.c_int32), _p(ac, C.c_uint8))
        try:
            _check(code, self._h)
        except REError as e:
            if code == RE_ETIMEOUT:
                e.log = (st, T, pa, ac)   # where every replica stopped
            raise
        return st, T, pa, ac

    def set_wait_limit(self, seconds):
        """Limit (seconds) of the bounded device waits of run_free."""
        _check(lib().re_set_wait_limit(self._h, float(seconds)), self._h)

    def inject_stall(self, replica, from_attempt=0):
        """Fault injection for the next run_free call: `replica` stops answering
        at its part in attempt `from_attempt` of that call (-1 cancels)."""
        _check(lib().re_inject_stall(self._h, int(replica), int(from_attempt)), self._h)

    def exchange(self, outputs=False):
        if not outputs:
            _check(lib().re_exchange(self._h, None, None), self._h)
            return None
        partner = np.zeros(self.n_rep, np.int32)
        acc = np.zeros(self.n_rep, np.uint8)
        _check(lib().re_exchange(self._h, _p(partner, C.c_int32), _p(acc, C.c_uint8)), self._h)
        return partner, acc

    def run(self, cycles, steps=None, graph=True):
        sp = None
        if steps is not None:
            s = np.ascontiguousarray(steps, dtype=np.int32).reshape(cycles, self.n_rep)
            sp = _p(s, C.c_int32)
        _check(lib().re_run(self._h, int(cycles), sp, 1 if graph else 0), self._h)

    def run_record(self, cycles, steps=None, graph=False):
        """re_run_record: `cycles` x {advance, exchange} with each cycle's
        budgets copied in and its record copied out (graph: as one CUDA graph,
        kept for the next call of the same length); returns arrays of shape
        (cycles, n_rep): partner, accepted, T, U, K, H."""
        n = int(cycles)
        sp = None
        if steps is not None:
            s = np.ascontiguousarray(steps, dtype=np.int32).reshape(n, self.n_rep)
            sp = _p(s, C.c_int32)
        out = {"partner": np.zeros((n, self.n_rep), np.int32),
               "accepted": np.zeros((n, self.n_rep), np.uint8)}
        for k in ("T", "U", "K", "H"):
            out[k] = np.zeros((n, self.n_rep))
        _check(lib().re_run_record(self._h, n, sp, 1 if graph else 0, _p(out["partner"], C.c_int32),
                                   _p(out["accepted"], C.c_uint8), _p(out["T"], C.c_double),
                                   _p(out["U"], C.c_double), _p(out["K"], C.c_double),
                                   _p(out["H"], C.c_double)), self._h)
        return out

    # -- getters / setters
    def energies(self):
        U, K, H = (np.zeros(self.n_rep) for _ in range(3))
        _check(lib().re_energies(self._h, _p(U, C.c_double), _p(K, C.c_double), _p(H, C.c_double)),
               self._h)
        return U, K, H

    def temps(self):
        T = np.zeros(self.n_rep)
        _check(lib().re_temps(self._h, _p(T, C.c_double)), self._h)
        return T

    def apply_exchange(self, T_new, vscale, lam_new=None, uscale=None):
        """Applies exchange results decided elsewhere (host arrays, n_rep)."""
        f = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
        T_new, vscale, lam_new, uscale = f(T_new), f(vscale), f(lam_new), f(uscale)
        q = lambda a: None if a is None else _p(a, C.c_double)
        _check(lib().re_apply_exchange(self._h, q(T_new), q(lam_new), q(vscale), q(uscale)),
               self._h)

    def lambdas(self):
        lam = np.zeros(self.n_rep)
        _check(lib().re_lambdas(self._h, _p(lam, C.c_double)), self._h)
        return lam

    def get_state(self):
        x = np.zeros((self.n_atoms, 3))
        v = np.zeros((self.n_atoms, 3))
        _check(lib().re_get_state(self._h, _p(x, C.c_double), _p(v, C.c_double)), self._h)
        return x, v

    def set_state(self, x=None, v=None):
        xp = vp = None
        if x is not None:
            x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.n_atoms, 3)
            xp = _p(x, C.c_double)
        if v is not None:
            v = np.ascontiguousarray(v, dtype=np.float64).reshape(self.n_atoms, 3)
            vp = _p(v, C.c_double)
        _check(lib().re_set_state(self._h, xp, vp), self._h)

    def checkpoint(self):
        """Everything the next call reads, as a host byte array (numpy uint8):
        restoring it into a context created with the same arguments continues
        the run bit for bit."""
        n = C.c_size_t(0)
        _check(lib().re_checkpoint_size(self._h, C.byref(n)), self._h)
        buf = np.zeros(n.value, np.uint8)
        _check(lib().re_checkpoint_save(self._h, buf.ctypes.data_as(C.c_void_p), n.value), self._h)
        return buf

    def restore(self, buf):
        """Loads a checkpoint taken from a context of the same shape, seed and
        options (raises REError with RE_EINVAL otherwise)."""
        b = np.ascontiguousarray(np.frombuffer(memoryview(buf), np.uint8))
        _check(lib().re_checkpoint_load(self._h, b.ctypes.data_as(C.c_void_p), b.size), self._h)

    def forces(self):
        f = np.zeros((self.n_atoms, 3))
        _check(lib().re_forces(self._h, _p(f, C.c_double)), self._h)
        return f

    def counters(self):
        s = np.zeros(self.n_rep, np.int64)
        r = np.zeros(self.n_rep, np.int64)
        _check(lib().re_counters(self._h, _p(s, C.c_int64), _p(r, C.c_int64)), self._h)
        return s, r

    def accept_stats(self):
        a = np.zeros(max(self.n_pairs, 1), np.int64)
        b = np.zeros(max(self.n_pairs, 1), np.int64)
        _check(lib().re_accept_stats(self._h, _p(a, C.c_int64), _p(b, C.c_int64)), self._h)
        return a[:self.n_pairs], b[:self.n_pairs]

    def config(self):
        cl, th, cd, at, ls = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
        lib().re_config_ex(self._h, C.byref(cl), C.byref(th), C.byref(cd), C.byref(at),
                           C.byref(ls))
        wn, wc, wt, wa = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        lib().re_config_wide(self._h, C.byref(wn), C.byref(wc), C.byref(wt), C.byref(wa))
        cfg = {"cluster": cl.value, "threads": th.value, "cell_div": cd.value,
               "atom_threads": at.value, "lists_smem": ls.value, "wide_n": wn.value,
               "wide_cluster": wc.value, "wide_threads": wt.value,
               "wide_atom_threads": wa.value}
        classes = []
        for e in range(self.n_ens):
            v = [C.c_int() for _ in range(5)]
            if lib().re_config_class(self._h, e, *[C.byref(x) for x in v]) != RE_OK:
                break
            classes.append(dict(zip(("cluster", "threads", "cell_div", "atom_threads",
                                     "lists_smem"), (x.value for x in v))))
        if classes:
            cfg["classes"] = classes
        return cfg

    def autotune(self, steps=10):
        _check(lib().re_autotune(self._h, int(steps)), self._h)
        return self.config()

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
        handle = getattr(stream, "cuda_stream", stream)
        _check(lib().re_set_stream(self._h, C.c_void_p(handle or 0)), self._h)

    def sync(self):
        _check(lib().re_sync(self._h), self._h)


def exchange_device(T, U, seed, attempt, parity_mode=0, stream=None):
    """One exchange attempt on device tensors T, U (float64, length R, CUDA).

    Returns (T_new, partner, accepted, vscale) as CUDA tensors."""
    import torch
    R = T.numel()
    T_out = torch.empty_like(T)
    partner = torch.empty(R, dtype=torch.int32, device=T.device)
    acc = torch.empty(R, dtype=torch.uint8, device=T.device)
    vs = torch.empty_like(T)
    st = stream if stream is not None else torch.cuda.current_stream(T.device).cuda_stream
    _check(lib().re_exchange_device(R, T.data_ptr(), U.data_ptr(), int(seed) & (2**64 - 1),
                                    int(attempt), int(parity_mode), T_out.data_ptr(),
                                    partner.data_ptr(), acc.data_ptr(), vs.data_ptr(),
                                    C.c_void_p(st)))
    return T_out, partner, acc, vs


def exchange_device_h(T, lam, U, seed, attempt, parity_mode=0, distance=1, stream=None):
    """Generalised exchange on device tensors (lam may be None: all 1).

    Returns (T_new, lam_new, partner, accepted, vscale, uscale) as CUDA tensors."""
    import torch
    R = T.numel()
    T_out = torch.empty_like(T)
    lam_out = torch.empty_like(T)
    partner = torch.empty(R, dtype=torch.int32, device=T.device)
    acc = torch.empty(R, dtype=torch.uint8, device=T.device)
    vs = torch.empty_like(T)
    us = torch.empty_like(T)
    st = stream if stream is not None else torch.cuda.current_stream(T.device).cuda_stream
    _check(lib().re_exchange_device_h(R, T.data_ptr(), None if lam is None else lam.data_ptr(),
                                      U.data_ptr(), int(seed) & (2**64 - 1), int(attempt),
                                      int(parity_mode), int(distance), T_out.data_ptr(),
                                      lam_out.data_ptr(), partner.data_ptr(), acc.data_ptr(),
                                      vs.data_ptr(), us.data_ptr(), C.c_void_p(st)))
    return T_out, lam_out, partner, acc, vs, us


def lj_forces_device(x, L, rc=2.5, shift=True, precision="fp64", stream=None):
    """Forces (N, 3) and potential energy of positions x (N, 3) float64 CUDA tensor."""
    import torch
    N = x.shape[0]
    x = x.contiguous()
    f = torch.empty_like(x)
    U = torch.empty(1, dtype=torch.float64, device=x.device)
    st = stream if stream is not None else torch.cuda.current_stream(x.device).cuda_stream
    _check(lib().re_lj_forces_device(N, float(L), float(rc), 1 if shift else 0, PREC[precision],
                                     x.data_ptr(), f.data_ptr(), U.data_ptr(), C.c_void_p(st)))
    return f, U


def lj_forces_device_noalloc(x, L, rc=2.5, shift=True, stream=None):
    """As lj_forces_device (FP64) with no allocation inside the library: for
    callers that cannot allocate device memory.  The outputs f and U are
    allocated here, by the caller's side (torch); N <= 4096."""
    import torch
    N = x.shape[0]
    x = x.contiguous()
    f = torch.empty_like(x)
    U = torch.empty(1, dtype=torch.float64, device=x.device)
    st = stream if stream is not None else torch.cuda.current_stream(x.device).cuda_stream
    code = lib().re_lj_forces_device_noalloc(N, float(L), float(rc), 1 if shift else 0,
                                             x.data_ptr(), f.data_ptr(), U.data_ptr(),
                                             C.c_void_p(st))
    if code != RE_OK:
        raise REError(code, "re_lj_forces_device_noalloc failed")
    return f, U
