"""FP64 CPU oracle for the smoothed-cubic random-laser Parallel-Tempering simulation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The product library (``paper_2511_13508_gb300``) never imports, links or executes it,
and the two share no code: this package loads ``liboracle.so`` built from
``pt_oracle.c`` (plain C99, FP64, no FMA contraction) plus the few pure-NumPy helpers
below, each written from the paper (arXiv 2511.13508) section it cites.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pt_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

NBINS = 201
NSTAT = 7   # n, sumE, sumE2, sumY2, sumY4, sumI, sumI2
NQSTAT = 5  # n, sumq, sumq2, sumq3, sumq4


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (FP64, -ffp-contract=off) if missing or stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        c_i64, c_i32, c_u32, c_u64, c_d = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
        vp = ctypes.c_void_p
        L.or_philox4x32_10.argtypes = [P(c_u32), P(c_u32), P(c_u32)]
        L.or_uniform.argtypes = [c_u32]; L.or_uniform.restype = c_d
        L.or_enumerate_quads.argtypes = [ctypes.c_int, vp]; L.or_enumerate_quads.restype = c_i64
        L.or_energy.argtypes = [ctypes.c_int, c_i64, vp, vp, c_d, vp]; L.or_energy.restype = c_d
        L.or_field.argtypes = [ctypes.c_int, c_i64, vp, vp, vp, ctypes.c_int, vp]
        L.or_delta_h.argtypes = [ctypes.c_int, c_i64, vp, vp, c_d, vp, ctypes.c_int, ctypes.c_int, vp, vp]
        L.or_delta_h.restype = c_d
        L.or_cross_terms.argtypes = [ctypes.c_int, c_i64, vp, vp, vp, ctypes.c_int, ctypes.c_int, vp, vp]
        L.or_pair.argtypes = [c_u64, c_u32, c_u32, c_u32, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int)]
        L.or_propose.argtypes = [c_u64, c_u32, c_u32, c_u32, vp, ctypes.c_int, ctypes.c_int, vp, vp]
        L.or_propose.restype = c_d
        L.or_init_config.argtypes = [c_u64, c_u32, ctypes.c_int, vp]
        L.or_sum_abs_pow.argtypes = [ctypes.c_int, vp, ctypes.c_int]; L.or_sum_abs_pow.restype = c_d
        L.or_ipr.argtypes = [ctypes.c_int, vp, ctypes.c_int]; L.or_ipr.restype = c_d
        L.or_overlap.argtypes = [ctypes.c_int, vp, vp]; L.or_overlap.restype = c_d
        L.or_qbin.argtypes = [c_d]; L.or_qbin.restype = ctypes.c_int
        L.or_pt_create.argtypes = [ctypes.c_int, vp, vp, vp, ctypes.c_int, vp, ctypes.c_int, c_u64, c_d,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.or_pt_create.restype = vp
        L.or_pt_create_graph.argtypes = [ctypes.c_int, vp, vp, vp, vp, ctypes.c_int, vp, ctypes.c_int, c_u64, c_d,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.or_pt_create_graph.restype = vp
        L.or_fmc_graph.argtypes = [ctypes.c_int, vp, c_d, vp]; L.or_fmc_graph.restype = c_i64
        L.or_pt_destroy.argtypes = [vp]
        L.or_pt_sweep.argtypes = [vp, c_i64]
        L.or_pt_swap.argtypes = [vp]
        L.or_pt_resync.argtypes = [vp]
        L.or_pt_measure_now.argtypes = [vp]
        L.or_pt_get_state.argtypes = [vp, vp, vp]
        L.or_pt_set_state.argtypes = [vp, vp]
        L.or_pt_get_observables.argtypes = [vp] * 8
        L.or_pt_reset_observables.argtypes = [vp]
        L.or_pt_sweeps_done.argtypes = [vp]; L.or_pt_sweeps_done.restype = c_i64
        _lib = L
    return _lib


def _p(x: np.ndarray):
    return x.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------ single-state functions
def philox(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xffffffff for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def fmc_graph(omega, gamma=None) -> np.ndarray:
    """Random-frequency mode-locked graph by brute force (reading R10): quadruplets in term order,
    [n, 4] int32.  omega sorted ascending; gamma defaults to 1/(2(N-1)) (Eq. (gamma_scaling))."""
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    N = len(omega)
    g = 1.0 / (2 * (N - 1)) if gamma is None else float(gamma)
    n = lib().or_fmc_graph(N, _p(omega), g, None)
    out = np.zeros((max(n, 1), 4), dtype=np.int32)
    lib().or_fmc_graph(N, _p(omega), g, _p(out))
    return out[:n]


def enumerate_quads(N: int) -> np.ndarray:
    n = lib().or_enumerate_quads(int(N), None)
    out = np.zeros((max(n, 1), 4), dtype=np.int32)
    lib().or_enumerate_quads(int(N), _p(out))
    return out[:n]


def energy(N, quads, J, a, cc=2.0) -> float:
    quads = np.ascontiguousarray(quads, dtype=np.int32); J = np.ascontiguousarray(J, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return lib().or_energy(int(N), len(J), _p(quads), _p(J), float(cc), _p(a))


def field(N, quads, J, a, l) -> complex:
    quads = np.ascontiguousarray(quads, dtype=np.int32); J = np.ascontiguousarray(J, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.complex128)
    h = np.zeros(2)
    lib().or_field(int(N), len(J), _p(quads), _p(J), _p(a), int(l), _p(h))
    return complex(h[0], h[1])


def delta_h(N, quads, J, a, j, k, aj_new, ak_new, cc=2.0) -> float:
    quads = np.ascontiguousarray(quads, dtype=np.int32); J = np.ascontiguousarray(J, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.complex128)
    aj = np.array([aj_new.real, aj_new.imag]); ak = np.array([ak_new.real, ak_new.imag])
    return lib().or_delta_h(int(N), len(J), _p(quads), _p(J), float(cc), _p(a), int(j), int(k), _p(aj), _p(ak))


def cross_terms(N, quads, J, a, j, k):
    """(B_jk, A_jk): the bilinear part of the pair-move energy change, -cc Re[conj(dj) dk B + conj(dj) conj(dk) A]."""
    quads = np.ascontiguousarray(quads, dtype=np.int32); J = np.ascontiguousarray(J, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.complex128)
    B = np.zeros(2); A = np.zeros(2)
    lib().or_cross_terms(int(N), len(J), _p(quads), _p(J), _p(a), int(j), int(k), _p(B), _p(A))
    return complex(B[0], B[1]), complex(A[0], A[1])


def pair(seed, sample, sweep, update, N):
    j, k = ctypes.c_int(), ctypes.c_int()
    lib().or_pair(seed, sample, sweep, update, int(N), ctypes.byref(j), ctypes.byref(k))
    return j.value, k.value


def propose(seed, chain, sweep, update, a, j, k):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    aj = np.zeros(2); ak = np.zeros(2)
    U = lib().or_propose(seed, chain, sweep, update, _p(a), int(j), int(k), _p(aj), _p(ak))
    return complex(aj[0], aj[1]), complex(ak[0], ak[1]), U


def init_config(seed, chain, N) -> np.ndarray:
    a = np.zeros(int(N), dtype=np.complex128)
    lib().or_init_config(seed, chain, int(N), _p(a))
    return a


def ipr(a, n) -> float:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return lib().or_ipr(len(a), _p(a), int(n))


def overlap(ac, ad) -> float:
    ac = np.ascontiguousarray(ac, dtype=np.complex128); ad = np.ascontiguousarray(ad, dtype=np.complex128)
    return lib().or_overlap(len(ac), _p(ac), _p(ad))


def qbin(q: float) -> int:
    return lib().or_qbin(float(q))


# ------------------------------------------------------------------ the PT engine
class OraclePT:
    """Configuration-swapping FP64 Parallel Tempering over S samples x R replicas x nT temperatures."""

    def __init__(self, Ns, J_list, temps, R, seed, cc=2.0, swap_every=64, measure_every=16, resync_every=64,
                 graphs=None):
        """graphs: None for the comb graph of every sample, else one [n_s, 4] quadruplet list (term order)
        per sample, with len(J_list[s]) == n_s."""
        L = lib()
        self.Ns = np.ascontiguousarray(Ns, dtype=np.int32)
        self.S = len(self.Ns); self.R = int(R); self.temps = np.ascontiguousarray(temps, dtype=np.float64)
        self.nT = len(self.temps)
        self.J = np.ascontiguousarray(np.concatenate([np.asarray(j, dtype=np.float64) for j in J_list])
                                      if len(J_list) else np.zeros(0))
        self.J_off = np.zeros(self.S + 1, dtype=np.int64)
        self.J_off[1:] = np.cumsum([len(j) for j in J_list])
        if graphs is None:
            self._h = L.or_pt_create(self.S, _p(self.Ns), _p(self.J), _p(self.J_off), self.nT, _p(self.temps),
                                     self.R, int(seed), float(cc), int(swap_every), int(measure_every),
                                     int(resync_every))
        else:
            gq = [np.asarray(g, dtype=np.int32).reshape(-1, 4) for g in graphs]
            assert [len(g) for g in gq] == [len(j) for j in J_list], "one coupling per quadruplet"
            self.graph = np.ascontiguousarray(np.concatenate(gq) if gq else np.zeros((0, 4), np.int32))
            self._h = L.or_pt_create_graph(self.S, _p(self.Ns), _p(self.graph), _p(self.J), _p(self.J_off), self.nT,
                                           _p(self.temps), self.R, int(seed), float(cc), int(swap_every),
                                           int(measure_every), int(resync_every))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_pt_destroy(h)
            self._h = None

    def sweep(self, n):
        lib().or_pt_sweep(self._h, int(n))

    def swap(self):
        lib().or_pt_swap(self._h)

    def resync(self):
        lib().or_pt_resync(self._h)

    def measure_now(self):
        lib().or_pt_measure_now(self._h)

    @property
    def sweeps_done(self):
        return lib().or_pt_sweeps_done(self._h)

    def state(self):
        """(list of complex arrays per (s, r, t) in canonical order, energies)."""
        tot = int(sum(int(n) for n in self.Ns)) * self.R * self.nT
        a = np.zeros(tot, dtype=np.complex128)
        E = np.zeros(self.S * self.R * self.nT)
        lib().or_pt_get_state(self._h, _p(a), _p(E))
        return a, E

    def set_state(self, a):
        a = np.ascontiguousarray(a, dtype=np.complex128)
        lib().or_pt_set_state(self._h, _p(a))

    def observables(self):
        ST = self.S * self.nT
        npair = self.S * self.R * max(self.nT - 1, 1)
        stat = np.zeros((self.S, self.nT, NSTAT)); qstat = np.zeros((self.S, self.nT, NQSTAT))
        qhist = np.zeros((self.S, self.nT, NBINS), dtype=np.uint64)
        sacc = np.zeros((self.S, self.R, max(self.nT - 1, 1)), dtype=np.uint64); satt = np.zeros_like(sacc)
        macc = np.zeros((self.S, self.nT), dtype=np.uint64); matt = np.zeros_like(macc)
        assert stat.size == ST * NSTAT and sacc.size == npair
        lib().or_pt_get_observables(self._h, _p(stat), _p(qstat), _p(qhist), _p(sacc), _p(satt), _p(macc), _p(matt))
        return dict(stat=stat, qstat=qstat, qhist=qhist, swap_acc=sacc, swap_att=satt, mc_acc=macc, mc_att=matt)

    def reset_observables(self):
        lib().or_pt_reset_observables(self._h)
