"""GB300 (sm_103a) Parallel-Tempering engine for the smoothed-cubic 4-body random-laser model
(arXiv 2511.13508).

Thin ctypes binding over the C ABI of ``libptgb.so`` (declared in ``include/pt.h``): argument
marshalling only; every step of the Monte Carlo path runs in the library's CUDA kernels.  PyTorch
supplies device memory (its caching allocator, through the ABI's allocator callbacks) and the
stream.  There is no CPU fallback: without the compiled library the import of the engine fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

__all__ = ["build", "lib", "PT", "enumerate_quads", "fma_probe", "fmc_graph", "PREC", "PTError", "NSTAT", "NQSTAT", "QBINS", "TRACE_REC"]

PREC = {"fp32": 0, "fp64": 1, "fp64_plain": 2}
NSTAT, NQSTAT, QBINS = 7, 5, 201
TRACE_REC = 20  # doubles per chain of pt_trace_update
_ERRORS = {-1: "PT_EINVAL", -2: "PT_ENOMEM", -3: "PT_ECUDA", -4: "PT_ETIMEOUT", -5: "PT_ENAN",
           -6: "PT_ESTATE", -7: "PT_EUNSUPPORTED"}


class PTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_ERRORS.get(code, "PT_E?"), code, msg))
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("cc_factor", ctypes.c_double), ("swap_every", ctypes.c_int),
                ("measure_every", ctypes.c_int), ("resync_every", ctypes.c_int),
                ("chains_per_block", ctypes.c_int), ("sweeps_per_unit", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("consumer_warps", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("watchdog_ms", ctypes.c_int)]


class Observables(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("stat", "qstat", "qhist", "swap_acc", "swap_att", "mc_acc", "mc_att",
                                               "gm_acc", "gm_att")]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

EXPORTS = ["pt_config_default", "pt_enumerate_quads", "pt_create", "pt_sweep", "pt_swap", "pt_resync",
           "pt_measure_now", "pt_measure", "pt_reset_observables", "pt_get_state", "pt_set_state", "pt_energy",
           "pt_fields", "pt_trace_update", "pt_save", "pt_load", "pt_autotune", "pt_counters", "pt_sync", "pt_destroy",
           "pt_last_error", "pt_learn_init", "pt_collect", "pt_train", "pt_global_move", "pt_set_global_every",
           "pt_learn_params", "pt_learn_shape", "pt_learn_eval", "pt_set_global_blocks", "pt_set_global_sampler", "pt_gemm_bf16",
           "pt_energy_fp64_static", "pt_fma_probe", "pt_fmc_graph", "pt_create_graph", "pt_check_wait",
           "pt_graph_records", "pt_default_shape"]

_lib = None


def build(force: bool = False) -> str:
    """Compiles libptgb.so for sm_103a (in-tree) if missing or stale."""
    return _build.build(force=force)


def lib() -> ctypes.CDLL:
    """Loads libptgb.so; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise ImportError("libptgb.so is not built: run paper_2511_13508_gb300.build() (needs nvcc)")
        L = ctypes.CDLL(_build.LIB)
        vp, i, i64, u64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        L.pt_config_default.argtypes = [ctypes.POINTER(Config)]; L.pt_config_default.restype = None
        L.pt_enumerate_quads.argtypes = [i, vp, ctypes.POINTER(i64)]
        L.pt_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Config), i, vp, vp, vp, i, vp, i, u64,
                                ALLOC_FN, FREE_FN, vp, vp]
        L.pt_create_graph.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Config), i, vp, vp, vp, vp, i, vp, i, u64,
                                      ALLOC_FN, FREE_FN, vp, vp]
        L.pt_fmc_graph.argtypes = [i, vp, d, vp, ctypes.POINTER(i64)]
        L.pt_check_wait.argtypes = [vp, i]
        L.pt_sweep.argtypes = [vp, i64]
        for n in ("pt_swap", "pt_resync", "pt_measure_now", "pt_reset_observables", "pt_sync", "pt_destroy"):
            getattr(L, n).argtypes = [vp]
        L.pt_measure.argtypes = [vp, ctypes.POINTER(Observables)]
        L.pt_get_state.argtypes = [vp, vp, vp]
        L.pt_set_state.argtypes = [vp, vp]
        L.pt_energy.argtypes = [vp, vp]
        L.pt_fields.argtypes = [vp, i, i, i, vp]
        L.pt_trace_update.argtypes = [vp, i, vp, vp]
        L.pt_save.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t)]
        L.pt_load.argtypes = [vp, vp, ctypes.c_size_t]
        L.pt_counters.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.pt_autotune.argtypes = [vp, i, vp]
        L.pt_default_shape.argtypes = [i, i, i, i, i, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.pt_learn_init.argtypes = [vp, i, i, i, u64]
        L.pt_collect.argtypes = [vp, i64, i]
        L.pt_train.argtypes = [vp, i, d, vp]
        L.pt_global_move.argtypes = [vp]
        L.pt_set_global_every.argtypes = [vp, i]
        L.pt_set_global_blocks.argtypes = [vp, i, i]
        L.pt_set_global_sampler.argtypes = [vp, i]
        L.pt_learn_params.argtypes = [vp, vp, i]
        L.pt_learn_shape.argtypes = [vp, vp]
        L.pt_learn_eval.argtypes = [vp, vp, vp, i, vp, vp, vp]
        L.pt_gemm_bf16.argtypes = [i, i, i, i, vp, vp, vp, vp]
        L.pt_energy_fp64_static.argtypes = [i, i, vp, vp, vp, d, vp]
        L.pt_fma_probe.argtypes = [i, i, i, i, vp, vp]
        L.pt_graph_records.argtypes = [i, i64, vp, vp, vp, vp, vp]
        L.pt_last_error.argtypes = [vp]; L.pt_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _p(x: np.ndarray):
    return x.ctypes.data_as(ctypes.c_void_p)


def fmc_graph(omega, gamma=None) -> np.ndarray:
    """Random-frequency mode-locked graph (pt_fmc_graph): [n, 4] int32 quadruplets in term order.
    omega: strictly ascending frequencies; gamma defaults to 1/(2(N-1))."""
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    N = len(omega)
    g = 1.0 / (2 * (N - 1)) if gamma is None else float(gamma)
    n = ctypes.c_int64()
    _check(None, lib().pt_fmc_graph(N, _p(omega), g, None, ctypes.byref(n)))
    out = np.zeros((max(n.value, 1), 4), dtype=np.int32)
    _check(None, lib().pt_fmc_graph(N, _p(omega), g, _p(out), ctypes.byref(n)))
    return out[: n.value]


def fma_probe(packed, blocks, threads, iters, sink_ptr, stream_ptr):
    """Launches the FP32 FMA-pipe probe (pt_fma_probe): blocks * threads * iters * 32 flops on the stream."""
    _check(None, lib().pt_fma_probe(int(packed), int(blocks), int(threads), int(iters), sink_ptr, stream_ptr))


def default_shape(precision, max_n, n_samples, chains_per_sample, sm_count):
    """Sweep-block shape pt_create picks by default (pt_default_shape, host only):
    (chains_per_block, consumer_warps)."""
    G, ncw = ctypes.c_int(), ctypes.c_int()
    prec = PREC[precision] if isinstance(precision, str) else int(precision)
    _check(None, lib().pt_default_shape(prec, int(max_n), int(n_samples), int(chains_per_sample), int(sm_count),
                                        ctypes.byref(G), ctypes.byref(ncw)))
    return G.value, ncw.value


def graph_records(N, quads, J):
    """Incidence records of the FP32 quadruplet-list kernels (pt_graph_records): (offsets [N+1], rec [4 nq, 4]
    int32 (A, B, C, w), recJ [4 nq] float32)."""
    quads = np.ascontiguousarray(quads, np.int32).reshape(-1, 4)
    J = np.ascontiguousarray(J, np.float64)
    nq = len(quads)
    off = np.zeros(int(N) + 1, np.int32)
    rec = np.zeros((max(4 * nq, 1), 4), np.int32)
    recJ = np.zeros(max(4 * nq, 1), np.float32)
    _check(None, lib().pt_graph_records(int(N), nq, _p(quads), _p(J), _p(off), _p(rec), _p(recJ)))
    return off, rec[: 4 * nq], recJ[: 4 * nq]


def enumerate_quads(N: int) -> np.ndarray:
    """Canonical quadruplets (a<b<c<d, a+d=b+c) of the N-mode comb, shape [|Q|, 4]."""
    n = ctypes.c_int64()
    _check(None, lib().pt_enumerate_quads(int(N), None, ctypes.byref(n)))
    out = np.zeros((max(n.value, 1), 4), dtype=np.int32)
    _check(None, lib().pt_enumerate_quads(int(N), _p(out), ctypes.byref(n)))
    return out[: n.value]


def _check(h, rc):
    if rc != 0:
        raise PTError(rc, (lib().pt_last_error(h) or b"").decode())


class _TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator."""

    def __init__(self, stream):
        import torch
        self.torch, self.stream, self.dev = torch, stream, torch.cuda.current_device()

        def _alloc(nbytes, user):
            try:
                return int(self.torch.cuda.caching_allocator_alloc(int(nbytes), self.dev, self.stream))
            except Exception:
                return None

        def _free(ptr, user):
            self.torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc, self.free = ALLOC_FN(_alloc), FREE_FN(_free)


class PT:
    """One Parallel-Tempering ensemble: S disorder samples x R replicas x n_T temperatures."""

    def __init__(self, Ns, J_list, temps, replicas, seed, precision="fp32", cc=2.0, swap_every=64,
                 measure_every=16, resync_every=64, chains_per_block=0, sweeps_per_unit=0, blocks_per_sm=0,
                 consumer_warps=0, use_graphs=True, watchdog_ms=600000, stream=None, torch_memory=True, graphs=None):
        """graphs: None for the comb graph of every sample; else one [n_s, 4] quadruplet list per sample
        (term order, e.g. from fmc_graph) with len(J_list[s]) == n_s, on the fp32 or fp64_plain path."""
        L = lib()
        self.Ns = np.ascontiguousarray(Ns, dtype=np.int32)
        self.S, self.R = len(self.Ns), int(replicas)
        self.temps = np.ascontiguousarray(temps, dtype=np.float64)
        self.nT = len(self.temps)
        self.precision = precision
        J = np.ascontiguousarray(np.concatenate([np.asarray(j, np.float64) for j in J_list]))
        off = np.zeros(self.S + 1, np.int64)
        off[1:] = np.cumsum([len(j) for j in J_list])
        cfg = Config()
        L.pt_config_default(ctypes.byref(cfg))
        cfg.precision = PREC[precision]; cfg.cc_factor = cc; cfg.swap_every = swap_every
        cfg.measure_every = measure_every; cfg.resync_every = resync_every
        cfg.chains_per_block = chains_per_block; cfg.sweeps_per_unit = sweeps_per_unit
        cfg.blocks_per_sm = blocks_per_sm; cfg.consumer_warps = consumer_warps; cfg.use_graphs = int(bool(use_graphs)); cfg.watchdog_ms = watchdog_ms
        self._alloc = None
        s_ptr = None
        if stream is not None:
            s_ptr = int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)
        if torch_memory:
            import torch
            if torch.cuda.is_available():
                if s_ptr is None or s_ptr == 0:
                    # a stream of our own (the legacy default stream cannot be captured into graphs)
                    self._stream = torch.cuda.Stream()
                    s_ptr = int(self._stream.cuda_stream)
                self._alloc = _TorchAllocator(s_ptr)
        h = ctypes.c_void_p()
        af = self._alloc.alloc if self._alloc else ALLOC_FN()
        ff = self._alloc.free if self._alloc else FREE_FN()
        if graphs is None:
            rc = L.pt_create(ctypes.byref(h), ctypes.byref(cfg), self.S, _p(self.Ns), _p(J), _p(off), self.nT,
                             _p(self.temps), self.R, ctypes.c_uint64(int(seed)), af, ff, None, s_ptr)
        else:
            gq = [np.asarray(g, dtype=np.int32).reshape(-1, 4) for g in graphs]
            if [len(g) for g in gq] != [len(j) for j in J_list]:
                raise ValueError("one coupling per quadruplet")
            Q = np.ascontiguousarray(np.concatenate(gq) if gq else np.zeros((0, 4), np.int32))
            rc = L.pt_create_graph(ctypes.byref(h), ctypes.byref(cfg), self.S, _p(self.Ns), _p(Q), _p(J), _p(off),
                                   self.nT, _p(self.temps), self.R, ctypes.c_uint64(int(seed)), af, ff, None, s_ptr)
        _check(None, rc)
        self._h = h
        self.n_chains = self.S * self.R * self.nT

    # -------------------------------------------------------------------------------------------
    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().pt_destroy(h)
            self._h = None

    __del__ = close

    def _c(self, rc):
        _check(self._h, rc)

    def sweep(self, n):
        self._c(lib().pt_sweep(self._h, int(n)))

    def swap(self):
        self._c(lib().pt_swap(self._h))

    def resync(self):
        self._c(lib().pt_resync(self._h))

    def measure_now(self):
        self._c(lib().pt_measure_now(self._h))

    def sync(self):
        self._c(lib().pt_sync(self._h))

    def reset_observables(self):
        self._c(lib().pt_reset_observables(self._h))

    def observables(self) -> dict:
        S, R, nT = self.S, self.R, self.nT
        np1 = max(nT - 1, 1)
        o = dict(stat=np.zeros((S, nT, NSTAT)), qstat=np.zeros((S, nT, NQSTAT)),
                 qhist=np.zeros((S, nT, QBINS), np.uint64), swap_acc=np.zeros((S, R, np1), np.uint64),
                 swap_att=np.zeros((S, R, np1), np.uint64), mc_acc=np.zeros((S, nT), np.uint64),
                 mc_att=np.zeros((S, nT), np.uint64), gm_acc=np.zeros((S, nT), np.uint64),
                 gm_att=np.zeros((S, nT), np.uint64))
        ob = Observables(*[o[k].ctypes.data for k in ("stat", "qstat", "qhist", "swap_acc", "swap_att", "mc_acc",
                                                      "mc_att", "gm_acc", "gm_att")])
        self._c(lib().pt_measure(self._h, ctypes.byref(ob)))
        return o

    def state(self):
        """(amplitudes: complex128 [sum_s N_s R nT] in canonical (s, r, t) order, energies [S R nT])."""
        tot = int(self.Ns.astype(np.int64).sum()) * self.R * self.nT
        a = np.zeros(tot, np.complex128)
        E = np.zeros(self.n_chains)
        self._c(lib().pt_get_state(self._h, _p(a), _p(E)))
        return a, E

    def set_state(self, a):
        a = np.ascontiguousarray(a, np.complex128)
        self._c(lib().pt_set_state(self._h, _p(a)))

    def energy(self):
        E = np.zeros(self.n_chains)
        self._c(lib().pt_energy(self._h, _p(E)))
        return E

    def fields(self, sample, j, k):
        """[R*nT, 4] complex: h_j, h_k, B_jk, A_jk for every chain of the sample, canonical (r, t) order."""
        out = np.zeros(self.R * self.nT * 8)
        self._c(lib().pt_fields(self._h, int(sample), int(j), int(k), _p(out)))
        return out.view(np.complex128).reshape(self.R * self.nT, 4)

    def trace_update(self, update):
        """Runs the next sweep with pair update `update` of the sweep kernel traced (pt_trace_update).
        Returns (rec [n_chains, TRACE_REC] float64, state before the update [sum_s N_s R nT] complex128),
        canonical (s, r, t) order; rec[:, 19] == 1 marks the traced chains."""
        rec = np.zeros((self.n_chains, TRACE_REC))
        a = np.zeros(int(self.Ns.astype(np.int64).sum()) * self.R * self.nT, np.complex128)
        self._c(lib().pt_trace_update(self._h, int(update), _p(rec), _p(a)))
        return rec, a

    def save(self) -> bytes:
        n = ctypes.c_size_t()
        self._c(lib().pt_save(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._c(lib().pt_save(self._h, buf, ctypes.byref(n)))
        return buf.raw[: n.value]

    def load(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._c(lib().pt_load(self._h, buf, len(blob)))

    def autotune(self, trial_sweeps=8):
        """Times the supported sweep-block shapes on the live ensemble, keeps the fastest and restores
        the ensemble; returns (chains_per_block, consumer_warps, sweeps_per_unit)."""
        out = (ctypes.c_int * 3)()
        self._c(lib().pt_autotune(self._h, int(trial_sweeps), out))
        return tuple(out)

    # ------------------------------------------------------------------ learned global-move proposal
    def check_wait(self, limit_ms=200) -> int:
        """Runs the bounded-wait health check (pt_check_wait); returns its status code (PT_ETIMEOUT = -4
        when the failure detection works) without raising."""
        return int(lib().pt_check_wait(self._h, int(limit_ms)))

    def learn_init(self, n_cold=8, batch=512, data_per_sample=1 << 14, seed=0):
        self._c(lib().pt_learn_init(self._h, int(n_cold), int(batch), int(data_per_sample), ctypes.c_uint64(int(seed))))

    def learn_shape(self) -> dict:
        out = np.zeros(14, np.int64)
        self._c(lib().pt_learn_shape(self._h, _p(out)))
        keys = ("N", "H", "Din", "Dout", "ncold", "psize", "oW1", "ob1", "oC1", "oW2", "ob2", "oW3", "ob3", "ndata")
        return {k: int(v) for k, v in zip(keys, out)}

    def collect(self, every, rounds):
        self._c(lib().pt_collect(self._h, int(every), int(rounds)))

    def train(self, steps, lr=1e-3):
        losses = np.zeros(max(int(steps), 1))
        self._c(lib().pt_train(self._h, int(steps), float(lr), _p(losses)))
        return losses[: int(steps)]

    def global_move(self):
        self._c(lib().pt_global_move(self._h))

    def set_global_blocks(self, lo, hi):
        self._c(lib().pt_set_global_blocks(self._h, int(lo), int(hi)))

    def set_global_sampler(self, one_launch=True):
        """One-launch autoregressive sampling (default, <= 64 proposal rows per sample) or one launch per block;
        both draw identical proposals."""
        self._c(lib().pt_set_global_sampler(self._h, 1 if one_launch else 0))

    def running_energies(self):
        """Running FP64 energies of all chains, canonical (s, r, t) order (no recompute)."""
        E = np.zeros(self.n_chains)
        self._c(lib().pt_get_state(self._h, None, _p(E)))
        return E

    def set_global_every(self, every):
        self._c(lib().pt_set_global_every(self._h, int(every)))

    def learn_params(self) -> np.ndarray:
        sh = self.learn_shape()
        P = np.zeros((self.S, sh["psize"]), np.float32)
        self._c(lib().pt_learn_params(self._h, _p(P), 0))
        return P

    def set_learn_params(self, P):
        P = np.ascontiguousarray(P, np.float32)
        self._c(lib().pt_learn_params(self._h, _p(P), 1))

    def learn_eval(self, a, cond, grad=False):
        """a: [S, rows, N] complex; cond: [S, rows] -> (logq [S, rows], extra [S, rows], grad [S, psize] or None)."""
        a = np.ascontiguousarray(a, np.complex128)
        cond = np.ascontiguousarray(cond, np.int32)
        S, rows = cond.shape
        logq = np.zeros((S, rows)); extra = np.zeros((S, rows))
        g = np.zeros((S, self.learn_shape()["psize"]), np.float32) if grad else None
        self._c(lib().pt_learn_eval(self._h, _p(a), _p(cond), int(rows), _p(logq), _p(extra),
                                     _p(g) if grad else None))
        return logq, extra, g

    @property
    def counters(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._c(lib().pt_counters(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value
