"""Host-side checks of the C ABI that need no GPU: the library builds for sm_103a, loads, exports
every symbol include/pt.h declares, enumerates the canonical quadruplets exactly like the oracle and
rejects bad arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2511_13508_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    pkg.build()
    return pkg.lib()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "pt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pt_[a-z_0-9]+)\s*\(", txt)) - {"pt_alloc_fn", "pt_free_fn"})


def test_exports_every_declared_symbol(L):
    syms = declared_symbols()
    assert "pt_create" in syms and "pt_sweep" in syms and len(syms) >= 15
    for s in syms:
        assert hasattr(L, s), s
    assert set(pkg.EXPORTS) <= set(syms)


@pytest.mark.parametrize("N", [4, 5, 6, 9, 16, 33, 64])
def test_enumeration_matches_oracle(L, N):
    assert np.array_equal(pkg.enumerate_quads(N), oracle.enumerate_quads(N))


def test_enumeration_counts_large(L):
    n = ctypes.c_int64()
    for N, ref in ((128, 168672), (256, 1373632)):
        assert L.pt_enumerate_quads(N, None, ctypes.byref(n)) == 0 and n.value == ref == len(oracle.enumerate_quads(N))
    assert L.pt_enumerate_quads(3, None, ctypes.byref(n)) == -1
    assert L.pt_enumerate_quads(513, None, ctypes.byref(n)) == -1


def test_config_defaults(L):
    c = pkg.Config()
    L.pt_config_default(ctypes.byref(c))
    assert (c.precision, c.cc_factor, c.swap_every, c.measure_every, c.resync_every, c.use_graphs) == (0, 2.0, 64, 16, 64, 1)


def _create(L, Ns, J, off, temps, R=2, cfg=None):
    h = ctypes.c_void_p()
    Ns = np.ascontiguousarray(Ns, np.int32); J = np.ascontiguousarray(J, np.float64)
    off = np.ascontiguousarray(off, np.int64); temps = np.ascontiguousarray(temps, np.float64)
    rc = L.pt_create(ctypes.byref(h), cfg, len(Ns), Ns.ctypes.data, J.ctypes.data, off.ctypes.data, len(temps),
                     temps.ctypes.data, R, 1, pkg.ALLOC_FN(), pkg.FREE_FN(), None, None)
    return rc, h, L.pt_last_error(None).decode()


def test_create_rejects_bad_arguments_before_device_work(L):
    J = np.zeros(252); off = [0, 252]
    assert _create(L, [15], J, off, [1.0])[0] == -1                 # odd N
    assert _create(L, [16], J, [0, 251], [1.0])[0] == -1            # wrong J length
    assert _create(L, [16], J, off, [1.0, 0.5])[0] == -1            # not ascending
    assert _create(L, [16], J, off, [-1.0])[0] == -1                # non-positive T
    assert _create(L, [16], J, off, [1.0], R=0)[0] == -1            # replicas
    Jn = J.copy(); Jn[7] = np.nan
    rc, h, msg = _create(L, [16], Jn, off, [1.0])
    assert rc == -5 and "non-finite" in msg
    assert L.pt_destroy(None) == 0


@pytest.mark.parametrize("prec,max_n,S,chains,sms,expect", [
    ("fp32", 256, 16, 96, 152, (8, 11)),    # the bench workload: 8 chains from N = 160 on
    ("fp32", 192, 32, 64, 152, (8, 11)),
    ("fp32", 128, 96, 48, 152, (16, 11)),   # the ragged batch (largest N 128): at most 16 chains from N = 96
    ("fp32", 96, 64, 64, 152, (16, 11)),
    ("fp32", 96, 2, 16, 152, (16, 11)),     # too few groups for any size: 16 chains from N = 96
    ("fp32", 64, 64, 64, 152, (32, 11)),    # the batched N = 64 workload: 128 groups of 32 >= 0.8 x 152
    ("fp32", 64, 16, 64, 152, (8, 11)),     # 16 samples: only groups of 8 give enough of them
    ("fp32", 64, 2, 64, 152, (32, 11)),     # none does: 32 chains
    ("fp32", 64, 64, 64, 0, (32, 11)),      # SM count unknown
    ("fp32", 48, 64, 64, 152, (32, 11)),
    ("fp32", 32, 8, 16, 152, (16, 7)),      # below N = 48: 16 x 7
    ("fp32", 16, 4, 8, 152, (8, 7)),        # at most 8 chains per sample: 8 per block
    ("fp64", 64, 64, 64, 152, (16, 3)),
    ("fp64", 128, 8, 16, 152, (8, 7)),
])
def test_default_shape_rule(L, prec, max_n, S, chains, sms, expect):
    assert pkg.default_shape(prec, max_n, S, chains, sms) == expect


def test_default_shape_rejects_bad_arguments(L):
    G, ncw = ctypes.c_int(), ctypes.c_int()
    for args in [(2, 64, 1, 1, 152), (0, 65, 1, 1, 152), (0, 2, 1, 1, 152), (0, 514, 1, 1, 152), (0, 64, 0, 1, 152),
                 (0, 64, 1, 0, 152), (0, 64, 1, 1, -1)]:
        assert L.pt_default_shape(*args, ctypes.byref(G), ctypes.byref(ncw)) == -1, args
    assert L.pt_default_shape(0, 64, 1, 1, 152, None, ctypes.byref(ncw)) == -1
