"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded inputs.

Tolerances.  FP64 kernels: 1e-12 relative on fields and energies (the sums differ from the oracle
only in order of summation; each field is a sum of deg ~ N^2/3 products of O(1) magnitude), and
trajectories agree to 1e-9 (identical Philox streams, rounding only).  FP32 kernels: 1e-5 relative
to the magnitude of the quantity (fields are FP32 sums of up to ~2e4 terms with relative rounding
~6e-8 per term, growing like sqrt(terms)).
"""
import numpy as np
import pytest

import oracle
import paper_2511_13508_gb300 as pkg
from paper_2511_13508_gb300 import workload

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-12
TOL_F32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()


def couplings(Ns, seed0=1000):
    return [workload.couplings(N, len(oracle.enumerate_quads(N)), seed0 + s) for s, N in enumerate(Ns)]


def rand_states(Ns, R, nT, rng):
    out = []
    for N in Ns:
        for _ in range(R * nT):
            g = rng.standard_normal(N)
            u = np.sqrt(N) * np.abs(g) / np.linalg.norm(g)
            out.append(np.sqrt(u) * np.exp(1j * rng.uniform(0, 2 * np.pi, N)))
    return np.concatenate(out)


def split(a, Ns, R, nT):
    res, p = [], 0
    for N in Ns:
        for _ in range(R * nT):
            res.append(a[p:p + N]); p += N
    return res


# ------------------------------------------------------------------------------------------- init / energy
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-7)])
def test_initial_state_matches_oracle(prec, tol):
    Ns, R, temps = [16, 16], 2, workload.geometric_ladder(0.4, 1.6, 4)
    Js = couplings(Ns)
    ref = oracle.OraclePT(Ns, Js, temps, R, 99)
    pt = pkg.PT(Ns, Js, temps, R, 99, precision=prec)
    a0, E0 = ref.state()
    a1, E1 = pt.state()
    assert np.abs(a1 - a0).max() < tol * 4
    assert np.allclose(E1, E0, rtol=1e-12 if prec == "fp64" else 1e-5, atol=1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp64_plain"])
@pytest.mark.parametrize("Ns", [[4], [6, 8], [16], [24, 40], [64], [130]])
def test_energy_matches_oracle(prec, Ns):
    rng = np.random.default_rng(sum(Ns))
    R, nT = 2, 3
    temps = workload.geometric_ladder(0.5, 1.5, nT)
    Js = couplings(Ns)
    pt = pkg.PT(Ns, Js, temps, R, 5, precision=prec)
    a = rand_states(Ns, R, nT, rng)
    pt.set_state(a)
    E = pt.energy()
    _, Es = pt.state()
    assert np.array_equal(E, Es)
    tol = TOL_F32 if prec == "fp32" else TOL_F64
    for c, x in enumerate(split(a, Ns, R, nT)):
        s = c // (R * nT)
        N = Ns[s]
        if prec == "fp32":
            x = x.astype(np.complex64).astype(np.complex128)
        ref = oracle.energy(N, oracle.enumerate_quads(N), Js[s], x)
        scale = np.sqrt((Js[s] ** 2).sum()) * 4 + abs(ref)
        assert abs(E[c] - ref) <= tol * scale, (c, E[c], ref)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 1e-7)])
def test_resync_energy_is_exact_and_split_independent(prec, tol):
    """The resync spreads a group's blocks over several thread blocks (how many depends on the group count)
    and adds their partial sums in a fixed order: a repeated resync returns bit-identical energies, contexts
    whose groups (and so splits) differ agree to rounding, and both agree with the oracle's H of the same
    state (N = 256, the bench's size; an item dropped or counted twice by the split would be off by O(1))."""
    Ns, R, nT = [256, 256, 256], 2, 8
    temps = workload.geometric_ladder(0.3, 1.6, nT)
    Js = couplings(Ns, 2100)
    rng = np.random.default_rng(77)
    a = rand_states(Ns, R, nT, rng)
    shapes = (8, 16)  # (32 chains per block do not fit next to an N = 256 table)
    Es = []
    for cpb in shapes:
        pt = pkg.PT(Ns, Js, temps, R, 5, precision=prec, chains_per_block=cpb, swap_every=0, measure_every=0,
                    resync_every=0)
        pt.set_state(a)
        E1 = pt.energy()
        E2 = pt.energy()
        assert np.array_equal(E1, E2)
        Es.append(E1)
        pt.close()
    ref_scale = np.abs(Es[0]).max() + 1.0
    for E in Es[1:]:
        assert np.abs(E - Es[0]).max() <= tol * ref_scale
    quads = oracle.enumerate_quads(256)
    for c, x in enumerate(split(a, Ns, R, nT)):
        if c % 7:
            continue
        s = c // (R * nT)
        if prec == "fp32":
            x = x.astype(np.complex64).astype(np.complex128)
        ref = oracle.energy(256, quads, Js[s], x)
        scale = np.sqrt((Js[s] ** 2).sum()) * 4 + abs(ref)
        assert abs(Es[0][c] - ref) <= (TOL_F32 if prec == "fp32" else TOL_F64) * scale, (c, Es[0][c], ref)


# ------------------------------------------------------------------------------------------- local fields
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("N", [4, 10, 16, 34, 64, 128])
def test_fields_and_delta_h_match_oracle(prec, N):
    rng = np.random.default_rng(N)
    R, nT = 2, 5  # 10 chains: partial groups for every chains_per_block
    temps = workload.geometric_ladder(0.5, 1.5, nT)
    Js = couplings([N])
    q = oracle.enumerate_quads(N)
    pt = pkg.PT([N], Js, temps, R, 3, precision=prec)
    a = rand_states([N], R, nT, rng)
    pt.set_state(a)
    chains = split(a, [N], R, nT)
    if prec == "fp32":
        chains = [x.astype(np.complex64).astype(np.complex128) for x in chains]
    tol = TOL_F32 if prec == "fp32" else TOL_F64
    pairs = [(0, N - 1), (N - 1, 0), (1, 2), (N // 2, N // 2 - 1)] + [tuple(rng.choice(N, 2, replace=False)) for _ in range(4)]
    for j, k in pairs:
        f = pt.fields(0, j, k)
        for c, x in enumerate(chains):
            hj, hk = oracle.field(N, q, Js[0], x, j), oracle.field(N, q, Js[0], x, k)
            scale = np.sqrt(len(q)) / N + abs(hj) + abs(hk)
            assert abs(f[c, 0] - hj) <= tol * scale and abs(f[c, 1] - hk) <= tol * scale, (j, k, c)
            # Delta H from the four GPU sums against the oracle's pair-move energy change
            aj, ak = complex(*rng.standard_normal(2)), complex(*rng.standard_normal(2))
            dj, dk = aj - x[j], ak - x[k]
            dH = -2 * (np.conj(dj) * f[c, 0] + np.conj(dk) * f[c, 1] + np.conj(dj) * dk * f[c, 2]
                       + np.conj(dj) * np.conj(dk) * f[c, 3]).real
            ref = oracle.delta_h(N, q, Js[0], x, j, k, aj, ak)
            assert abs(dH - ref) <= tol * (abs(ref) + scale * 4), (j, k, c, dH, ref)


# ------------------------------------------------------------------------------------------- trajectories
@pytest.mark.parametrize("prec", ["fp64", "fp64_plain"])
@pytest.mark.parametrize("Ns,R,nT,sweeps", [([16, 16], 2, 4, 48), ([4], 3, 3, 64), ([8, 12, 16], 2, 5, 40),
                                            ([64], 2, 3, 8)])
def test_fp64_trajectory_matches_oracle(prec, Ns, R, nT, sweeps):
    """Same seeds and Philox counters: the FP64 GPU paths follow the oracle's Markov chain (moves, pair
    sequence, swaps with label exchange, resync) and accumulate the same observables."""
    temps = workload.geometric_ladder(0.3, 1.6, nT)
    Js = couplings(Ns)
    kw = dict(swap_every=8, measure_every=4, resync_every=16)
    ref = oracle.OraclePT(Ns, Js, temps, R, 2024, **kw)
    ref.sweep(sweeps)
    pt = pkg.PT(Ns, Js, temps, R, 2024, precision=prec, **kw)
    pt.sweep(sweeps // 2)
    pt.sweep(sweeps - sweeps // 2)
    a0, E0 = ref.state()
    a1, E1 = pt.state()
    assert np.abs(a1 - a0).max() < 1e-9
    assert np.allclose(E1, E0, rtol=1e-9, atol=1e-11)
    o0, o1 = ref.observables(), pt.observables()
    for key in ("qhist", "swap_acc", "swap_att", "mc_acc", "mc_att"):
        assert np.array_equal(o0[key], o1[key]), key
    assert np.allclose(o0["stat"], o1["stat"], rtol=1e-9, atol=1e-10)
    assert np.allclose(o0["qstat"], o1["qstat"], rtol=1e-9, atol=1e-10)
    assert pt.counters == (sweeps, sweeps // 8)


def test_fp32_short_trajectory_tracks_oracle():
    """FP32 fields: over a few sweeps almost every Metropolis decision equals the FP64 oracle's."""
    Ns, R, nT = [32, 32], 2, 4
    temps = workload.geometric_ladder(0.3, 1.6, nT)
    Js = couplings(Ns)
    kw = dict(swap_every=0, measure_every=0, resync_every=0)
    ref = oracle.OraclePT(Ns, Js, temps, R, 11, **kw)
    pt = pkg.PT(Ns, Js, temps, R, 11, precision="fp32", **kw)
    ref.sweep(2)
    pt.sweep(2)
    a0, _ = ref.state()
    a1, _ = pt.state()
    close = [np.abs(x - y).max() < 1e-4 for x, y in zip(split(a0, Ns, R, nT), split(a1, Ns, R, nT))]
    assert np.mean(close) > 0.9


# ------------------------------------------------------------------------------------------- robustness
def test_checkpoint_resume_is_bit_identical():
    Ns, R, nT = [32, 48], 2, 6
    temps = workload.geometric_ladder(0.3, 1.6, nT)
    Js = couplings(Ns)
    kw = dict(swap_every=8, measure_every=4, resync_every=16, precision="fp32")
    a = pkg.PT(Ns, Js, temps, R, 5, **kw)
    a.sweep(40)
    blob = a.save()
    a.sweep(40)
    b = pkg.PT(Ns, Js, temps, R, 5, **kw)
    b.load(blob)
    b.sweep(40)
    sa, Ea = a.state()
    sb, Eb = b.state()
    assert np.array_equal(sa, sb) and np.array_equal(Ea, Eb)
    oa, ob = a.observables(), b.observables()
    for k in oa:
        assert np.array_equal(oa[k], ob[k]), k
    bad = bytearray(blob); bad[100] ^= 1
    with pytest.raises(pkg.PTError) as e:
        b.load(bytes(bad))
    assert e.value.code == -6
    c = pkg.PT(Ns, Js, temps, R, 6, **kw)  # other seed -> other context
    with pytest.raises(pkg.PTError):
        c.load(blob)


def test_graphs_and_direct_launches_agree():
    Ns, R, nT = [64], 2, 8
    temps = workload.geometric_ladder(0.3, 1.6, nT)
    Js = couplings(Ns)
    res = []
    for g in (True, False):
        pt = pkg.PT(Ns, Js, temps, R, 8, precision="fp32", use_graphs=g)
        pt.sweep(70)
        res.append(pt.state())
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


@pytest.mark.parametrize("cpb", [8, 16, 32])
def test_chains_per_block_variants_agree_fp32(cpb):
    """Every thread-block shape runs the same Markov chain (the J-sharing kernel is shape-agnostic up to
    FP32 summation order): compare the first sweep's accept decisions through the state."""
    Ns, R, nT = [48], 2, 9
    temps = workload.geometric_ladder(0.3, 1.6, nT)
    Js = couplings(Ns)
    kw = dict(swap_every=0, measure_every=0, resync_every=0)
    ref = oracle.OraclePT(Ns, Js, temps, R, 4, **kw)
    ref.sweep(1)
    pt = pkg.PT(Ns, Js, temps, R, 4, precision="fp32", chains_per_block=cpb, **kw)
    pt.sweep(1)
    a0, _ = ref.state()
    a1, _ = pt.state()
    close = [np.abs(x - y).max() < 1e-4 for x, y in zip(split(a0, Ns, R, nT), split(a1, Ns, R, nT))]
    assert np.mean(close) > 0.9


def test_degenerate_shapes():
    """nT = 1 (no swaps), R = 1 (no overlaps), N = 4 (one quadruplet)."""
    Js = couplings([4, 8])
    pt = pkg.PT([4, 8], Js, [0.7], 1, 1, precision="fp64", swap_every=4, measure_every=2, resync_every=4)
    pt.sweep(16)
    o = pt.observables()
    assert o["qstat"][..., 0].sum() == 0 and o["stat"][..., 0].sum() == 2 * 8
    ref = oracle.OraclePT([4, 8], Js, [0.7], 1, 1, swap_every=4, measure_every=2, resync_every=4)
    ref.sweep(16)
    assert np.abs(pt.state()[0] - ref.state()[0]).max() < 1e-10


def test_zero_sweeps_and_errors():
    Js = couplings([16])
    pt = pkg.PT([16], Js, [0.5, 1.0], 2, 1)
    pt.sweep(0)
    with pytest.raises(pkg.PTError):
        pt.sweep(-1)
    with pytest.raises(pkg.PTError):
        pt.fields(0, 3, 3)
    with pytest.raises(pkg.PTError):
        pt.fields(1, 0, 1)
    a, _ = pt.state()
    a[5] = np.nan
    with pytest.raises(pkg.PTError) as e:
        pt.set_state(a)
    assert e.value.code == -5


# ------------------------------------------------------------------------------------------- full size
def test_n256_bench_configuration_sampled_parity():
    """The N = 256 workload at full size (16 samples x 48 T x 2 replicas, FP32, the bench's launch shape):
    sampled fields and energies against the oracle, then a short run stays finite and on the constraint."""
    W = workload.workloads()["n256_large"]
    N = 256
    q = oracle.enumerate_quads(N)
    Js = [workload.couplings(N, len(q), s) for s in W.seeds]
    pt = pkg.PT(W.Ns, Js, W.temps, W.replicas, 1, precision="fp32")
    a, E = pt.state()
    chains = split(a, W.Ns, W.replicas, W.n_temps)
    rng = np.random.default_rng(0)
    for s in (0, 7, 15):
        j, k = rng.choice(N, 2, replace=False)
        f = pt.fields(s, j, k)
        for c in (0, 47, 95):
            x = chains[s * 96 + c]
            hj = oracle.field(N, q, Js[s], x, j)
            scale = np.sqrt(len(q)) / N + abs(hj)
            assert abs(f[c, 0] - hj) <= TOL_F32 * scale
            Er = oracle.energy(N, q, Js[s], x)
            assert abs(E[s * 96 + c] - Er) <= TOL_F32 * (abs(Er) + 1)
    pt.sweep(2)
    a2, E2 = pt.state()
    assert np.isfinite(a2).all() and np.isfinite(E2).all()
    quart = np.array([(np.abs(x) ** 4).sum() for x in split(a2, W.Ns, W.replicas, W.n_temps)])
    assert np.abs(quart - N).max() < 1e-3 * N
    Ef = pt.energy()
    assert np.abs(Ef - E2).max() < 1e-3 * (np.abs(Ef).max() + 1)
